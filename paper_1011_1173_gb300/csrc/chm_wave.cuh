// Wave-pipelined rank-k up/downdate kernel (Walder 2010, Algorithm 1, with
// the CPU/GPU panelling of Sec. 4 replaced by one device-resident launch).
//
// A rank-k modification is k waves: wave q is the rank-1 modification of the
// factor left by waves < q by column q of V (Sec. 4.1 processes columns in
// order; any dependency-respecting order gives the same factor).
//
// Per wave, with F the current factor and v the vector (sign sigma):
//   chain:  p = F^{-T} v (forward substitution), T_0 = 1, T_{i+1} = T_i + sigma p_i^2,
//           which give Algorithm 1's Compute: c_i = sqrt(T_{i+1}/T_i), s_i = p_i/sqrt(T_i);
//   sweep:  Algorithm 1's Apply in its mixed form (the V update uses the new
//           L_ij), written for u = sqrt(T_i) u_hat and S_ij = L_ij / e_i:
//           S' = S + a_i u_hat, u_hat' = u_hat - b_i S',
//           a_i = sigma p_i / e_i, b_i = p_i e_i / T_{i+1}, e_i' = e_i / c_i.
// The chain carries no square root or division; the sweep is two FMAs per
// element and vector.
//
// Work split (one launch):
//   * wave workers: one warp per wave, on a few SMs that run nothing else
//     (claimed at start-up through %smid).  Wave q walks the diagonal blocks
//     in order, forms z for the block from the sweep's carry and a 32-row dot
//     product, runs the forward substitution through the block with ratios
//     precomputed by the sweep, and publishes the block's rotation panel.
//   * sweep workers: every other warp takes tasks (wave q, column block b)
//     in ticket order t = b * nwaves + q and rotates the block's tiles with
//     wave q's panels, the update vector held in registers.  It also hands
//     the wave worker what it needs next: the carry z for the block, and the
//     ratio matrices of the next wave.
// Every wait is bounded (%globaltimer), and a task only waits on events of
// tasks with smaller tickets or on wave workers, which always run.
//
// Storage between waves of one launch: the diagonal holds true values, an
// off-diagonal L_ij is held as S_ij = L_ij / e_i; the last wave of the launch
// stores true values again.
#pragma once

#include "chm_device.cuh"

namespace chm {

constexpr int kMaxSm = 1024;
constexpr int kTracePoints = 16;
constexpr int kRoleSweep = 1, kRoleDiag = 2;

// Sweep coefficients of one row of one wave, in the Apply type T.
template <typename T>
struct CoefRow {
    T a, b, e1, pad;
};

// Row data of one wave (double): new row scale and its inverse, new
// diagonal and its inverse.  The "wave -1" entries (chain0) hold the
// original factor's data: {1, 1, L_ii, 1 / L_ii}.
struct ChainRow {
    double e1, ie1, d1, id1;
};

template <typename T>
struct WaveParams {
    T *L;
    long long n, ld;
    const T *V;
    long long ldv;
    int nwaves;                    // waves in this launch (<= kMaxWaves)
    int nblocks;                   // column blocks of kW columns
    int fstride;                   // row stride (in blocks) of the flag arrays
    unsigned long long down_mask;  // bit q set: wave q is a downdate
    CoefRow<T> *coef;              // [nw][nb][kW]
    ChainRow *chain;               // [nw][nb][kW]
    ChainRow *chain0;              // [nb][kW]      original diagonal data
    double *tend;                  // [nw][nb]      T after the block's last row
    int *pflag;                    // [nw][fstride] panel published (== epoch)
    long long *progress;           // [nw][fstride] (epoch << 32) + tiles done (b + 1 = all)
    double *zbuf;                  // [nw][nb][kW]  T u_hat before the block's last tile
    int *zflag;                    // [nw][fstride]
    double *rdiag;                 // [nw][nb][kW][kW] -S_rc e_r / D_r, r < c (diagonal block)
    double *rtile;                 // [nw][nb][kW][kW] -S_rc e_r (tile: rows of block b, cols of b+1)
    int *rflag0;                   // [nb]          wave-0 data of block b ready
    int *smslot;                   // [kMaxSm]      arrivals per SM (zero at launch)
    int *smrole;                   // [kMaxSm]      role decided by the SM's first block
    int *ndiag;                    // diag-role blocks claimed so far
    int ndiag_blocks;              // blocks of 4 wave workers needed
    long long *trace;              // optional per-task timestamps
    SyncArgs sync;
};

// Per-warp shared memory: the larger of the wave worker's two ratio
// matrices and the sweep worker's tile and row data.
constexpr int kWarpSmemBytes = 2 * kW * kW * 8 + 2 * kW * 32;

// ---------------------------------------------------------------- small helpers

__device__ __forceinline__ CoefRow<double> ld_coef(const CoefRow<double> *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 x = __ldcg(q), y = __ldcg(q + 1);
    return CoefRow<double>{x.x, x.y, y.x, y.y};
}
__device__ __forceinline__ CoefRow<float> ld_coef(const CoefRow<float> *p)
{
    const float4 x = __ldcg(reinterpret_cast<const float4 *>(p));
    return CoefRow<float>{x.x, x.y, x.z, x.w};
}
__device__ __forceinline__ void st_coef(CoefRow<double> *p, const CoefRow<double> &c)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    __stcg(q, make_double2(c.a, c.b));
    __stcg(q + 1, make_double2(c.e1, c.pad));
}
__device__ __forceinline__ void st_coef(CoefRow<float> *p, const CoefRow<float> &c)
{
    __stcg(reinterpret_cast<float4 *>(p), make_float4(c.a, c.b, c.e1, c.pad));
}
__device__ __forceinline__ ChainRow ld_chain(const ChainRow *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 x = __ldcg(q), y = __ldcg(q + 1);
    return ChainRow{x.x, x.y, y.x, y.y};
}
__device__ __forceinline__ void st_chain(ChainRow *p, const ChainRow &c)
{
    double2 *q = reinterpret_cast<double2 *>(p);
    __stcg(q, make_double2(c.e1, c.ie1));
    __stcg(q + 1, make_double2(c.d1, c.id1));
}

// Reciprocal and reciprocal square root to ~1 ulp: the hardware's coarse
// approximations refined by one third-order Newton-Raphson (Householder)
// step, e = 1 - x y: y' = y (1 + e + e^2) for 1/x; e = 1 - x y^2:
// y' = y (1 + e/2 + 3 e^2 / 8) for 1/sqrt(x).
__device__ __forceinline__ double rcp_refined(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    const double t = fma(e, e, e);
    return fma(y, t, y);
}
__device__ __forceinline__ double rsqrt_refined(double x)
{
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double xy = x * y;
    const double e = fma(-xy, y, 1.0);
    const double h = fma(0.375, e, 0.5);
    return fma(y * e, h, y);
}

// Wait helpers (one thread).
__device__ __forceinline__ bool wait_eq(const SyncArgs &s, const int *p, int want, long long who)
{
    return bounded_wait(s, [&] { return ld_acquire_gpu(p) == want; }, [] {}, who);
}
__device__ __forceinline__ bool wait_ge(const SyncArgs &s, const long long *p, long long want,
                                        long long who)
{
    return bounded_wait(s, [&] { return ld_acquire_gpu(p) >= want; }, [] {}, who);
}

// Asynchronous 16-byte global -> shared copies (L2 only), completed by cp_async_wait.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy one kW x kW double matrix (8 KB, row-major) into shared memory with
// the 32 lanes of a warp.
__device__ __forceinline__ void fetch_matrix(double (*dst)[kW], const double *src, int lane)
{
    const char *g = reinterpret_cast<const char *>(src);
    char *d = reinterpret_cast<char *>(&dst[0][0]);
#pragma unroll
    for (int i = 0; i < kW * kW * 8 / (16 * 32); ++i) {
        const int off = (i * 32 + lane) * 16;
        cp_async16(d + off, g + off);
    }
}

// Warp-wide: lane 0 waits, every lane gets the verdict; the __syncwarp
// orders the other lanes' later loads after lane 0's acquire.
#define CHM_WARP_WAIT(expr)                                   \
    do {                                                      \
        int ok_ = 1;                                          \
        if (lane == 0) ok_ = (expr) ? 1 : 0;                  \
        ok_ = __shfl_sync(0xffffffffu, ok_, 0);               \
        if (!ok_) return;                                     \
        __syncwarp();                                         \
    } while (0)

#define CHM_TRACE(pt)                                                                            \
    do {                                                                                         \
        if (P.trace && lane == 0) P.trace[(size_t)trace_row * kTracePoints + (pt)] = global_ns(); \
    } while (0)

// ---------------------------------------------------------------- sweep task

template <typename T>
__device__ void sweep_task(const WaveParams<T> &P, int q, int b, unsigned char *sm)
{
    T(*tile)[kW + 1] = reinterpret_cast<T(*)[kW + 1]>(sm);
    CoefRow<T> *cf = reinterpret_cast<CoefRow<T> *>(sm + sizeof(T) * kW * (kW + 1) + 64);
    ChainRow *ch = reinterpret_cast<ChainRow *>(cf + kW);
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = P.sync;
    const long long n = P.n, ld = P.ld;
    const int nw = P.nwaves, nb = P.nblocks;
    const long long c0 = (long long)b * kW;
    const int ncols = (int)min((long long)kW, n - c0);
    const bool active = lane < ncols;
    const bool last = q == nw - 1;
    const bool has_next = q + 1 < nw;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    const long long who = (long long)b * nw + q;
    const long long *prog_prev = q > 0 ? P.progress + (size_t)(q - 1) * P.fstride + b : nullptr;
    long long *prog_me = P.progress + (size_t)q * P.fstride + b;
    const size_t trace_row = (size_t)who;
    CHM_TRACE(0);

    T uh = active ? P.V[c0 + lane + (long long)q * P.ldv] : T(0);

    if (q == 0) {
        // Original-factor data of block b for wave 0: the diagonal and its
        // inverse, the diagonal block's chain ratios, and (b >= 1) a copy of
        // the tile above the block, taken before any wave rotates it.
        T x[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c)
            x[c] = (lane <= c && c < ncols) ? __ldcg(P.L + c0 + lane + (c0 + c) * ld) : T(0);
        double dl = 1.0;
#pragma unroll
        for (int c = 0; c < kW; ++c)
            if (c == lane) dl = (double)x[c];
        const double idl = active ? rcp_refined(dl) : 1.0;
        if (active) st_chain(P.chain0 + (size_t)b * kW + lane, ChainRow{1.0, 1.0, dl, idl});
        double *rd = P.rdiag + (size_t)b * kW * kW;  // wave 0
#pragma unroll
        for (int c = 0; c < kW; ++c) {
            const double v = (lane < c && c < ncols) ? -(double)x[c] * idl : 0.0;
            __stcg(rd + (size_t)lane * kW + c, v);
        }
        if (b >= 1) {
            const long long r0 = c0 - kW;
#pragma unroll
            for (int c = 0; c < kW; ++c) x[c] = (c < ncols) ? __ldcg(P.L + r0 + lane + (c0 + c) * ld) : T(0);
            double *rt = P.rtile + (size_t)(b - 1) * kW * kW;  // wave 0, tile (b-1, b)
#pragma unroll
            for (int c = 0; c < kW; ++c) __stcg(rt + (size_t)lane * kW + c, -(double)x[c]);
        }
        __syncwarp();
        if (lane == 0) st_release_gpu(P.rflag0 + b, epoch);
    }

    for (int p = 0; p < b; ++p) {
        const bool lastTile = p == b - 1;
        // the tile as the previous wave left it, fetched while the panel is pending
        if (prog_prev) CHM_WARP_WAIT(wait_ge(sy, prog_prev, ep64 + p + 1, who));
        T x[kW];
        {
            const T *src = P.L + (long long)p * kW + lane;
#pragma unroll
            for (int c = 0; c < kW; ++c) x[c] = (c < ncols) ? __ldcg(src + (c0 + c) * ld) : T(0);
        }
        CHM_WARP_WAIT(wait_eq(sy, P.pflag + (size_t)q * P.fstride + p, epoch, who));
        if (lastTile) CHM_TRACE(1);
        const size_t prow = ((size_t)q * nb + p) * kW;
        cf[lane] = ld_coef(P.coef + prow + lane);
        if (lastTile && has_next) ch[lane] = ld_chain(P.chain + prow + lane);
        const double tnext = (p == b - 2) ? __ldcg(P.tend + (size_t)q * nb + p) : 0.0;
#pragma unroll
        for (int c = 0; c < kW; ++c) tile[c][lane] = x[c];
        __syncwarp();
        if (p == b - 2) CHM_TRACE(4);
        T S[kW];
#pragma unroll
        for (int r = 0; r < kW; ++r) S[r] = tile[lane][r];
        if (active) {
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                const CoefRow<T> c = cf[r];
                S[r] = fma(c.a, uh, S[r]);
                uh = fma(-c.b, S[r], uh);
            }
        }
        if (p == b - 2) {
            // the wave worker's carry for block b: z = T u_hat after rows < (b-1) kW
            __stcg(P.zbuf + ((size_t)q * nb + b) * kW + lane, active ? tnext * (double)uh : 0.0);
            __syncwarp();
            if (lane == 0) st_release_gpu(P.zflag + (size_t)q * P.fstride + b, epoch);
            CHM_TRACE(5);
        }
        if (lastTile && has_next) {
            // next wave's dot-product matrix for tile (b-1, b): -S' e'
            double *rt = P.rtile + (((size_t)(q + 1) * nb) + (b - 1)) * kW * kW;
#pragma unroll
            for (int r = 0; r < kW; ++r)
                __stcg(rt + (size_t)r * kW + lane, active ? -(double)S[r] * ch[r].e1 : 0.0);
        }
        if (active) {
            if (last) {
#pragma unroll
                for (int r = 0; r < kW; ++r) S[r] *= cf[r].e1;
            }
#pragma unroll
            for (int r = 0; r < kW; ++r) tile[lane][r] = S[r];
        }
        __syncwarp();
        {
            T *dst = P.L + (long long)p * kW + lane;
#pragma unroll
            for (int c = 0; c < kW; ++c)
                if (c < ncols) __stcg(dst + (c0 + c) * ld, tile[c][lane]);
        }
        __syncwarp();
        if (lane == 0) st_release_gpu(prog_me, ep64 + p + 1);
        if (p == b - 2) CHM_TRACE(6);
    }

    // Diagonal block: wave q's rotations inside it.  The diagonal tile as
    // the previous wave left it is fetched while the panel is pending.
    if (prog_prev) CHM_WARP_WAIT(wait_ge(sy, prog_prev, ep64 + b + 1, who));
    {
        T x[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c)
            x[c] = (lane <= c && c < ncols) ? __ldcg(P.L + c0 + lane + (c0 + c) * ld) : T(0);
        CHM_WARP_WAIT(wait_eq(sy, P.pflag + (size_t)q * P.fstride + b, epoch, who));
        CHM_TRACE(2);
        const size_t drow = ((size_t)q * nb + b) * kW;
        cf[lane] = ld_coef(P.coef + drow + lane);
        ch[lane] = ld_chain(P.chain + drow + lane);
#pragma unroll
        for (int c = 0; c < kW; ++c) tile[c][lane] = x[c];
    }
    __syncwarp();
    {
        T S[kW];
#pragma unroll
        for (int r = 0; r < kW; ++r) S[r] = tile[lane][r];
#pragma unroll
        for (int r = 0; r < kW; ++r) {
            if (r < lane) {
                const CoefRow<T> c = cf[r];
                S[r] = fma(c.a, uh, S[r]);
                uh = fma(-c.b, S[r], uh);
            }
        }
        if (has_next) {
            // next wave's chain ratios for this block: -S'_rc e'_r / D'_r (r < c)
            double *rd = P.rdiag + (((size_t)(q + 1) * nb) + b) * kW * kW;
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                const double v = (r < lane && active) ? -(double)S[r] * ch[r].e1 * ch[r].id1 : 0.0;
                __stcg(rd + (size_t)r * kW + lane, v);
            }
        }
        if (last) {
#pragma unroll
            for (int r = 0; r < kW; ++r)
                if (r < lane) S[r] *= cf[r].e1;
        }
#pragma unroll
        for (int r = 0; r < kW; ++r)
            if (r < lane) tile[lane][r] = S[r];
        if (active) tile[lane][lane] = (T)ch[lane].d1;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kW; ++c)
        if (lane <= c && c < ncols) __stcg(P.L + c0 + lane + (c0 + c) * ld, tile[c][lane]);
    __syncwarp();
    CHM_TRACE(3);
    if (lane == 0) st_release_gpu(prog_me, ep64 + b + 1);
}

// ---------------------------------------------------------------- wave worker

template <typename T>
__device__ void wave_worker(const WaveParams<T> &P, int q, unsigned char *sm)
{
    double(*R)[kW] = reinterpret_cast<double(*)[kW]>(sm);                 // chain ratios [r][c]
    double(*Rt)[kW] = reinterpret_cast<double(*)[kW]>(sm + kW * kW * 8);  // tile above [r][c]
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = P.sync;
    const long long n = P.n;
    const int nw = P.nwaves, nb = P.nblocks;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    const int sg = ((P.down_mask >> q) & 1ull) ? -1 : 1;
    const double sgd = (double)sg;
    const long long who = -1 - q;
    const long long *prog_prev = q > 0 ? P.progress + (size_t)(q - 1) * P.fstride : nullptr;

    // Inputs of block b: row data, ratio matrices, carry z.
    auto rowdata = [&](int b) -> ChainRow {
        const int rows = (int)min((long long)kW, n - (long long)b * kW);
        if (lane >= rows) return ChainRow{1.0, 1.0, 1.0, 1.0};
        return ld_chain((q == 0 ? P.chain0 + (size_t)b * kW : P.chain + ((size_t)(q - 1) * nb + b) * kW) +
                        lane);
    };
    auto carry = [&](int b) -> double {
        const long long c0 = (long long)b * kW;
        if (b >= 2) return __ldcg(P.zbuf + ((size_t)q * nb + b) * kW + lane);
        return (c0 + lane < n) ? (double)P.V[c0 + lane + (long long)q * P.ldv] : 0.0;
    };
    auto fetch = [&](int b) {
        fetch_matrix(R, P.rdiag + ((size_t)q * nb + b) * kW * kW, lane);
        if (b >= 1) fetch_matrix(Rt, P.rtile + ((size_t)q * nb + (b - 1)) * kW * kW, lane);
        cp_async_commit();
    };

    double pprev = 0.0;  // p of the previous block's row `lane`
    double Tend = 1.0;   // T before the current block
    double iTend = 1.0;  // 1 / Tend
    bool have = false;   // block b's inputs already requested
    ChainRow rowd{1.0, 1.0, 1.0, 1.0};
    double z = 0.0;
    for (int b = 0; b < nb; ++b) {
        const long long c0 = (long long)b * kW;
        const int rows = (int)min((long long)kW, n - c0);
        const bool active = lane < rows;
        const size_t trace_row = (size_t)nw * nb + (size_t)q * nb + b;
        CHM_TRACE(0);
        if (!have) {
            if (q == 0) {
                CHM_WARP_WAIT(wait_eq(sy, P.rflag0 + b, epoch, who));
            } else {
                CHM_WARP_WAIT(wait_ge(sy, prog_prev + b, ep64 + b + 1, who));
            }
            if (b >= 2) CHM_WARP_WAIT(wait_eq(sy, P.zflag + (size_t)q * P.fstride + b, epoch, who));
            fetch(b);
            rowd = rowdata(b);
            z = carry(b);
        }
        cp_async_wait();
        __syncwarp();
        CHM_TRACE(1);
        // early look at the next block's flags: every lane issues the same
        // acquiring loads now and compares after the arithmetic below, so
        // the loads are in flight meanwhile
        int fz = epoch;
        long long fr = 0;
        if (b + 1 < nb) {
            if (b + 1 >= 2) fz = ld_acquire_gpu(P.zflag + (size_t)q * P.fstride + b + 1);
            fr = q == 0 ? (long long)ld_acquire_gpu(P.rflag0 + b + 1) : ld_acquire_gpu(prog_prev + b + 1);
        }
        if (b >= 1) {
            // rows of the block above: z_c += sum_r (-S_rc e_r) p_r
            double z1 = 0.0, z2 = 0.0, z3 = 0.0;
#pragma unroll
            for (int r = 0; r < kW; r += 4) {
                z = fma(Rt[r][lane], __shfl_sync(FULL, pprev, r), z);
                z1 = fma(Rt[r + 1][lane], __shfl_sync(FULL, pprev, r + 1), z1);
                z2 = fma(Rt[r + 2][lane], __shfl_sync(FULL, pprev, r + 2), z2);
                z3 = fma(Rt[r + 3][lane], __shfl_sync(FULL, pprev, r + 3), z3);
            }
            z = (z + z1) + (z2 + z3);
        }
        // forward substitution through the block
#pragma unroll
        for (int r = 0; r < kW; ++r) {
            const double zr = __shfl_sync(FULL, z, r);
            z = fma(R[r][lane], zr, z);
        }
        __syncwarp();
        // the ratio buffers are free again: request the next block's inputs
        const bool rr = q == 0 ? fr == (long long)epoch : fr >= ep64 + b + 2;
        const int nready = __all_sync(FULL, b + 1 < nb && fz == epoch && rr);
        ChainRow rowd_next{1.0, 1.0, 1.0, 1.0};
        double z_next = 0.0;
        have = false;
        if (nready) {
            fetch(b + 1);
            rowd_next = rowdata(b + 1);
            z_next = carry(b + 1);
            have = true;
        }
        CHM_TRACE(2);
        const double p = active ? z * rowd.id1 : 0.0;
        double x = sgd * p * p;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        const double Tn = Tend + x;
        const double Tlast = __shfl_sync(FULL, Tn, rows - 1);
        const bool bad = active && !(rowd.d1 > 0.0 && rowd.d1 <= DBL_MAX && Tn > 0.0 && Tn <= DBL_MAX);
        const unsigned badm = __ballot_sync(FULL, bad);
        if (badm && lane == 0) record_error(sy, kStatusNotPD, c0 + (__ffs(badm) - 1));
        const double iTn = rcp_refined(Tn);
        double iTp = __shfl_up_sync(FULL, iTn, 1);
        if (lane == 0) iTp = iTend;
        const double ratio = Tn * iTp;           // c^2
        const double rc = rsqrt_refined(ratio);  // 1/c
        const double c = ratio * rc;
        const double a = sgd * p * rowd.ie1;
        const double bb = p * rowd.e1 * iTn;
        const ChainRow nrow{rowd.e1 * rc, rowd.ie1 * c, rowd.d1 * c, rowd.id1 * rc};
        if (active) {
            const size_t prow = ((size_t)q * nb + b) * kW + lane;
            st_coef(P.coef + prow, CoefRow<T>{(T)a, (T)bb, (T)nrow.e1, T(0)});
            st_chain(P.chain + prow, nrow);
        }
        if (lane == 0) __stcg(P.tend + (size_t)q * nb + b, Tlast);
        __syncwarp();
        if (lane == 0) st_release_gpu(P.pflag + (size_t)q * P.fstride + b, epoch);
        CHM_TRACE(3);
        pprev = p;
        Tend = Tlast;
        iTend = __shfl_sync(FULL, iTn, rows - 1);
        rowd = rowd_next;
        z = z_next;
    }
}

// ---------------------------------------------------------------- entry

template <typename T>
__global__ void __launch_bounds__(128, 3) wave_kernel(WaveParams<T> P)
{
    extern __shared__ __align__(16) unsigned char chm_smem[];
    __shared__ int s_role, s_didx;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const SyncArgs &sy = P.sync;
    if (threadIdx.x == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        int role = kRoleSweep, didx = -1;
        if (smid < (unsigned)kMaxSm) {
            if (atomicAdd(P.smslot + smid, 1) == 0) {
                const int d = atomicAdd(P.ndiag, 1);
                if (d < P.ndiag_blocks) {
                    role = kRoleDiag;
                    didx = d;
                }
                st_release_gpu(P.smrole + smid, role);
            } else {
                const int *pr = P.smrole + smid;
                int seen = 0;
                bounded_wait(
                    sy, [&] { return (seen = ld_relaxed_gpu(pr)) != 0; },
                    [&] { (void)ld_acquire_gpu(pr); }, -1000);
                role = seen == kRoleDiag ? 0 : kRoleSweep;  // a wave-worker SM runs nothing else
            }
        }
        s_role = role;
        s_didx = didx;
    }
    __syncthreads();
    const int role = s_role;
    if (role == 0) return;
    unsigned char *sm = chm_smem + (size_t)warp * kWarpSmemBytes;
    if (role == kRoleDiag) {
        const int q = s_didx * 4 + warp;
        if (q < P.nwaves) wave_worker<T>(P, q, sm);
        return;
    }
    const int ntasks = P.nwaves * P.nblocks;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(sy.ticket, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntasks || aborted(sy)) return;
        sweep_task<T>(P, t % P.nwaves, t / P.nwaves, sm);
        if (aborted(sy)) return;
    }
}

#undef CHM_WARP_WAIT
#undef CHM_TRACE

}  // namespace chm
