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
//   * wave blocks: one thread block per wave, each on an SM of its own
//     (claimed at start-up through %smid), walks the diagonal blocks in
//     order with four specialised warps that hand work to each other through
//     shared memory:
//       A  the forward substitution through the diagonal block, with ratio
//          matrices prepared in advance;
//       B  the 32-row dot product that carries the previous block's p into
//          this block, then p, T and the rotation coefficients, and the
//          publication of the block's panel;
//       C  the wave's rotations inside the diagonal block, the next wave's
//          ratio matrix of that block, and its store;
//       D  prefetch of the next block's inputs (cp.async).
//   * sweep workers: every other warp takes tasks (wave q, column block b)
//     in ticket order t = b * nwaves + q and rotates the block's off-diagonal
//     tiles with wave q's panels, the update vector held in registers.  It
//     also publishes what the wave block needs: the carry z for the block,
//     the carry u_hat at the diagonal, and the next wave's dot-product matrix.
// Every wait is bounded (%globaltimer); a sweep task only waits on events of
// tasks with smaller tickets or on wave blocks, which always run.
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
    double *zbuf;                  // [nw][nb][kW]  T u_hat before the block's last tile
    double *carry;                 // [nw][nb][kW]  u_hat at the diagonal block
    double *rdiag;                 // [nw][nb][kW][kW] -S_rc e_r / D_r, r < c (diagonal block)
    double *rtile;                 // [nw][nb][kW][kW] -S_rc e_r (tile: rows of block b, cols of b+1)
    int *pflag;                    // [nw][fstride] panel published (== epoch)
    long long *progress;           // [nw][fstride] (epoch << 32) + off-diagonal tiles done
    int *zflag;                    // [nw][fstride] zbuf ready
    int *cflag;                    // [nw][fstride] carry ready
    int *dflag;                    // [nw][fstride] diagonal block done, next wave's rdiag ready
    int *rflag0;                   // [nb]          wave-0 data of block b ready
    int *smslot;                   // [kMaxSm]      arrivals per SM (zero at launch)
    int *smrole;                   // [kMaxSm]      role decided by the SM's first block
    int *ndiag;                    // wave blocks claimed so far
    long long *trace;              // optional per-task timestamps
    SyncArgs sync;
};

// Dynamic shared memory per thread block: four warps' worth.
constexpr int kWarpSmemBytes = 18432;
constexpr int kBlockSmemBytes = 4 * kWarpSmemBytes;

// Shared memory of a wave block.
template <typename T>
struct WaveSmem {
    double R[2][kW][kW];   // chain ratios of the block, [r][c]
    double Rt[2][kW][kW];  // dot-product matrix of the tile above, [r][c]
    ChainRow rowd[2][kW];  // row data of the block before this wave
    double zpart[2][kW];   // carry z before the tile above
    double zbox[kW];       // B -> A: z entering the chain
    double cbox[kW];       // A -> B: z after the chain
    CoefRow<T> cf[2][kW];  // B -> C: sweep coefficients of the block
    ChainRow cnew[2][kW];  // B -> C: row data after this wave
    T DT[kW][kW + 1];      // C: the diagonal tile, [c][r]
    int dseq, zseq, cseq, bseq, fseq, bail;
};
static_assert(sizeof(WaveSmem<double>) <= kBlockSmemBytes, "wave block shared memory");

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

// Shared-memory sequence counters between the warps of a wave block.  The
// writer stores its data, fences the block and raises the counter; the
// reader waits for the counter (bounded) and fences before reading.  `bail`
// is raised by a warp that stops early, so that the others stop waiting.
__device__ __forceinline__ void seq_post(int *seq, int v)
{
    __threadfence_block();
    *reinterpret_cast<volatile int *>(seq) = v;
}
__device__ __forceinline__ bool seq_wait(const SyncArgs &s, int *seq, int want, int *bail,
                                         long long who)
{
    volatile int *vs = reinterpret_cast<volatile int *>(seq);
    volatile int *vb = reinterpret_cast<volatile int *>(bail);
    if (*vs >= want) {
        __threadfence_block();
        return true;
    }
    const long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        __nanosleep(8);
        if (*vs >= want) {
            __threadfence_block();
            return true;
        }
        if ((it & 255u) == 0u) {
            if (*vb || aborted(s)) return false;
            if (global_ns() - t0 > s.timeout_ns || it > (1u << 28)) {
                record_error(s, kStatusTimeout, who);
                *vb = 1;
                return false;
            }
        }
    }
}

// Asynchronous 16-byte global -> shared copies (L2 only), completed by cp_async_wait.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Copy `bytes` (a multiple of 16) from global to shared memory with the 32
// lanes of a warp.
__device__ __forceinline__ void fetch_bytes(void *dst, const void *src, int bytes, int lane)
{
    const char *g = reinterpret_cast<const char *>(src);
    char *d = reinterpret_cast<char *>(dst);
    for (int off = lane * 16; off < bytes; off += 32 * 16) cp_async16(d + off, g + off);
}

// Warp-wide wait: all 32 lanes poll together and lane 0's verdict is the
// warp's.  The poll loop is warp-uniform on purpose: a loop taken by lane 0
// alone leaves the warp split, and on this part every later shfl.sync of the
// warp then pays a resynchronisation (measured: a 32-deep dependent shuffle
// chain 8.6 times slower), which is exactly the latency-bound path of the
// chain and of the sweep tasks.
#define CHM_WARP_WAIT(expr)                                   \
    do {                                                      \
        int ok_ = (expr) ? 1 : 0;                             \
        ok_ = __shfl_sync(0xffffffffu, ok_, 0);               \
        if (!ok_) return;                                     \
        __syncwarp();                                         \
    } while (0)

// The same for a shared-memory sequence counter of the wave block.
#define CHM_SEQ_WAIT(seqp, want) CHM_WARP_WAIT(seq_wait(sy, (seqp), (want), &S.bail, who))

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
        // inverse, the diagonal block's chain ratios, and (b >= 1) the dot
        // product matrix of the tile above, taken before any wave rotates it.
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
            // the wave block's carry for block b: z = T u_hat after rows < (b-1) kW
            __stcg(P.zbuf + ((size_t)q * nb + b) * kW + lane, active ? tnext * (double)uh : 0.0);
            __syncwarp();
            if (lane == 0) st_release_gpu(P.zflag + (size_t)q * P.fstride + b, epoch);
        }
        if (lastTile) {
            // u_hat entering the diagonal block, for the wave block's rotations there
            __stcg(P.carry + ((size_t)q * nb + b) * kW + lane, active ? (double)uh : 0.0);
            __syncwarp();
            if (lane == 0) st_release_gpu(P.cflag + (size_t)q * P.fstride + b, epoch);
            CHM_TRACE(2);
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
    }
    CHM_TRACE(3);
}

// ---------------------------------------------------------------- wave block

#define CHM_WTRACE(b, pt)                                                                      \
    do {                                                                                       \
        if (P.trace && lane == 0)                                                              \
            P.trace[((size_t)P.nwaves * P.nblocks + (size_t)q * P.nblocks + (b)) * kTracePoints + \
                    (pt)] = global_ns();                                                       \
    } while (0)

// Warp D: the inputs of each block for warps A and B, one block ahead.
template <typename T>
__device__ void wave_prefetch(const WaveParams<T> &P, int q, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = P.sync;
    const long long n = P.n;
    const int nb = P.nblocks;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    const long long who = -1 - q;
    const long long *prog_prev = q > 0 ? P.progress + (size_t)(q - 1) * P.fstride : nullptr;
    for (int b = 0; b < nb; ++b) {
        const int s = b & 1;
        const long long c0 = (long long)b * kW;
        // the slot's previous block (b - 2) must be finished by warps A, B, C
        if (b >= 2) CHM_SEQ_WAIT(&S.fseq, b - 1);
        CHM_WTRACE(b, 0);
        if (q == 0) {
            CHM_WARP_WAIT(wait_eq(sy, P.rflag0 + b, epoch, who));
        } else {
            CHM_WARP_WAIT(wait_eq(sy, P.dflag + (size_t)(q - 1) * P.fstride + b, epoch, who) &&
                          (b == 0 || wait_ge(sy, prog_prev + b, ep64 + b, who)));
        }
        CHM_WTRACE(b, 1);
        if (b >= 2) CHM_WARP_WAIT(wait_eq(sy, P.zflag + (size_t)q * P.fstride + b, epoch, who));
        CHM_WTRACE(b, 2);
        fetch_bytes(&S.R[s][0][0], P.rdiag + ((size_t)q * nb + b) * kW * kW, kW * kW * 8, lane);
        if (b >= 1) fetch_bytes(&S.Rt[s][0][0], P.rtile + ((size_t)q * nb + (b - 1)) * kW * kW, kW * kW * 8, lane);
        fetch_bytes(&S.rowd[s][0], (q == 0 ? P.chain0 + (size_t)b * kW : P.chain + ((size_t)(q - 1) * nb + b) * kW),
                    kW * (int)sizeof(ChainRow), lane);
        if (b >= 2) {
            fetch_bytes(&S.zpart[s][0], P.zbuf + ((size_t)q * nb + b) * kW, kW * 8, lane);
        } else {
            S.zpart[s][lane] = (c0 + lane < n) ? (double)P.V[c0 + lane + (long long)q * P.ldv] : 0.0;
        }
        cp_async_commit();
        cp_async_wait();
        __syncwarp();
        CHM_WTRACE(b, 3);
        if (lane == 0) seq_post(&S.dseq, b + 1);
    }
}

// Warp A: the forward substitution through each diagonal block.
template <typename T>
__device__ void wave_chain(const WaveParams<T> &P, int q, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = P.sync;
    const long long who = -1 - q;
    for (int b = 0; b < P.nblocks; ++b) {
        CHM_SEQ_WAIT(&S.zseq, b + 1);
        CHM_WTRACE(b, 8);
        double(*R)[kW] = S.R[b & 1];
        double z = S.zbox[lane];
#pragma unroll
        for (int r = 0; r < kW; ++r) {
            const double zr = __shfl_sync(FULL, z, r);
            z = fma(R[r][lane], zr, z);
        }
        S.cbox[lane] = z;
        __syncwarp();
        CHM_WTRACE(b, 9);
        if (lane == 0) seq_post(&S.cseq, b + 1);
    }
}

// Warp B: the dot product into each block, then p, T and the coefficients
// of the block just chained, and the panel's publication.  The next chain
// is started before a panel is published whenever its inputs are already in.
template <typename T>
__device__ void wave_coef(const WaveParams<T> &P, int q, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = P.sync;
    const long long n = P.n;
    const int nb = P.nblocks;
    const int epoch = sy.epoch;
    const double sgd = ((P.down_mask >> q) & 1ull) ? -1.0 : 1.0;
    const long long who = -1 - q;
    double pprev = 0.0;  // p of the block last chained, row `lane`
    double Tend = 1.0, iTend = 1.0;
    int pending = -1;    // block chained (or being chained) but not yet published
    int next = 0;        // next block whose chain input is to be formed
    bool ok = true;
    auto wait_seq = [&](int *seq, int want) -> bool {
        int v = seq_wait(sy, seq, want, &S.bail, who) ? 1 : 0;  // all lanes: see CHM_WARP_WAIT
        v = __shfl_sync(FULL, v, 0);
        __syncwarp();
        return v != 0;
    };
    auto form_input = [&](int b) {
        // z entering block b's chain: the carry plus the rows of the block above
        const int s = b & 1;
        double z = S.zpart[s][lane];
        if (b >= 1) {
            double z1 = 0.0, z2 = 0.0, z3 = 0.0;
#pragma unroll
            for (int r = 0; r < kW; r += 4) {
                z = fma(S.Rt[s][r][lane], __shfl_sync(FULL, pprev, r), z);
                z1 = fma(S.Rt[s][r + 1][lane], __shfl_sync(FULL, pprev, r + 1), z1);
                z2 = fma(S.Rt[s][r + 2][lane], __shfl_sync(FULL, pprev, r + 2), z2);
                z3 = fma(S.Rt[s][r + 3][lane], __shfl_sync(FULL, pprev, r + 3), z3);
            }
            z = (z + z1) + (z2 + z3);
        }
        S.zbox[lane] = z;
        __syncwarp();
        CHM_WTRACE(b, 4);
        if (lane == 0) seq_post(&S.zseq, b + 1);
    };
    auto publish = [&](int b, double p) {
        // T and the coefficients of block b (already chained), given its p
        const int s = b & 1;
        const long long c0 = (long long)b * kW;
        const int rows = (int)min((long long)kW, n - c0);
        const bool active = lane < rows;
        const ChainRow rowd = S.rowd[s][lane];
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
        const CoefRow<T> cr{(T)(sgd * p * rowd.ie1), (T)(p * rowd.e1 * iTn), (T)(rowd.e1 * rc), T(0)};
        const ChainRow nrow{rowd.e1 * rc, rowd.ie1 * c, rowd.d1 * c, rowd.id1 * rc};
        S.cf[s][lane] = cr;
        S.cnew[s][lane] = nrow;
        __syncwarp();
        if (lane == 0) seq_post(&S.bseq, b + 1);
        if (active) {
            const size_t prow = ((size_t)q * nb + b) * kW + lane;
            st_coef(P.coef + prow, cr);
            st_chain(P.chain + prow, nrow);
        }
        if (lane == 0) __stcg(P.tend + (size_t)q * nb + b, Tlast);
        __syncwarp();
        if (lane == 0) st_release_gpu(P.pflag + (size_t)q * P.fstride + b, epoch);
        CHM_WTRACE(b, 5);
        Tend = Tlast;
        iTend = __shfl_sync(FULL, iTn, rows - 1);
    };

    while (ok && (next < nb || pending >= 0)) {
        if (pending < 0) {
            // nothing is being chained: form the next input (waiting for it)
            if (!wait_seq(&S.dseq, next + 1)) return;
            form_input(next);
            pending = next++;
        }
        // collect the chain of `pending`; its p feeds the next dot product
        if (!wait_seq(&S.cseq, pending + 1)) return;
        const int done = pending;
        pending = -1;
        {
            const long long c0 = (long long)done * kW;
            pprev = (c0 + lane < n) ? S.cbox[lane] * S.rowd[done & 1][lane].id1 : 0.0;
        }
        if (next < nb) {
            const int ready = __shfl_sync(FULL, *reinterpret_cast<volatile int *>(&S.dseq) >= next + 1 ? 1 : 0, 0);
            if (ready) {
                __threadfence_block();
                form_input(next);
                pending = next++;
            }
        }
        publish(done, pprev);
    }
}

// Warp C: the wave's rotations inside each diagonal block.
template <typename T>
__device__ void wave_diag(const WaveParams<T> &P, int q, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = P.sync;
    const long long n = P.n, ld = P.ld;
    const int nw = P.nwaves, nb = P.nblocks;
    const int epoch = sy.epoch;
    const bool last = q == nw - 1;
    const bool has_next = q + 1 < nw;
    const long long who = -1 - q;
    for (int b = 0; b < nb; ++b) {
        const int s = b & 1;
        const long long c0 = (long long)b * kW;
        const int ncols = (int)min((long long)kW, n - c0);
        const bool active = lane < ncols;
        // u_hat entering the block (from the sweep of its last off-diagonal tile)
        T uh = T(0);
        if (b == 0) {
            uh = active ? P.V[c0 + lane + (long long)q * P.ldv] : T(0);
        } else {
            CHM_WARP_WAIT(wait_eq(sy, P.cflag + (size_t)q * P.fstride + b, epoch, who));
            uh = (T)__ldcg(P.carry + ((size_t)q * nb + b) * kW + lane);
        }
        CHM_WTRACE(b, 10);
        // the tile as the previous wave left it: warp D acquired that wave's
        // release of this block before announcing the block's inputs
        CHM_SEQ_WAIT(&S.dseq, b + 1);
        {
            T x[kW];
#pragma unroll
            for (int c = 0; c < kW; ++c)
                x[c] = (lane <= c && c < ncols) ? __ldcg(P.L + c0 + lane + (c0 + c) * ld) : T(0);
#pragma unroll
            for (int c = 0; c < kW; ++c) S.DT[c][lane] = x[c];
        }
        CHM_WTRACE(b, 11);
        CHM_SEQ_WAIT(&S.bseq, b + 1);
        CHM_WTRACE(b, 12);
        T Sv[kW];
#pragma unroll
        for (int r = 0; r < kW; ++r) Sv[r] = S.DT[lane][r];
#pragma unroll
        for (int r = 0; r < kW; ++r) {
            if (r < lane) {
                const CoefRow<T> c = S.cf[s][r];
                Sv[r] = fma(c.a, uh, Sv[r]);
                uh = fma(-c.b, Sv[r], uh);
            }
        }
        if (has_next) {
            // next wave's chain ratios for this block: -S'_rc e'_r / D'_r (r < c)
            double *rd = P.rdiag + (((size_t)(q + 1) * nb) + b) * kW * kW;
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                const ChainRow cn = S.cnew[s][r];
                const double v = (r < lane && active) ? -(double)Sv[r] * cn.e1 * cn.id1 : 0.0;
                __stcg(rd + (size_t)r * kW + lane, v);
            }
        }
        if (last) {
#pragma unroll
            for (int r = 0; r < kW; ++r)
                if (r < lane) Sv[r] *= S.cf[s][r].e1;
        }
#pragma unroll
        for (int r = 0; r < kW; ++r)
            if (r < lane) S.DT[lane][r] = Sv[r];
        if (active) S.DT[lane][lane] = (T)S.cnew[s][lane].d1;
        __syncwarp();
#pragma unroll
        for (int c = 0; c < kW; ++c)
            if (lane <= c && c < ncols) __stcg(P.L + c0 + lane + (c0 + c) * ld, S.DT[c][lane]);
        __syncwarp();
        if (lane == 0) st_release_gpu(P.dflag + (size_t)q * P.fstride + b, epoch);
        CHM_WTRACE(b, 13);
        if (lane == 0) seq_post(&S.fseq, b + 1);
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
                if (d < P.nwaves) {
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
                role = seen == kRoleDiag ? 0 : kRoleSweep;  // a wave block's SM runs nothing else
            }
        }
        s_role = role;
        s_didx = didx;
    }
    __syncthreads();
    const int role = s_role;
    if (role == 0) return;
    if (role == kRoleDiag) {
        WaveSmem<T> &S = *reinterpret_cast<WaveSmem<T> *>(chm_smem);
        if (threadIdx.x == 0) S.dseq = S.zseq = S.cseq = S.bseq = S.fseq = S.bail = 0;
        __syncthreads();
        const int q = s_didx;
        if (warp == 0) wave_chain<T>(P, q, S);
        else if (warp == 1) wave_coef<T>(P, q, S);
        else if (warp == 2) wave_diag<T>(P, q, S);
        else wave_prefetch<T>(P, q, S);
        return;
    }
    unsigned char *sm = chm_smem + (size_t)warp * kWarpSmemBytes;
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
#undef CHM_SEQ_WAIT
#undef CHM_TRACE
#undef CHM_WTRACE

}  // namespace chm
