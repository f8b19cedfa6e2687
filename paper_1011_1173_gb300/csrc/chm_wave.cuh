// Wave-pipelined rank-k up/downdate kernel (Walder 2010, Algorithm 1, with
// the CPU/GPU panelling of Sec. 4 replaced by one device-resident launch
// that may carry many independent factors).
//
// A rank-k modification is k waves: wave q is the rank-1 modification of the
// factor left by waves < q by column q of V (Sec. 4.1 processes columns in
// order; any dependency-respecting order gives the same factor).  A launch
// holds one or more problems (factor, V, signs); a (problem, wave) pair is
// the unit of scheduling.
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
// Work split.  The SMs of the launch form G groups, each one wave SM plus
// sweep SMs.  A group takes pairs from a global counter, in pair order, and
// runs one pair at a time:
//   * the wave block (the one thread block on the wave SM) walks the pair's
//     diagonal blocks in order with four specialised warps that hand work to
//     each other through shared memory:
//       A  the forward substitution through the diagonal block, with ratio
//          matrices prepared in advance;
//       B  the 32-row dot product that carries the previous block's p into
//          this block, then p, T and the rotation coefficients, and the
//          publication of the block's panel;
//       C  the wave's rotations inside the diagonal block and the next
//          wave's ratio matrix of that block;
//       D  prefetch of the next blocks' inputs (cp.async), the store of
//          each rotated diagonal tile and the block's release.
//   * every warp of the group's sweep blocks takes tasks (column block b of
//     the group's current pair) from the group's ticket word and rotates the
//     block's off-diagonal tiles with the pair's panels, the update vector
//     held in registers.  It also publishes what the wave block needs: the
//     carry z for the block, the carry u_hat at the diagonal, and the next
//     wave's dot-product matrix.
// A pair waits only on itself and on the previous wave of its problem, which
// was taken from the counter earlier and is running or done, so the launch
// always progresses.  Every wait is bounded (%globaltimer).
//
// Storage between waves of one launch: the diagonal holds true values, an
// off-diagonal L_ij is held as S_ij = L_ij / e_i.  Each problem's last pair
// is a final pass that multiplies the last wave's scales back in, trailing
// that wave tile by tile.
#pragma once

#include "chm_device.cuh"
#include "chm_layout.h"

namespace chm {

template <typename T>
struct Launch {
    const Prob *probs;      // device array [nprobs]; null: the one problem is prob0
    Prob prob0;
    const int *pair_prob;   // device array [npairs]: problem of each pair; null: all 0
    int nprobs, npairs, ngroups, nbmax;
    int *ctl;               // kCtlInts control words
    long long *status;      // sticky {status, row} of the scratch owner
    long long *trace;       // optional timestamps, [2][npairs][nbmax][kTracePoints]
    long long timeout_ns;
    int skip_publish;       // test hook: wave blocks never release this block's panel (-1: none)
    // the workspace allocations the problems' regions are carved from (bounds-checked builds)
    const char *ws_data;
    size_t ws_data_bytes;
    const int *ws_iflags;
    size_t ws_iflags_n;
    const long long *ws_progress;
    size_t ws_progress_n;
    long long chk_cut;      // bounds-checked build: columns taken off each factor's declared extent
};

// Everything one task needs about its pair.
template <typename T>
struct Wave {
    T *L;
    const T *V;                 // column q of the problem's V
    long long n, ld;
    int nb, q, pair;
    bool has_next;
    bool unscale;               // the problem's final pass: rows times the last wave's scale
    double sg;                  // +1 update, -1 downdate
    CoefRow<T> *coef;           // [nb][kW] this wave
    ChainRow *chain;            // [nb][kW] this wave's output row data
    const ChainRow *chain_in;   // [nb][kW] row data before this wave
    ChainRow *chain0;           // [nb][kW] original factor's row data (wave 0 writes)
    double *tend, *rdiag, *rtile;
    double *rdiag_next, *rtile_next;  // the next wave's (null without one)
    int *pflag, *dflag, *rflag0;
    const int *dflag_prev;
    long long *progress;
    const long long *progress_prev;
    long long *ztag, *ctag;     // [nb][kW][2] tagged carries z and u_hat
    long long *final_done;      // final pass: tagged count of finished column tasks
    long long *trace_sweep, *trace_wave;  // this pair's rows, or null
    int skip_publish;                     // test hook (see Launch)
    bool ok;                              // false: a region failed its bounds check; skip the task
    SyncArgs sync;
};

template <typename T>
__device__ Wave<T> make_wave(const Launch<T> &P, int j)
{
    const int i = P.pair_prob ? __ldg(P.pair_prob + j) : 0;
    const Prob pr = P.probs ? P.probs[i] : P.prob0;
    Wave<T> w;
    const int q = j - pr.pair0, nb = pr.nb;
    const PairRec rc = pair_rec(nb);
    char *d = pr.data + (size_t)q * rc.bytes;
    w.L = static_cast<T *>(pr.L);
    w.V = static_cast<const T *>(pr.V) + (long long)q * pr.ldv;
    w.n = pr.n;
    w.ld = pr.ld;
    w.nb = nb;
    w.q = q;
    w.pair = j;
    w.has_next = q + 1 < pr.k;
    w.unscale = q == pr.k;  // the pair after the last wave; it owns no scratch of its own
    w.sg = ((pr.down_mask >> q) & 1ull) ? -1.0 : 1.0;
    w.coef = reinterpret_cast<CoefRow<T> *>(d + rc.coef);
    w.chain = reinterpret_cast<ChainRow *>(d + rc.chain);
    w.chain0 = reinterpret_cast<ChainRow *>(pr.data + (size_t)pr.k * rc.bytes);
    w.chain_in = q == 0 ? w.chain0 : reinterpret_cast<const ChainRow *>(d - rc.bytes + rc.chain);
    w.tend = reinterpret_cast<double *>(d + rc.tend);
    w.rdiag = reinterpret_cast<double *>(d + rc.rdiag);
    w.rtile = reinterpret_cast<double *>(d + rc.rtile);
    w.rdiag_next = w.has_next ? reinterpret_cast<double *>(d + rc.bytes + rc.rdiag) : nullptr;
    w.rtile_next = w.has_next ? reinterpret_cast<double *>(d + rc.bytes + rc.rtile) : nullptr;
    int *f = pr.iflags + (size_t)q * 2 * nb;
    w.pflag = f;
    w.dflag = f + nb;
    w.dflag_prev = q > 0 ? f - nb : nullptr;
    w.rflag0 = pr.iflags + (size_t)pr.k * 2 * nb;
    w.progress = pr.progress + (size_t)q * nb;
    w.progress_prev = q > 0 ? w.progress - nb : nullptr;
    w.ztag = pr.progress + (size_t)pr.k * nb + (size_t)q * nb * kW * 2;
    w.ctag = pr.progress + (size_t)pr.k * nb * (1 + kW * 2) + (size_t)q * nb * kW * 2;
    w.final_done = pr.progress + prob_final_done(nb, pr.k);
    if (P.trace) {
        const size_t row = (size_t)j * P.nbmax * kTracePoints;
        w.trace_sweep = P.trace + row;
        w.trace_wave = P.trace + (size_t)P.npairs * P.nbmax * kTracePoints + row;
    } else {
        w.trace_sweep = w.trace_wave = nullptr;
    }
    w.skip_publish = P.skip_publish;
    w.sync.abort_flag = P.ctl + kCtlAbort;
    w.sync.status = P.status;
    w.sync.user_info = pr.info;
    w.sync.epoch = ld_relaxed_gpu(P.ctl + kCtlEpoch);
    w.sync.timeout_ns = P.timeout_ns;
    w.sync.chk_cut = P.chk_cut;
    w.ok = true;
#ifdef CHM_CHECK
    // the problem's regions inside the workspace allocations, and this pair's
    // slice (or, for the final pass, the row data after the k slices) inside
    // the problem's data region
    w.ok = CHK_REGION(w.sync, pr.data, prob_data_bytes(nb, pr.k), P.ws_data, P.ws_data_bytes) &&
           CHK_REGION(w.sync, pr.iflags, prob_iflags(nb, pr.k) * sizeof(int), P.ws_iflags,
                      P.ws_iflags_n * sizeof(int)) &&
           CHK_REGION(w.sync, pr.progress, prob_progress(nb, pr.k) * sizeof(long long), P.ws_progress,
                      P.ws_progress_n * sizeof(long long)) &&
           CHK_REGION(w.sync, d, q < pr.k ? rc.bytes : (size_t)nb * kW * sizeof(ChainRow), pr.data,
                      prob_data_bytes(nb, pr.k)) &&
           CHK_RECT(w.sync, (long long)q, (long long)pr.k + 1, 1, 1 << 30);
#endif
    return w;
}

// Input slots of the wave block: block b's inputs live in slot b % kSlots,
// so the prefetch may run up to kSlots - 1 blocks ahead of the finish.
constexpr int kSlots = 3;

// Shared memory of a wave block.
template <typename T>
struct WaveSmem {
    double R[kSlots][kW][kW];   // chain ratios of the block, [r][c]
    double Rt[kSlots][kW][kW];  // dot-product matrix of the tile above, [r][c]
    ChainRow rowd[kSlots][kW];  // row data of the block before this wave
    double zpart[kSlots][kW];   // carry z before the tile above
    double zbox[kW];            // B -> A: z entering the chain
    double cbox[kW];            // A -> B: z after the chain
    CoefRow<T> cf[kSlots][kW];  // B -> C: sweep coefficients of the block
    ChainRow cnew[kSlots][kW];  // B -> C, D: row data after this wave
    T DT[kW][kW + 1];           // C -> D: the rotated diagonal tile, [c][r]
    int dseq;                   // D: inputs of blocks < dseq fetched
    int zseq;                   // B: chain inputs of blocks < zseq formed
    int cseq;                   // A: blocks < cseq chained
    int bseq;                   // B: coefficients of blocks < bseq formed
    int cdone;                  // C: blocks < cdone rotated (in DT)
    int fseq;                   // D: blocks < fseq finished (stored, released)
    int bail;
};

// Dynamic shared memory per thread block: a sweep warp's tile and panel
// rows, four warps per block, or a wave block's WaveSmem.
constexpr int kWarpSmemBytes = 10752;
constexpr int kBlockSmemBytes =
    (int)(((sizeof(WaveSmem<double>) > 4 * (size_t)kWarpSmemBytes ? sizeof(WaveSmem<double>)
                                                                   : 4 * (size_t)kWarpSmemBytes) +
           1023) & ~(size_t)1023);
static_assert(sizeof(double) * kW * (kW + 1) + 64 + kW * sizeof(CoefRow<double>) + kW * sizeof(ChainRow) <=
                  (size_t)kWarpSmemBytes,
              "sweep warp shared memory");

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
    __stcg(q + 1, make_double2(c.e1, c.g));
}
__device__ __forceinline__ void st_coef(CoefRow<float> *p, const CoefRow<float> &c)
{
    __stcg(reinterpret_cast<float4 *>(p), make_float4(c.a, c.b, c.e1, c.g));
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

#define CHM_TRACE(pt)                                                               \
    do {                                                                            \
        if (w.trace_sweep && lane == 0)                                             \
            w.trace_sweep[(size_t)b * kTracePoints + (pt)] = global_ns();           \
    } while (0)

// ---------------------------------------------------------------- sweep task

// Column block b of wave w: rotate its off-diagonal tiles (row blocks p < b)
// in order, the block's update vector u_hat held in registers (lane = column).
template <typename T>
__device__ void sweep_task(const Wave<T> &w, int b, unsigned char *sm)
{
    T(*tile)[kW + 1] = reinterpret_cast<T(*)[kW + 1]>(sm);
    CoefRow<T> *cf = reinterpret_cast<CoefRow<T> *>(sm + sizeof(T) * kW * (kW + 1) + 64);
    ChainRow *ch = reinterpret_cast<ChainRow *>(cf + kW);
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = w.sync;
    const long long n = w.n, ld = w.ld;
    const long long c0 = (long long)b * kW;
    const int ncols = (int)min((long long)kW, n - c0);
    const bool active = lane < ncols;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    const long long who = b;
    const long long *prog_prev = w.progress_prev ? w.progress_prev + b : nullptr;
    long long *prog_me = w.progress + b;
    CHM_TRACE(0);

    if (!CHK_RECT(sy, (long long)b, (long long)w.nb, 1, 1 << 30)) return;
    T uh = (active && CHK_RECT(sy, c0 + lane, n, 1, n)) ? w.V[c0 + lane] : T(0);

    if (w.q == 0) {
        // Original-factor data of block b for wave 0: the diagonal and its
        // inverse, the diagonal block's chain ratios, and (b >= 1) the dot
        // product matrix of the tile above, taken before any wave rotates it.
        T x[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c)
            x[c] = (lane <= c && c < ncols && CHK_TRI(sy, c0 + lane + (c0 + c) * ld, n, ld))
                       ? __ldcg(w.L + c0 + lane + (c0 + c) * ld) : T(0);
        double dl = 1.0;
#pragma unroll
        for (int c = 0; c < kW; ++c)
            if (c == lane) dl = (double)x[c];
        const double idl = active ? rcp_refined(dl) : 1.0;
        if (active) st_chain(w.chain0 + (size_t)b * kW + lane, ChainRow{1.0, 1.0, dl, idl});
        double *rd = w.rdiag + (size_t)b * kW * kW;
#pragma unroll
        for (int c = 0; c < kW; ++c) {
            const double v = (lane < c && c < ncols) ? -(double)x[c] * idl : 0.0;
            __stcg(rd + (size_t)lane * kW + c, v);
        }
        if (b >= 1) {
            const long long r0 = c0 - kW;
#pragma unroll
            for (int c = 0; c < kW; ++c)
                x[c] = (c < ncols && CHK_TRI(sy, r0 + lane + (c0 + c) * ld, n, ld))
                           ? __ldcg(w.L + r0 + lane + (c0 + c) * ld) : T(0);
            double *rt = w.rtile + (size_t)(b - 1) * kW * kW;  // tile (b-1, b)
#pragma unroll
            for (int c = 0; c < kW; ++c) __stcg(rt + (size_t)lane * kW + c, -(double)x[c]);
        }
        __syncwarp();
        if (lane == 0) st_release_gpu(w.rflag0 + b, epoch);
    }

    // The shared tile is staged with the next tile right after this tile's
    // stores are issued, when the previous wave has released it, so that its
    // load overlaps the acknowledgement the progress release waits for.
    bool staged = false;
    double tz = 1.0;  // T after block b - 3 (1 before the first block): the scale of the carry z
    for (int p = 0; p < b; ++p) {
        const bool lastTile = p == b - 1;
        if (!staged) {
            // the tile as the previous wave left it, fetched while the panel is pending
            if (prog_prev) CHM_WARP_WAIT(wait_ge(sy, prog_prev, ep64 + p + 1, who));
            T x[kW];
            const long long o = (long long)p * kW + lane;
#pragma unroll
            for (int c = 0; c < kW; ++c)
                x[c] = (c < ncols && CHK_TRI(sy, o + (c0 + c) * ld, n, ld)) ? __ldcg(w.L + o + (c0 + c) * ld) : T(0);
#pragma unroll
            for (int c = 0; c < kW; ++c) tile[c][lane] = x[c];
        }
        CHM_WARP_WAIT(wait_eq(sy, w.pflag + p, epoch, who));
        if (lastTile) CHM_TRACE(1);
        cf[lane] = ld_coef(w.coef + (size_t)p * kW + lane);
        if (lastTile && w.has_next) ch[lane] = ld_chain(w.chain + (size_t)p * kW + lane);
        if (p == b - 3) tz = __ldcg(w.tend + p);
        __syncwarp();
        T S[kW];
#pragma unroll
        for (int r = 0; r < kW; ++r) S[r] = tile[lane][r];
        if (p == b - 2) {
            // the wave block's carry for block b, z after rows < (b - 1) kW, put
            // before this tile's rotations: T u_hat after the rows above the
            // tile, less the tile rows' terms F_rj p_r = g_r S_rj
            T zt = T(0);
#pragma unroll
            for (int r = 0; r < kW; ++r) zt = fma(cf[r].g, S[r], zt);
            put_tagged(w.ztag + ((size_t)b * kW + lane) * 2, active ? tz * (double)uh - (double)zt : 0.0, ep64);
            CHM_TRACE(4);
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                const CoefRow<T> c = cf[r];
                S[r] = fma(c.a, uh, S[r]);
                uh = fma(-c.b, S[r], uh);
            }
        }
        if (lastTile) {  // u_hat entering the diagonal block, for the wave block's rotations there
            put_tagged(w.ctag + ((size_t)b * kW + lane) * 2, active ? (double)uh : 0.0, ep64);
            CHM_TRACE(2);
        }
        if (lastTile && w.has_next) {
            // next wave's dot-product matrix for tile (b-1, b): -S' e'
            double *rt = w.rtile_next + (size_t)(b - 1) * kW * kW;
#pragma unroll
            for (int r = 0; r < kW; ++r)
                __stcg(rt + (size_t)r * kW + lane, active ? -(double)S[r] * ch[r].e1 : 0.0);
        }
        if (active) {
#pragma unroll
            for (int r = 0; r < kW; ++r) tile[lane][r] = S[r];
        }
        __syncwarp();
        {
            const long long o = (long long)p * kW + lane;
#pragma unroll
            for (int c = 0; c < kW; ++c)
                if (c < ncols && CHK_TRI(sy, o + (c0 + c) * ld, n, ld)) __stcg(w.L + o + (c0 + c) * ld, tile[c][lane]);
        }
        __syncwarp();
        staged = false;
        if (p + 1 < b) {
            const int ready = prog_prev ? __shfl_sync(0xffffffffu, ld_acquire_gpu(prog_prev) >= ep64 + p + 2 ? 1 : 0, 0)
                                        : 1;
            if (ready) {
                T x[kW];
                const long long o = (long long)(p + 1) * kW + lane;
#pragma unroll
                for (int c = 0; c < kW; ++c)
                    x[c] = (c < ncols && CHK_TRI(sy, o + (c0 + c) * ld, n, ld)) ? __ldcg(w.L + o + (c0 + c) * ld) : T(0);
#pragma unroll
                for (int c = 0; c < kW; ++c) tile[c][lane] = x[c];
                staged = true;
            }
        }
        __syncwarp();
        if (lane == 0) st_release_gpu(prog_me, ep64 + p + 1);
    }
    CHM_TRACE(3);
}

// ---------------------------------------------------------------- final pass

// Between the waves of a launch an off-diagonal entry is stored as
// S_ij = L_ij / e_i.  After a problem's last wave the true values are
// S_ij e'_i, e'_i the last wave's row scale; this pass multiplies them in,
// tile by tile as the last wave releases each tile, so that the waves
// themselves never spend FP64 issue on it.  (The row scale is taken in the
// storage type, as the rotations' coefficients are.)

// Column block b's off-diagonal tiles, row by row (lane = row).
template <typename T>
__device__ void unscale_task(const Wave<T> &w, int b)
{
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = w.sync;
    const long long n = w.n, ld = w.ld;
    const long long c0 = (long long)b * kW;
    const int ncols = (int)min((long long)kW, n - c0);
    const long long ep64 = (long long)sy.epoch << 32;
    const long long who = b;
    if (!CHK_RECT(sy, (long long)b, (long long)w.nb, 1, 1 << 30)) return;
    for (int p = 0; p < b; ++p) {
        CHM_WARP_WAIT(wait_ge(sy, w.progress_prev + b, ep64 + p + 1, who));
        const T e = (T)__ldcg(&w.chain_in[(size_t)p * kW + lane].e1);
        const long long o = (long long)p * kW + lane;
        T x[kW];
        bool in[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c) in[c] = c < ncols && CHK_TRI(sy, o + (c0 + c) * ld, n, ld);
#pragma unroll
        for (int c = 0; c < kW; ++c) x[c] = in[c] ? __ldcg(w.L + o + (c0 + c) * ld) : T(0);
#pragma unroll
        for (int c = 0; c < kW; ++c)
            if (in[c]) __stcg(w.L + o + (c0 + c) * ld, x[c] * e);
    }
    // count this task done (the pair's wave block waits for all of them);
    // the count word is tagged with the epoch, so it restarts every launch
    fence_acq_rel_gpu();
    __syncwarp();
    if (lane == 0) {
        // lift a count left by an earlier launch to (epoch << 32), then count
        unsigned long long *cnt = reinterpret_cast<unsigned long long *>(w.final_done);
        atomicMax(cnt, (unsigned long long)ep64);
        atomicAdd(cnt, 1ull);
    }
}

// The strictly upper part of the diagonal blocks, after the last wave has
// released each block; block b goes to warp b % 4 of the wave block.
template <typename T>
__device__ void unscale_diag(const Wave<T> &w, int warp)
{
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = w.sync;
    const long long n = w.n, ld = w.ld;
    const int epoch = sy.epoch;
    const long long who = -1;
    for (int b = warp; b < w.nb; b += 4) {
        const long long c0 = (long long)b * kW;
        const int ncols = (int)min((long long)kW, n - c0);
        CHM_WARP_WAIT(wait_eq(sy, w.dflag_prev + b, epoch, who));
        if (lane < ncols) {
            const T e = (T)__ldcg(&w.chain_in[(size_t)b * kW + lane].e1);
            const long long o = c0 + lane;
#pragma unroll
            for (int c = 0; c < kW; ++c)
                if (lane < c && c < ncols && CHK_TRI(sy, o + (c0 + c) * ld, n, ld))
                    __stcg(w.L + o + (c0 + c) * ld, __ldcg(w.L + o + (c0 + c) * ld) * e);
        }
    }
    // the pair is done only when its column tasks are: idle sweep warps stop
    // once every pair is done, so none of those tasks may still be unclaimed
    const int ntasks = w.nb - 1;
    if (warp == 0 && ntasks > 0) {
        const long long want = ((long long)epoch << 32) + ntasks;
        CHM_WARP_WAIT(wait_ge(sy, w.final_done, want, who));
    }
}

// ---------------------------------------------------------------- wave block

#define CHM_WTRACE(b, pt)                                                              \
    do {                                                                               \
        if (w.trace_wave && lane == 0)                                                 \
            w.trace_wave[(size_t)(b) * kTracePoints + (pt)] = global_ns();             \
    } while (0)

// Warp D: the wave block's memory traffic.  It fetches each block's inputs
// for warps A, B and C into slot b % kSlots (up to kSlots - 1 blocks ahead)
// and finishes each block warp C has rotated: the store of the diagonal
// tile and the release of the block to the next wave.  Neither job blocks
// the other: the warp polls both, and the finish is short (the FP64 work of
// a block stays with warp C) so that a fetch on the critical path is not
// held up behind it.
template <typename T>
__device__ void wave_io(const Wave<T> &w, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = w.sync;
    const long long n = w.n, ld = w.ld;
    const int nb = w.nb;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    volatile int *cdone = &S.cdone;
    int next_fetch = 0, next_fin = 0;
    const int nb_end = nb;
    long long idle_since = -1;
    unsigned idle_iters = 0;
    while (next_fin < nb_end) {
        bool progressed = false;
        // finish block next_fin once warp C has rotated it
        if (next_fin < next_fetch && __shfl_sync(FULL, *cdone > next_fin ? 1 : 0, 0)) {
            __threadfence_block();
            const int b = next_fin;
            const long long c0 = (long long)b * kW;
            const int ncols = (int)min((long long)kW, n - c0);
#pragma unroll
            for (int c = 0; c < kW; ++c)
                if (lane <= c && c < ncols && CHK_TRI(sy, c0 + lane + (c0 + c) * ld, n, ld))
                    __stcg(w.L + c0 + lane + (c0 + c) * ld, S.DT[c][lane]);
            __syncwarp();
            if (lane == 0) st_release_gpu(w.dflag + b, epoch);
            CHM_WTRACE(b, 13);
            if (lane == 0) seq_post(&S.fseq, b + 1);
            ++next_fin;
            progressed = true;
        }
        // fetch the inputs of block next_fetch once they are published and its slot is free
        if (next_fetch < nb_end && next_fetch - next_fin < kSlots) {
            const int b = next_fetch, s = b % kSlots;
            int ready = 1;
            if (lane == 0) {
                if (w.q == 0) {
                    ready = ld_relaxed_gpu(w.rflag0 + b) == epoch;
                } else {
                    ready = ld_relaxed_gpu(w.dflag_prev + b) == epoch &&
                            (b == 0 || ld_relaxed_gpu(w.progress_prev + b) >= ep64 + b);
                }
                if (ready) __threadfence();  // acquire what those flags released
            }
            ready = __shfl_sync(FULL, ready, 0);
            // the carry z of the block (b >= 2), from the sweep's tagged words
            double zc = 0.0;
            if (ready && b >= 2) ready = __all_sync(FULL, get_tagged(w.ztag + ((size_t)b * kW + lane) * 2, ep64, &zc));
            if (ready) {
                __syncwarp();
                CHM_WTRACE(b, 2);
                const long long c0 = (long long)b * kW;
                fetch_bytes(&S.R[s][0][0], w.rdiag + (size_t)b * kW * kW, kW * kW * 8, lane);
                if (b >= 1) fetch_bytes(&S.Rt[s][0][0], w.rtile + (size_t)(b - 1) * kW * kW, kW * kW * 8, lane);
                fetch_bytes(&S.rowd[s][0], w.chain_in + (size_t)b * kW, kW * (int)sizeof(ChainRow), lane);
                if (b >= 2) {
                    S.zpart[s][lane] = zc;
                } else {
                    S.zpart[s][lane] = (c0 + lane < n && CHK_RECT(sy, c0 + lane, n, 1, n)) ? (double)w.V[c0 + lane] : 0.0;
                }
                cp_async_commit();
                cp_async_wait();
                __syncwarp();
                CHM_WTRACE(b, 3);
                if (lane == 0) seq_post(&S.dseq, b + 1);
                ++next_fetch;
                progressed = true;
            }
        }
        if (progressed) {
            idle_since = -1;
            idle_iters = 0;
            continue;
        }
        // neither: stop on an abort or a stopped warp, else wait a little (bounded)
        const int stop = __shfl_sync(FULL, (*reinterpret_cast<volatile int *>(&S.bail) || aborted(sy)) ? 1 : 0, 0);
        if (stop) return;
        const long long now = global_ns();
        if (idle_since < 0) {
            idle_since = now;
        } else if (now - idle_since > sy.timeout_ns || ++idle_iters > (1u << 27)) {
            if (lane == 0) {
                record_error(sy, kStatusTimeout, -4);
                S.bail = 1;
            }
            return;
        }
        __nanosleep(32);
    }
}

// Warp A: the forward substitution through each diagonal block.
template <typename T>
__device__ void wave_chain(const Wave<T> &w, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = w.sync;
    const long long who = -1;
    for (int b = 0; b < w.nb; ++b) {
        CHM_SEQ_WAIT(&S.zseq, b + 1);
        CHM_WTRACE(b, 8);
        double(*R)[kW] = S.R[b % kSlots];
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
__device__ void wave_coef(const Wave<T> &w, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = w.sync;
    const long long n = w.n;
    const int nb = w.nb;
    const int epoch = sy.epoch;
    const double sgd = w.sg;
    const long long who = -1;
    double pprev = 0.0;  // p of the block last chained, row `lane`
    double Tend = 1.0, iTend = 1.0;
    int pending = -1;    // block chained (or being chained) but not yet published
    int next = 0;        // next block whose chain input is to be formed
    const int nb_end = nb;
    bool ok = true;
    auto wait_seq = [&](int *seq, int want) -> bool {
        int v = seq_wait(sy, seq, want, &S.bail, who) ? 1 : 0;  // all lanes: see CHM_WARP_WAIT
        v = __shfl_sync(FULL, v, 0);
        __syncwarp();
        return v != 0;
    };
    auto form_input = [&](int b) {
        // z entering block b's chain: the carry plus the rows of the block above
        const int s = b % kSlots;
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
        const int s = b % kSlots;
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
        const CoefRow<T> cr{(T)(sgd * p * rowd.ie1), (T)(p * rowd.e1 * iTn), (T)(rowd.e1 * rc), (T)(p * rowd.e1)};
        const ChainRow nrow{rowd.e1 * rc, rowd.ie1 * c, rowd.d1 * c, rowd.id1 * rc};
        // the block's global row data first: everything warps C and D later
        // release at GPU scope (the next wave's inputs) is ordered after it
        if (active) {
            const size_t prow = (size_t)b * kW + lane;
            st_coef(w.coef + prow, cr);
            st_chain(w.chain + prow, nrow);
        }
        if (lane == 0) __stcg(w.tend + b, Tlast);
        S.cf[s][lane] = cr;
        S.cnew[s][lane] = nrow;
        __syncwarp();
        if (lane == 0) seq_post(&S.bseq, b + 1);
        if (lane == 0 && b != w.skip_publish) st_release_gpu(w.pflag + b, epoch);
        CHM_WTRACE(b, 5);
        Tend = Tlast;
        iTend = __shfl_sync(FULL, iTn, rows - 1);
    };

    while (ok && (next < nb_end || pending >= 0)) {
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
            pprev = (c0 + lane < n) ? S.cbox[lane] * S.rowd[done % kSlots][lane].id1 : 0.0;
        }
        if (next < nb_end) {
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

// Warp C: the wave's rotations inside each diagonal block and the next
// wave's chain ratios of the block; warp D stores the rotated tile.
template <typename T>
__device__ void wave_diag(const Wave<T> &w, WaveSmem<T> &S)
{
    const int lane = threadIdx.x & 31;
    const SyncArgs &sy = w.sync;
    const long long n = w.n, ld = w.ld;
    const int nb = w.nb;
    const int epoch = sy.epoch;
    const long long ep64 = (long long)epoch << 32;
    const long long who = -1;
    for (int b = 0; b < nb; ++b) {
        const int s = b % kSlots;
        const long long c0 = (long long)b * kW;
        const int ncols = (int)min((long long)kW, n - c0);
        const bool active = lane < ncols;
        // u_hat entering the block (from the sweep of its last off-diagonal tile)
        T uh = T(0);
        if (b == 0) {
            uh = (active && CHK_RECT(sy, c0 + lane, n, 1, n)) ? w.V[c0 + lane] : T(0);
        } else {
            double u = 0.0;
            if (!warp_wait_tagged(sy, w.ctag + ((size_t)b * kW + lane) * 2, ep64, who, &u)) return;
            uh = (T)u;
        }
        CHM_WTRACE(b, 10);
        // the tile as the previous wave left it: warp D acquired that wave's
        // release of this block before announcing the block's inputs
        CHM_SEQ_WAIT(&S.dseq, b + 1);
        T x[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c)
            x[c] = (lane <= c && c < ncols && CHK_TRI(sy, c0 + lane + (c0 + c) * ld, n, ld))
                       ? __ldcg(w.L + c0 + lane + (c0 + c) * ld) : T(0);
        // the tile buffer is free once warp D has finished the previous block
        CHM_SEQ_WAIT(&S.fseq, b);
#pragma unroll
        for (int c = 0; c < kW; ++c) S.DT[c][lane] = x[c];
        __syncwarp();
        CHM_WTRACE(b, 11);
        T Sv[kW];
#pragma unroll
        for (int r = 0; r < kW; ++r) Sv[r] = S.DT[lane][r];
        CHM_SEQ_WAIT(&S.bseq, b + 1);
        CHM_WTRACE(b, 12);
#pragma unroll
        for (int r = 0; r < kW; ++r) {
            if (r < lane) {
                const CoefRow<T> c = S.cf[s][r];
                Sv[r] = fma(c.a, uh, Sv[r]);
                uh = fma(-c.b, Sv[r], uh);
            }
        }
#pragma unroll
        for (int r = 0; r < kW; ++r)
            if (r < lane) S.DT[lane][r] = Sv[r];
        const ChainRow cn = S.cnew[s][lane];
        if (active) S.DT[lane][lane] = (T)cn.d1;
        __syncwarp();
        if (w.has_next) {
            // next wave's chain ratios for this block: S'_rc (-e'_r / D'_r), r < c;
            // warp D's release of the block orders these stores for the next wave
            const double f = -cn.e1 * cn.id1;
            double *rd = w.rdiag_next + (size_t)b * kW * kW;
#pragma unroll
            for (int r = 0; r < kW; ++r) {
                const double fr = __shfl_sync(0xffffffffu, f, r);
                __stcg(rd + (size_t)r * kW + lane, (r < lane && active) ? (double)Sv[r] * fr : 0.0);
            }
        }
        if (lane == 0) seq_post(&S.cdone, b + 1);
    }
}

// ---------------------------------------------------------------- entry

// Roles, decided per SM by the first block that starts there.
constexpr int kRoleIdle = 0, kRoleWave = 1, kRoleSweep = 2;
__device__ __forceinline__ int role_code(int role, int group) { return role | (group << 4); }

// Column blocks of pair j that carry sweep tasks: [first, nb); returns the
// pair's ticket word.
template <typename T>
__device__ __forceinline__ unsigned long long *task_range(const Launch<T> &P, int j, int *first, int *nb)
{
    const int i = P.pair_prob ? __ldg(P.pair_prob + j) : 0;
    const Prob *pr = P.probs ? P.probs + i : &P.prob0;
    *first = j > pr->pair0 ? 1 : 0;  // block 0 of a later wave has no off-diagonal tile
    *nb = pr->nb;
    return reinterpret_cast<unsigned long long *>(pr->progress + prob_ticket(pr->nb, pr->k, j - pr->pair0));
}
// Take one sweep task: from the own group's current pair first, then, when
// it has no task left, from another group's pair that is lower than the own
// group's current pair; a warp whose group has no pair yet takes nothing,
// and one whose group takes no more pairs may take from any pair.  A group
// word names the group's current pair; a pair's tasks are handed out by its
// own ticket word, so an increment always yields a task of the pair that
// was looked at (or nothing), whatever the groups do meanwhile.
//
// Why the launch cannot stall: every warp holds only tasks of pairs up to
// its group's current pair (tasks of that pair, or of lower pairs).  A
// pair's tasks wait only on lower pairs, so the lowest running pair's group
// holds tasks of finished pairs (which end without waiting) or of its own
// pair, and its warps always come back to its pair's remaining tasks.
// Without the bound the launch can stall: groups take pairs from the
// counter in one order and name them in another, so warps of the group that
// took pair j but has not named it yet can all take tasks of pair j + 1,
// which wait for pair j's first tasks, which only those warps would take.
// (Seen on the GPU: no task of wave 0 started, every warp held a task of a
// later wave, the launch ended in CHM_ERR_TIMEOUT.)
//
// A ticket word is read first, so that an exhausted pair is not counted up;
// one whose epoch tag is not this launch's is not yet set up and is looked
// at again later.  Returns the pair (or -1) and the column block; all lanes
// get the same answer.
template <typename T>
__device__ __forceinline__ int take_task(const Launch<T> &P, int group, long long ep64, int *block)
{
    const long long *gts = reinterpret_cast<const long long *>(P.ctl + kCtlGroupTicket);
    const int lane = threadIdx.x & 31;
    const long long tagmask = ~0xffffffffll;
    int j = -1, b = -1;
    const unsigned own = (unsigned)((unsigned long long)ld_relaxed_gpu(gts + group) >> 32);  // pair + 1
    if (own == 0u) {  // no pair yet: nothing may be taken
        *block = -1;
        return -1;
    }
    const bool bounded = own != kGroupDone;
    for (int d = 0; d < P.ngroups && j < 0; ++d) {
        int g = group + d;
        if (g >= P.ngroups) g -= P.ngroups;
        const unsigned hi = d == 0 ? own : (unsigned)((unsigned long long)ld_relaxed_gpu(gts + g) >> 32);
        if (hi == 0u || hi == kGroupDone) continue;
        if (d > 0 && bounded && hi >= own) continue;  // only pairs below the own group's
        int first = 0, nb = 0;
        unsigned long long *tk = task_range(P, (int)hi - 1, &first, &nb);
        const long long v = ld_relaxed_gpu(reinterpret_cast<const long long *>(tk));
        if ((v & tagmask) != ep64 || (long long)(unsigned)v + first >= nb) continue;
        long long v2 = 0;
        if (lane == 0) v2 = (long long)atomicAdd(tk, 1ull);
        v2 = __shfl_sync(0xffffffffu, v2, 0);
        if ((v2 & tagmask) == ep64 && (long long)(unsigned)v2 + first < nb) {
            j = (int)hi - 1;
            b = (int)(unsigned)v2 + first;
        }
    }
    *block = b;
    return j;
}

template <typename T>
__global__ void __launch_bounds__(128, 3) wave_kernel(Launch<T> P)
{
    extern __shared__ __align__(16) unsigned char chm_smem[];
    __shared__ int s_role, s_pair, s_last, s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *ctl = P.ctl;
    SyncArgs sy;  // launch-level waits
    sy.abort_flag = ctl + kCtlAbort;
    sy.status = P.status;
    sy.user_info = nullptr;
    sy.epoch = 0;
    sy.timeout_ns = P.timeout_ns;
    sy.chk_cut = P.chk_cut;

    if (threadIdx.x == 0) {
        atomicAdd(ctl + kCtlStarted, 1);
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        int code = role_code(kRoleIdle, 0);
        if (smid < (unsigned)kMaxSm) {
            if (atomicAdd(ctl + kCtlSmSlot + smid, 1) == 0) {
                // the SM's first block: rank the SM; the first G SMs carry the
                // groups' wave blocks, the others are dealt to the groups
                const int r = atomicAdd(ctl + kCtlSmRank, 1);
                const int G = P.ngroups;
                code = r < G ? role_code(kRoleWave, r) : role_code(kRoleSweep, (r - G) % G);
                if (r >= G) atomicAdd(ctl + kCtlGroupSweepers + (r - G) % G, 1);
                st_release_gpu(ctl + kCtlSmRole + smid, code + 1);
            } else {
                const int *pr = ctl + kCtlSmRole + smid;
                int seen = 0;
                bounded_wait(
                    sy, [&] { return (seen = ld_relaxed_gpu(pr)) != 0; },
                    [&] { (void)ld_acquire_gpu(pr); }, -1000);
                code = seen - 1;
                // a wave SM runs its wave block alone
                if (seen == 0 || (code & 15) == kRoleWave) code = role_code(kRoleIdle, 0);
            }
        }
        s_role = code;
    }
    __syncthreads();
    const int role = s_role & 15, group = s_role >> 4;
    unsigned long long *gt = reinterpret_cast<unsigned long long *>(ctl + kCtlGroupTicket) + group;
    // this launch's tag (the epoch changes only when the launch's last block ends)
    const long long ep64 = (long long)ld_relaxed_gpu(ctl + kCtlEpoch) << 32;

    if (role == kRoleWave) {
        WaveSmem<T> &S = *reinterpret_cast<WaveSmem<T> *>(chm_smem);
        if (threadIdx.x == 0) {
            // every block of the launch is resident before pairs are taken,
            // so that the group's sweep SMs are all known
            const bool all = bounded_wait(
                sy, [&] { return ld_relaxed_gpu(ctl + kCtlStarted) >= (int)gridDim.x; },
                [] { __threadfence(); }, -3);
            s_pair = (all && ld_relaxed_gpu(ctl + kCtlGroupSweepers + group) > 0) ? 0 : -1;
        }
        __syncthreads();
        const bool can_run = s_pair == 0;
        for (;;) {
            if (threadIdx.x == 0) {
                int j = -1;
                if (can_run && !aborted(sy)) j = atomicAdd(ctl + kCtlPairNext, 1);
                if (j < 0 || j >= P.npairs) {
                    j = -1;
                    __threadfence();
                    atomicExch(gt, (unsigned long long)kGroupDone << 32);
                } else {
                    // sequence counters count blocks
                    S.dseq = S.zseq = S.cseq = S.bseq = S.cdone = S.fseq = 0;
                    S.bail = 0;
                    // the pair's ticket word starts at this launch's tag before the pair is named
                    int f_ = 0, n_ = 0;
                    st_relaxed_gpu(reinterpret_cast<long long *>(task_range(P, j, &f_, &n_)), ep64);
                    __threadfence();
                    atomicExch(gt, (unsigned long long)(j + 1) << 32);
                }
                s_pair = j;
            }
            __syncthreads();
            const int j = s_pair;
            if (j < 0) break;
            const Wave<T> w = make_wave(P, j);
            if (!w.ok) {
                // a region failed its bounds check (recorded, the launch is aborting)
            } else if (w.unscale) unscale_diag<T>(w, warp);
            else if (warp == 0) wave_chain<T>(w, S);
            else if (warp == 1) wave_coef<T>(w, S);
            else if (warp == 2) wave_diag<T>(w, S);
            else wave_io<T>(w, S);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(ctl + kCtlPairsDone, 1);
            }
        }
    } else if (role == kRoleSweep) {
        unsigned char *sm = chm_smem + (size_t)warp * kWarpSmemBytes;
        long long idle_since = -1;
        unsigned idle_iters = 0;
        for (;;) {
            if (aborted(sy)) break;
            int b = -1;
            const int j = take_task(P, group, ep64, &b);
            if (j >= 0) {
                const Wave<T> w = make_wave(P, j);
                if (!w.ok) break;
                if (w.unscale) unscale_task<T>(w, b);
                else sweep_task<T>(w, b, sm);
                idle_since = -1;
                idle_iters = 0;
                continue;
            }
            // nothing to take: stop once every pair is done, else look again
            if (ld_relaxed_gpu(ctl + kCtlPairsDone) >= P.npairs) break;
            const long long now = global_ns();
            if (idle_since < 0) {
                idle_since = now;
            } else if (now - idle_since > P.timeout_ns || ++idle_iters > (1u << 24)) {
                if (lane == 0) record_error(sy, kStatusTimeout, -2);
                break;
            }
            __nanosleep(500);
        }
    }

    // The last block to finish zeroes the control words for the next launch
    // and advances the epoch.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(ctl + kCtlExited, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        // A wait that ran out aborted the whole launch: every problem that
        // recorded nothing stopped unfinished, so it is marked too (info -5:
        // stopped by another problem's failure) and none reads as complete.
        if (threadIdx.x == 0) s_abort = ld_relaxed_gpu(ctl + kCtlAbort);
        __syncthreads();
        if (s_abort) {
            for (int i = threadIdx.x; i < P.nprobs; i += blockDim.x) {
                long long *info = P.probs ? P.probs[i].info : P.prob0.info;
                if (info) record_one(info, kStatusTimeout, -5);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kCtlInts; i += blockDim.x)
            if (i != kCtlEpoch) ctl[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            ctl[kCtlEpoch] = ctl[kCtlEpoch] + 1;
            __threadfence();
        }
    }
}

#undef CHM_WARP_WAIT
#undef CHM_SEQ_WAIT
#undef CHM_TRACE
#undef CHM_WTRACE

}  // namespace chm
