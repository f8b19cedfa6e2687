// Rank-k Cholesky up/downdate by hyperbolic rotations on one GPU
// (Walder 2010, Algorithm 1 in the column order of CholeskyModifyA, with the
// panelling of Sec. 4 replaced by a device-resident wavefront).
//
// One launch handles up to kKB update vectors (Sec. 4.1: k / ElementsPerThread
// successive sweeps).  Column block b (columns [b*kW, b*kW + kW)) is owned by
// one thread block, which takes its block index from a ticket counter so that
// a block only ever waits on panels owned by blocks that started earlier.
// For each earlier row panel p it waits for panel p's rotations, then sweeps
// the kW x kW tile (rows of panel p, its own columns) with the update vectors
// held in registers.  It then runs the Compute steps of its own diagonal
// triangle, applies them inside the triangle, and publishes the panel of
// rotations (c, s, 1/c, sigma s/c per row and vector) with a release flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "chm.h"
#include "chm_device.cuh"

namespace chm {

// Sweep coefficients of one row for one wave, in the Apply type T:
//   S' = S + a*u,  u' = u - b*S'  (scaled mixed rotation), e1 = new row scale.
template <typename T>
struct CoefRow {
    T a, b, e1, pad;
};

// Chain data of one row for one wave (always double): ep = e*p (old row
// scale times the forward-substitution value), e1 = new row scale, d1 = new
// diagonal, tn = T after this row.
struct ChainRow {
    double ep, e1, d1, tn;
};

template <typename T>
struct WaveParams {
    T *L;
    long long n, ld;
    const T *V;
    long long ldv;
    int nwaves;                   // update vectors in this launch (<= kMaxWaves)
    int nblocks;                  // column blocks of kW columns
    unsigned long long down_mask; // bit q set: wave q is a downdate
    CoefRow<T> *coef;             // [nwaves][nblocks][kW]
    ChainRow *chain;              // [nwaves][nblocks][kW]
    int *pflag;                   // [nwaves][nblocks]: panel published when == epoch
    long long *progress;          // [nwaves][nblocks]: (epoch << 32) + tiles done
    SyncArgs sync;
};

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

// One task = (wave q, column block b), one warp, lane = column.  Tasks are
// taken in ticket order t = b * nwaves + q, so a task only waits on tasks
// with smaller tickets: (q, p < b) for rotation panels and (q - 1, b) for
// the factor as the previous wave left it.
//
// Storage between waves: the diagonal holds the true L_ii; an off-diagonal
// L_ij (i < j) is stored as S_ij = L_ij / e_i, with e_i the row scale that the
// last wave's panel published (1 at the start).  The last wave of the
// launch stores true values again.
//
// Per wave (rank-1 modification of the current factor F by v, sign sigma):
//   chain:  p = F^{-T} v by forward substitution, T_0 = 1,
//           T_{i+1} = T_i + sigma p_i^2;
//   these give Algorithm 1's c_i = sqrt(T_{i+1}/T_i) and s_i = p_i/sqrt(T_i);
//   sweep:  with u = sqrt(T_i) u_hat, the mixed Apply L' = (L + sigma s u)/c,
//           u' = c u - s L' becomes S' = S + a_i u_hat, u_hat' = u_hat - b_i S'
//           with a_i = sigma p_i / e_i and b_i = p_i e_i / T_{i+1}.
template <typename T>
__global__ void __launch_bounds__(kW) wave_kernel(WaveParams<T> P)
{
    __shared__ T tile[kW][kW + 1];  // [column][row]
    __shared__ CoefRow<T> cf[kW];
    __shared__ double sep[kW];
    const int lane = threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = P.sync;
    const long long n = P.n, ld = P.ld;
    const int nw = P.nwaves, nb = P.nblocks;
    const long long ep64 = (long long)sy.epoch << 32;

    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(sy.ticket, 1);
        t = __shfl_sync(FULL, t, 0);
        if (t >= nw * nb) return;
        if (aborted(sy)) return;
        const int b = t / nw, q = t % nw;
        const int sg = ((P.down_mask >> q) & 1ull) ? -1 : 1;
        const bool last = (q == nw - 1);
        const long long c0 = (long long)b * kW;
        const int ncols = (int)min((long long)kW, n - c0);
        const bool active = lane < ncols;
        const long long j = c0 + lane;
        T uh = active ? P.V[j + (long long)q * P.ldv] : T(0);
        double z = (double)uh;
        const long long *prog_prev = q > 0 ? P.progress + (size_t)(q - 1) * nb + b : nullptr;
        long long *prog_me = P.progress + (size_t)q * nb + b;

        // ---- off-diagonal tiles (p, b), p < b
        for (int p = 0; p < b; ++p) {
            int ok = 1;
            if (lane == 0) {
                const int *pf = P.pflag + (size_t)q * nb + p;
                const int epoch = sy.epoch;
                ok = bounded_wait(sy, [&] { return ld_acquire_gpu(pf) == epoch; }, t);
                if (ok && prog_prev) {
                    const long long want = ep64 + p + 1;
                    ok = bounded_wait(sy, [&] { return ld_acquire_gpu(prog_prev) >= want; }, t);
                }
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) return;
            __syncwarp();
            const bool lastTile = (p == b - 1);
            const size_t prow = ((size_t)q * nb + p) * kW;
            cf[lane] = ld_coef(P.coef + prow + lane);
            double tstart = 1.0;
            if (lastTile) {
                sep[lane] = __ldcg(&P.chain[prow + lane].ep);
                if (p > 0) tstart = __ldcg(&P.chain[prow - 1].tn);
            }
            {
                const T *src = P.L + (long long)p * kW + lane;
                for (int c = 0; c < ncols; ++c) tile[c][lane] = __ldcg(src + (c0 + c) * ld);
            }
            __syncwarp();
            if (active) {
                if (lastTile) {
                    // z = T u (the forward-substitution carry) after the rows
                    // above this tile, then the rows of this tile.
                    double z0 = tstart * (double)uh, z1 = 0.0, z2 = 0.0, z3 = 0.0;
#pragma unroll
                    for (int r = 0; r < kW; r += 4) {
                        z0 = fma(-sep[r], (double)tile[lane][r], z0);
                        z1 = fma(-sep[r + 1], (double)tile[lane][r + 1], z1);
                        z2 = fma(-sep[r + 2], (double)tile[lane][r + 2], z2);
                        z3 = fma(-sep[r + 3], (double)tile[lane][r + 3], z3);
                    }
                    z = (z0 + z1) + (z2 + z3);
                }
#pragma unroll 8
                for (int r = 0; r < kW; ++r) {
                    const CoefRow<T> c = cf[r];
                    const T s = fma(c.a, uh, tile[lane][r]);
                    uh = fma(-c.b, s, uh);
                    tile[lane][r] = last ? s * c.e1 : s;
                }
            }
            __syncwarp();
            {
                T *dst = P.L + (long long)p * kW + lane;
                for (int c = 0; c < ncols; ++c) __stcg(dst + (c0 + c) * ld, tile[c][lane]);
            }
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(prog_me, ep64 + p + 1);
        }

        // ---- diagonal block b
        {
            int ok = 1;
            if (lane == 0 && prog_prev) {
                const long long want = ep64 + b + 1;
                ok = bounded_wait(sy, [&] { return ld_acquire_gpu(prog_prev) >= want; }, t);
            }
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) return;
            __syncwarp();
        }
        const int rows = ncols;
        if (lane < rows) {
            const T *src = P.L + c0 + lane;
            for (int c = lane; c < ncols; ++c) tile[c][lane] = __ldcg(src + (c0 + c) * ld);
        }
        const size_t drow = ((size_t)q * nb + b) * kW;
        double e = 1.0;
        if (q > 0 && lane < rows) e = __ldcg(&P.chain[((size_t)(q - 1) * nb + b) * kW + lane].e1);
        const double T0 = b > 0 ? __ldcg(&P.chain[drow - 1].tn) : 1.0;
        __syncwarp();
        const double D = lane < rows ? (double)tile[lane][lane] : 1.0;
        const double g = e / D;
        // forward substitution through the diagonal block
        for (int r = 0; r < rows; ++r) {
            const double qr = __shfl_sync(FULL, z * g, r);
            if (lane > r && lane < rows) z = fma(-(double)tile[lane][r], qr, z);
        }
        const double pv = lane < rows ? z / D : 0.0;
        double x = lane < rows ? (double)sg * pv * pv : 0.0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double y = __shfl_up_sync(FULL, x, off);
            if (lane >= off) x += y;
        }
        const double Tn = T0 + x;
        double Tp = __shfl_up_sync(FULL, Tn, 1);
        if (lane == 0) Tp = T0;
        const bool bad = lane < rows && !(D > 0.0 && D <= DBL_MAX && Tn > 0.0 && Tn <= DBL_MAX);
        const unsigned badm = __ballot_sync(FULL, bad);
        if (badm && lane == 0) record_error(sy, kStatusNotPD, c0 + (__ffs(badm) - 1));
        const double av = (double)sg * pv / e;
        const double bv = pv * e / Tn;
        const double cc = sqrt(Tn / Tp);
        const double e1 = e / cc;
        const double d1 = D * cc;
        if (lane < rows) {
            st_coef(P.coef + drow + lane, CoefRow<T>{(T)av, (T)bv, (T)e1, T(0)});
            double2 *ch = reinterpret_cast<double2 *>(P.chain + drow + lane);
            __stcg(ch, make_double2(e * pv, e1));
            __stcg(ch + 1, make_double2(d1, Tn));
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_gpu(P.pflag + (size_t)q * nb + b, sy.epoch);

        // the wave's rotations inside the diagonal block
        const T at = (T)av, bt = (T)bv, et = (T)e1;
        for (int r = 0; r < rows; ++r) {
            const T ar = __shfl_sync(FULL, at, r);
            const T br = __shfl_sync(FULL, bt, r);
            const T er = __shfl_sync(FULL, et, r);
            if (lane > r && lane < ncols) {
                const T s = fma(ar, uh, tile[lane][r]);
                uh = fma(-br, s, uh);
                tile[lane][r] = last ? s * er : s;
            }
        }
        if (lane < rows) tile[lane][lane] = (T)d1;
        __syncwarp();
        if (lane < rows) {
            T *dst = P.L + c0 + lane;
            for (int c = lane; c < ncols; ++c) __stcg(dst + (c0 + c) * ld, tile[c][lane]);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_gpu(prog_me, ep64 + b + 1);
    }
}


// ---------------------------------------------------------------- host side

struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    void *coef = nullptr;          // CoefRow panels
    void *chain = nullptr;         // ChainRow panels
    size_t panel_rows = 0;         // capacity of coef/chain in rows
    int *pflag = nullptr;          // panel flags
    long long *progress = nullptr; // progress counters
    size_t nflags = 0;
    int *misc = nullptr;           // [0] ticket, [32] abort (separate cache lines)
    long long *status = nullptr;   // {status, info}
    int epoch = 0;
};

static std::mutex g_mu;
static std::vector<Workspace *> g_ws;

static long long timeout_ns()
{
    static long long v = [] {
        const char *e = getenv("CHM_TIMEOUT_NS");
        long long t = e ? atoll(e) : 0;
        return t > 0 ? t : 4000000000ll;
    }();
    return v;
}

static int sm_count(int dev)
{
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev];
}

static const long long kStatusInit[2] = {0, -1};

static int alloc_workspace(Workspace *w, size_t rows, size_t nflags)
{
    if (w->panel_rows >= rows && w->nflags >= nflags && w->misc) return CHM_OK;
    // Queued work on this stream may still use the old buffers.
    if (cudaStreamSynchronize(w->stream) != cudaSuccess) return CHM_ERR_CUDA;
    if (w->panel_rows < rows) {
        cudaFree(w->coef);
        cudaFree(w->chain);
        w->coef = w->chain = nullptr;
        w->panel_rows = 0;
        if (cudaMalloc(&w->coef, rows * sizeof(CoefRow<double>)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&w->chain, rows * sizeof(ChainRow)) != cudaSuccess) return CHM_ERR_NOMEM;
        w->panel_rows = rows;
    }
    if (w->nflags < nflags) {
        cudaFree(w->pflag);
        cudaFree(w->progress);
        w->pflag = nullptr;
        w->progress = nullptr;
        w->nflags = 0;
        if (cudaMalloc(&w->pflag, sizeof(int) * nflags) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&w->progress, sizeof(long long) * nflags) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(w->pflag, 0, sizeof(int) * nflags) != cudaSuccess) return CHM_ERR_CUDA;
        if (cudaMemset(w->progress, 0, sizeof(long long) * nflags) != cudaSuccess) return CHM_ERR_CUDA;
        w->nflags = nflags;
        w->epoch = 0;
    }
    if (!w->misc) {
        if (cudaMalloc(&w->misc, 64 * sizeof(int)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&w->status, 2 * sizeof(long long)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(w->misc, 0, 64 * sizeof(int)) != cudaSuccess) return CHM_ERR_CUDA;
        if (cudaMemcpy(w->status, kStatusInit, sizeof(kStatusInit), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return CHM_ERR_CUDA;
    }
    return CHM_OK;
}

static Workspace *find_workspace(int dev, cudaStream_t s, bool create)
{
    for (Workspace *w : g_ws)
        if (w->device == dev && w->stream == s) return w;
    if (!create) return nullptr;
    Workspace *w = new Workspace();
    w->device = dev;
    w->stream = s;
    g_ws.push_back(w);
    return w;
}

__global__ void info_init_kernel(long long *info)
{
    info[0] = 0;
    info[1] = -1;
}

template <typename T>
static int launch_modify(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                         const int8_t *sigma, int sign, cudaStream_t stream, long long *d_info)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    const int nblocks = (int)((n + kW - 1) / kW);
    const int wmax = (int)std::min<long long>(k, kMaxWaves);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *w = find_workspace(dev, stream, true);
    int rc = alloc_workspace(w, (size_t)wmax * nblocks * kW, (size_t)wmax * nblocks);
    if (rc != CHM_OK) return rc;
    if (d_info) {
        info_init_kernel<<<1, 1, 0, stream>>>(d_info);
        if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
    }
    static int occ[2][64] = {{0}};
    int &bps = occ[sizeof(T) == 8 ? 0 : 1][dev & 63];
    if (!bps) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, wave_kernel<T>, kW, 0);
        if (bps < 1) bps = 1;
    }
    for (long long q0 = 0; q0 < k; q0 += kMaxWaves) {
        const int nw = (int)std::min<long long>(kMaxWaves, k - q0);
        unsigned long long mask = 0;
        for (int q = 0; q < nw; ++q) {
            const int sg = sigma ? sigma[q0 + q] : sign;
            if (sg < 0) mask |= 1ull << q;
        }
        // ticket and abort flag start at zero for every launch
        if (cudaMemsetAsync(w->misc, 0, 64 * sizeof(int), stream) != cudaSuccess) return CHM_ERR_CUDA;
        WaveParams<T> prm;
        prm.L = L;
        prm.n = n;
        prm.ld = ld;
        prm.V = V + q0 * ldv;
        prm.ldv = ldv;
        prm.nwaves = nw;
        prm.nblocks = nblocks;
        prm.down_mask = mask;
        prm.coef = static_cast<CoefRow<T> *>(w->coef);
        prm.chain = static_cast<ChainRow *>(w->chain);
        prm.pflag = w->pflag;
        prm.progress = w->progress;
        prm.sync.ticket = w->misc;
        prm.sync.abort_flag = w->misc + 32;
        prm.sync.status = w->status;
        prm.sync.user_info = d_info;
        prm.sync.epoch = ++w->epoch;
        prm.sync.timeout_ns = timeout_ns();
        const long long tasks = (long long)nw * nblocks;
        const int grid = (int)std::max(1ll, std::min<long long>(tasks, (long long)sm_count(dev) * bps));
        wave_kernel<T><<<grid, kW, 0, stream>>>(prm);
        if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
    }
    return CHM_OK;
}

static int check_args(const void *L, long long n, long long ld, const void *V, long long ldv,
                      long long k, const int8_t *sigma, int sign, int dtype)
{
    if (n < 0 || k < 0) return CHM_ERR_ARG;
    if (dtype != CHM_F64 && dtype != CHM_F32_MIXED) return CHM_ERR_ARG;
    if (ld < std::max(1ll, n) || ldv < std::max(1ll, n)) return CHM_ERR_ARG;
    if (n > (1ll << 26)) return CHM_ERR_ARG;
    const size_t elt = dtype == CHM_F64 ? 8 : 4;
    if (n > 0 && (!L || ((uintptr_t)L % elt))) return CHM_ERR_ARG;
    if (n > 0 && k > 0 && (!V || ((uintptr_t)V % elt))) return CHM_ERR_ARG;
    if (sigma) {
        for (long long q = 0; q < k; ++q)
            if (sigma[q] != 1 && sigma[q] != -1) return CHM_ERR_ARG;
    } else if (sign != 1 && sign != -1) {
        return CHM_ERR_ARG;
    }
    return CHM_OK;
}

static int modify_dispatch(void *L, long long n, long long ld, const void *V, long long ldv,
                           long long k, const int8_t *sigma, int sign, int dtype,
                           cudaStream_t stream, long long *d_info)
{
    int rc = check_args(L, n, ld, V, ldv, k, sigma, sign, dtype);
    if (rc != CHM_OK) return rc;
    if (n == 0 || k == 0) {
        if (d_info) {
            info_init_kernel<<<1, 1, 0, stream>>>(d_info);
            if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
        }
        return CHM_OK;
    }
    if (dtype == CHM_F64)
        return launch_modify<double>(static_cast<double *>(L), n, ld, static_cast<const double *>(V),
                                     ldv, k, sigma, sign, stream, d_info);
    return launch_modify<float>(static_cast<float *>(L), n, ld, static_cast<const float *>(V), ldv,
                                k, sigma, sign, stream, d_info);
}

}  // namespace chm

extern "C" {

int chm_update(void *L, int64_t n, int64_t ld, const void *V, int64_t k, int dtype,
               chm_stream_t stream)
{
    return chm::modify_dispatch(L, n, ld, V, n > 1 ? n : 1, k, nullptr, 1, dtype, (cudaStream_t)stream,
                                nullptr);
}

int chm_downdate(void *L, int64_t n, int64_t ld, const void *V, int64_t k, int dtype,
                 chm_stream_t stream)
{
    return chm::modify_dispatch(L, n, ld, V, n > 1 ? n : 1, k, nullptr, -1, dtype, (cudaStream_t)stream,
                                nullptr);
}

int chm_modify_ex(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k,
                  const int8_t *sigma, int sign, int dtype, chm_stream_t stream, int64_t *d_info)
{
    return chm::modify_dispatch(L, n, ld, V, ldv, k, sigma, sign, dtype, (cudaStream_t)stream,
                                reinterpret_cast<long long *>(d_info));
}

int chm_status_sync(chm_stream_t stream, int64_t *info)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return CHM_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    long long h[2] = {0, -1};
    {
        std::lock_guard<std::mutex> lock(chm::g_mu);
        chm::Workspace *w = chm::find_workspace(dev, (cudaStream_t)stream, false);
        if (w && w->status) {
            if (cudaMemcpy(h, w->status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
                return CHM_ERR_CUDA;
            if (cudaMemcpy(w->status, chm::kStatusInit, sizeof(chm::kStatusInit),
                           cudaMemcpyHostToDevice) != cudaSuccess)
                return CHM_ERR_CUDA;
        }
    }
    if (info) {
        info[0] = h[0];
        info[1] = h[1];
    }
    return (int)h[0];
}

const char *chm_status_string(int status)
{
    switch (status) {
    case CHM_OK: return "CHM_OK";
    case CHM_ERR_ARG: return "CHM_ERR_ARG: invalid argument";
    case CHM_ERR_NOT_PD: return "CHM_ERR_NOT_PD: modified matrix not positive definite";
    case CHM_ERR_TIMEOUT: return "CHM_ERR_TIMEOUT: a wait between thread blocks ran out of time";
    case CHM_ERR_CUDA: return "CHM_ERR_CUDA: CUDA runtime error";
    case CHM_ERR_NOMEM: return "CHM_ERR_NOMEM: device allocation failed";
    case CHM_ERR_BUDGET: return "CHM_ERR_BUDGET: memory budget exceeded";
    case CHM_ERR_STATE: return "CHM_ERR_STATE: invalid object state";
    default: return "unknown status";
    }
}

int chm_version(void) { return 100; }

}  // extern "C"
