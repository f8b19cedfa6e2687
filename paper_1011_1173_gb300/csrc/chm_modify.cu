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

template <typename T>
struct ModifyParams {
    T *L;
    long long n, ld;
    const T *V;
    long long ldv;
    int kb;              // vectors in this launch (<= kKB)
    unsigned sign_mask;  // bit q set: vector q is a downdate
    int nblocks;         // column blocks
    T *coef;             // [nblocks][kW][kKB] Coef<T> (row-major)
    SyncArgs sync;
};

template <typename T>
__global__ void __launch_bounds__(kW) modify_wavefront_kernel(ModifyParams<T> prm)
{
    __shared__ __align__(16) Coef<T> pan[kW][kKB];
    const int lane = threadIdx.x;
    const unsigned FULL = 0xffffffffu;
    const SyncArgs &sy = prm.sync;
    const long long n = prm.n, ld = prm.ld;
    const int kb = prm.kb;

    for (;;) {
        int b = 0;
        if (lane == 0) b = atomicAdd(sy.ticket, 1);
        b = __shfl_sync(FULL, b, 0);
        if (b >= prm.nblocks) return;
        if (aborted(sy)) return;

        const long long j = (long long)b * kW + lane;
        const bool active = j < n;
        T u[kKB];
#pragma unroll
        for (int q = 0; q < kKB; ++q)
            u[q] = (active && q < kb) ? prm.V[j + (long long)q * prm.ldv] : T(0);

        // Trailing sweep: rotations of every earlier row panel.
        for (int p = 0; p < b; ++p) {
            int ok = 1;
            if (lane == 0) ok = wait_panel(sy, p, b) ? 1 : 0;
            ok = __shfl_sync(FULL, ok, 0);
            if (!ok) return;
            __syncwarp();
            {
                constexpr int kWords = (int)(sizeof(Coef<T>) * kW * kKB / 16);
                const int4 *src = reinterpret_cast<const int4 *>(prm.coef + (size_t)p * kW * kKB * 4);
                int4 *dst = reinterpret_cast<int4 *>(&pan[0][0]);
                for (int e = lane; e < kWords; e += 32) dst[e] = __ldcg(src + e);
            }
            __syncwarp();
            if (active) {
                T *col = prm.L + j * ld + (long long)p * kW;
                for (int r = 0; r < kW; ++r) {
                    T x = col[r];
#pragma unroll
                    for (int q = 0; q < kKB; ++q) {
                        if (q < kb) {
                            const Coef<T> cf = pan[r][q];
                            apply_rotation(x, u[q], cf.c, cf.s, cf.a, cf.b);
                        }
                    }
                    col[r] = x;
                }
            }
            __syncwarp();
        }

        // Diagonal triangle of block b.
        const int rows = (int)min((long long)kW, n - (long long)b * kW);
        for (int r = 0; r < rows; ++r) {
            const long long i = (long long)b * kW + r;
            if (lane == r) {
                T *dg = prm.L + i + i * ld;
                double l = (double)*dg;
                bool okc = true;
#pragma unroll
                for (int q = 0; q < kKB; ++q) {
                    if (q < kb && okc) {
                        const int sg = ((prm.sign_mask >> q) & 1u) ? -1 : 1;
                        double c, s, a, bb;
                        if (compute_rotation(l, (double)u[q], sg, c, s, a, bb)) {
                            l = (double)(T)l;  // the stored precision of the new diagonal
                            pan[r][q] = Coef<T>{(T)c, (T)s, (T)a, (T)bb};
                        } else {
                            okc = false;
                            record_error(sy, kStatusNotPD, i);
                        }
                    }
                }
                if (okc) *dg = (T)l;
            }
            __syncwarp();
            if (aborted(sy)) return;
            if (active && lane > r) {
                T *e = prm.L + i + j * ld;
                T x = *e;
#pragma unroll
                for (int q = 0; q < kKB; ++q) {
                    if (q < kb) {
                        const Coef<T> cf = pan[r][q];
                        apply_rotation(x, u[q], cf.c, cf.s, cf.a, cf.b);
                    }
                }
                *e = x;
            }
            __syncwarp();
        }

        // Publish this block's panel for the blocks to its right.
        if (b + 1 < prm.nblocks) {
            constexpr int kWords = (int)(sizeof(Coef<T>) * kW * kKB / 16);
            int4 *dst = reinterpret_cast<int4 *>(prm.coef + (size_t)b * kW * kKB * 4);
            const int4 *src = reinterpret_cast<const int4 *>(&pan[0][0]);
            for (int e = lane; e < kWords; e += 32) __stcg(dst + e, src[e]);
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(sy.flags + b, sy.epoch);
        }
        __syncwarp();
    }
}

__global__ void info_init_kernel(long long *info)
{
    info[0] = 0;
    info[1] = -1;
}

// ---------------------------------------------------------------- host side

struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    void *coef = nullptr;
    size_t coef_bytes = 0;
    int *flags = nullptr;
    int nflags = 0;
    int *misc = nullptr;         // [0] ticket, [32] abort (separate cache lines)
    long long *status = nullptr; // {status, info}
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

static int alloc_workspace(Workspace *w, size_t coef_bytes, int nflags)
{
    if (w->coef_bytes >= coef_bytes && w->nflags >= nflags && w->misc) return CHM_OK;
    // Queued work on this stream may still use the old buffers.
    if (cudaStreamSynchronize(w->stream) != cudaSuccess) return CHM_ERR_CUDA;
    if (w->coef_bytes < coef_bytes) {
        cudaFree(w->coef);
        w->coef = nullptr;
        w->coef_bytes = 0;
        if (cudaMalloc(&w->coef, coef_bytes) != cudaSuccess) return CHM_ERR_NOMEM;
        w->coef_bytes = coef_bytes;
    }
    if (w->nflags < nflags) {
        cudaFree(w->flags);
        w->flags = nullptr;
        w->nflags = 0;
        if (cudaMalloc(&w->flags, sizeof(int) * (size_t)nflags) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(w->flags, 0, sizeof(int) * (size_t)nflags) != cudaSuccess) return CHM_ERR_CUDA;
        w->nflags = nflags;
        w->epoch = 0;
    }
    if (!w->misc) {
        if (cudaMalloc(&w->misc, 64 * sizeof(int)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&w->status, 2 * sizeof(long long)) != cudaSuccess) return CHM_ERR_NOMEM;
        const long long init[2] = {0, -1};
        if (cudaMemset(w->misc, 0, 64 * sizeof(int)) != cudaSuccess) return CHM_ERR_CUDA;
        if (cudaMemcpy(w->status, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess)
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

template <typename T>
static int launch_modify(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                         const int8_t *sigma, int sign, cudaStream_t stream, long long *d_info)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    const int nblocks = (int)((n + kW - 1) / kW);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *w = find_workspace(dev, stream, true);
    int rc = alloc_workspace(w, sizeof(T) * 4 * (size_t)kW * kKB * (size_t)nblocks, nblocks);
    if (rc != CHM_OK) return rc;
    if (d_info) info_init_kernel<<<1, 1, 0, stream>>>(d_info);

    static int occ[2][64] = {{0}};
    int &bps = occ[sizeof(T) == 8 ? 0 : 1][dev & 63];
    if (!bps) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, modify_wavefront_kernel<T>, kW, 0);
        if (bps < 1) bps = 1;
    }
    const int grid = std::max(1, std::min(nblocks, sm_count(dev) * bps));

    for (long long q0 = 0; q0 < k; q0 += kKB) {
        const int kb = (int)std::min<long long>(kKB, k - q0);
        unsigned mask = 0;
        for (int q = 0; q < kb; ++q) {
            const int sg = sigma ? sigma[q0 + q] : sign;
            if (sg < 0) mask |= 1u << q;
        }
        // ticket and abort flag start at zero for every launch
        if (cudaMemsetAsync(w->misc, 0, 64 * sizeof(int), stream) != cudaSuccess) return CHM_ERR_CUDA;
        ModifyParams<T> prm;
        prm.L = L;
        prm.n = n;
        prm.ld = ld;
        prm.V = V + q0 * ldv;
        prm.ldv = ldv;
        prm.kb = kb;
        prm.sign_mask = mask;
        prm.nblocks = nblocks;
        prm.coef = static_cast<T *>(w->coef);
        prm.sync.flags = w->flags;
        prm.sync.ticket = w->misc;
        prm.sync.abort_flag = w->misc + 32;
        prm.sync.status = w->status;
        prm.sync.user_info = d_info;
        prm.sync.epoch = ++w->epoch;
        prm.sync.timeout_ns = timeout_ns();
        modify_wavefront_kernel<T><<<grid, kW, 0, stream>>>(prm);
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
    if (n > (1ll << 31) - kW) return CHM_ERR_ARG;
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
            const long long init[2] = {0, -1};
            if (cudaMemcpy(w->status, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess)
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
