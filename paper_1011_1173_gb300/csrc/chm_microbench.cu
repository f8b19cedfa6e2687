// Microbenchmarks of the hardware facts the up/downdate kernel is designed
// around (chm_microbench in chm.h): FP64 and FP32 FMA rates, the FP64 issue
// rate of one warp, the dependent FP64 FMA latency, a shuffle chain in a
// converged warp and after a wait that lane 0 ran alone, HBM copy bandwidth
// and the round trip of a flag between two thread blocks.  Every wait is
// bounded.  Diagnostics only; no part of the up/downdate calls these.
#include <cuda_runtime.h>

#include <algorithm>

#include "chm.h"
#include "chm_device.cuh"

namespace chm {
namespace {

constexpr unsigned FULL = 0xffffffffu;

// Independent FMA chains (8 per thread), `iters` steps each.
template <typename T>
__global__ void fma_rate(T *out, int iters)
{
    T a0 = (T)threadIdx.x * (T)1e-9, a1 = a0 + (T)1e-9, a2 = a0 + (T)2e-9, a3 = a0 + (T)3e-9;
    T a4 = a0 + (T)4e-9, a5 = a0 + (T)5e-9, a6 = a0 + (T)6e-9, a7 = a0 + (T)7e-9;
    const T m = (T)0.9999999 + (T)out[0] * (T)1e-30, c = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
        a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
        a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
    }
    out[1 + (blockIdx.x * blockDim.x + threadIdx.x) % 1024] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// One warp: `iters` rounds of 8 independent FP64 FMAs (issue rate), or one
// dependent chain (latency); cycles per instruction in cyc[0].
__global__ void fp64_warp(double *out, long long *cyc, int iters, int dependent)
{
    double a0 = 1.0 + threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5,
           a6 = a0 + 6, a7 = a0 + 7;
    const double m = 0.999999 + out[0] * 1e-30, c = 1e-9;
    __syncwarp();
    const long long t0 = clock64();
    if (dependent) {
        for (int i = 0; i < iters; ++i) a0 = fma(a0, m, c);
    } else {
        for (int i = 0; i < iters; ++i) {
            a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
            a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
        }
    }
    const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    const long long t1 = clock64() + (s == 12345.0 ? 1 : 0);
    out[1 + threadIdx.x] = s;
    if (threadIdx.x == 0) cyc[0] = t1 - t0;
}

// Warps of one block running dependent FP64 FMA chains on their first
// `active` lanes; cycles per instruction of warp w in cyc[w].
__global__ void fp64_lanes(double *out, long long *cyc, int iters, int active)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a0 = 1.0 + threadIdx.x * 1e-3;
    const double m = 0.999999 + out[0] * 1e-30, c = 1e-9;
    __syncwarp();
    const long long t0 = clock64();
    if (lane < active)
        for (int i = 0; i < iters; ++i) a0 = fma(a0, m, c);
    __syncwarp();
    const long long t1 = clock64() + (a0 == 12345.0 ? 1 : 0);
    out[1 + threadIdx.x] = a0;
    if (lane == 0) cyc[warp] = t1 - t0;
}

// The shape of wait that split warps in an earlier version of the kernel: a
// poll loop with early returns, run by lane 0 alone, whose verdict the warp
// then takes by shuffle.
__device__ __noinline__ bool lane_wait(volatile int *flag, volatile int *bail)
{
    if (*flag) {
        __threadfence_block();
        return true;
    }
    for (unsigned it = 1;; ++it) {
        __nanosleep(8);
        if (*flag) {
            __threadfence_block();
            return true;
        }
        if ((it & 255u) == 0u && (*bail || it > (1u << 22))) return false;
    }
}

// A chain of 32 dependent shuffles, timed in a warp that is converged and
// again after lane 0 alone has run such a wait on a shared flag (set by warp 1).
__global__ void shfl_after_wait(long long *cyc, int *out, int reps)
{
    __shared__ volatile int flag, bail;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) flag = bail = 0;
    __syncthreads();
    if (warp == 1) {
        __nanosleep(2000);
        flag = 1;
        return;
    }
    int v = lane;
    long long conv = 0, split = 0;
    for (int r = 0; r < reps; ++r) {
        __syncwarp();
        long long t0 = clock64();
#pragma unroll
        for (int i = 0; i < 32; ++i) v = __shfl_sync(FULL, v, (v + 1) & 31);
        conv += clock64() - t0 + (v == 12345 ? 1 : 0);
    }
    int ok = 1;
    if (lane == 0) ok = lane_wait(&flag, &bail) ? 1 : 0;
    if (!__shfl_sync(FULL, ok, 0)) {
        if (lane == 0) cyc[0] = cyc[1] = -1;
        return;
    }
    __syncwarp();
    for (int r = 0; r < reps; ++r) {
        __syncwarp();
        long long t0 = clock64();
#pragma unroll
        for (int i = 0; i < 32; ++i) v = __shfl_sync(FULL, v, (v + 1) & 31);
        split += clock64() - t0 + (v == 12345 ? 1 : 0);
    }
    out[lane] = v;
    if (lane == 0) {
        cyc[0] = conv / reps;
        cyc[1] = split / reps;
    }
}

__global__ void copy_kernel(const double2 *src, double2 *dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        __stcs(dst + i, __ldcs(src + i));
}

// Two blocks pass a token back and forth `rounds` times through global
// flags (release / acquire); every wait is bounded by an iteration cap.
__global__ void ping_pong(int *flags, int rounds, long long *ns, int *failed)
{
    if (threadIdx.x != 0) return;
    const int me = blockIdx.x;
    long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int r = 0; r < rounds; ++r) {
        if (me == 0) {
            asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flags), "r"(2 * r + 1) : "memory");
        }
        const int want = me == 0 ? 2 * r + 2 : 2 * r + 1;
        int v = 0;
        unsigned it = 0;
        do {
            asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(flags) : "memory");
        } while (v < want && ++it < (1u << 20));
        if (v < want) {
            *failed = 1;
            return;
        }
        if (me == 1) {
            asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(flags), "r"(2 * r + 2) : "memory");
        }
    }
    long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (me == 0) *ns = t1 - t0;
}

float time_ms(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

// The library's reciprocal and reciprocal square root (chm_device.cuh) of
// each x, beside CUDA's IEEE-rounded 1 / x and 1 / sqrt(x).
__global__ void reciprocals(const double *x, long long count, double *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        out[4 * i] = rcp_refined(v);
        out[4 * i + 1] = rsqrt_refined(v);
        out[4 * i + 2] = 1.0 / v;
        out[4 * i + 3] = 1.0 / sqrt(v);
    }
}

}  // namespace
}  // namespace chm

extern "C" int chm_selftest_reciprocals(const double *x, int64_t count, double *out)
{
    using namespace chm;
    if (count < 0 || (count > 0 && (!x || !out))) return CHM_ERR_ARG;
    if (count == 0) return CHM_OK;
    double *dx = nullptr, *dout = nullptr;
    int rc = CHM_OK;
    if (cudaMalloc(&dx, (size_t)count * 8) != cudaSuccess || cudaMalloc(&dout, (size_t)count * 32) != cudaSuccess)
        rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && cudaMemcpy(dx, x, (size_t)count * 8, cudaMemcpyHostToDevice) != cudaSuccess) rc = CHM_ERR_CUDA;
    if (rc == CHM_OK) {
        const int grid = (int)std::min<long long>(1024, (count + 255) / 256);
        reciprocals<<<grid, 256>>>(dx, (long long)count, dout);
        if (cudaGetLastError() != cudaSuccess) rc = CHM_ERR_CUDA;
    }
    if (rc == CHM_OK && cudaMemcpy(out, dout, (size_t)count * 32, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = CHM_ERR_CUDA;
    cudaFree(dx);
    cudaFree(dout);
    return rc;
}

extern "C" int chm_microbench(int which, double *out, int nout)
{
    using namespace chm;
    if (!out || nout < 2) return CHM_ERR_ARG;
    int dev = 0, nsm = 0, clk_khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int rc = CHM_OK;
    out[0] = out[1] = 0.0;
    switch (which) {
    case CHM_MB_FP64_RATE:
    case CHM_MB_FP32_RATE: {
        const bool f64 = which == CHM_MB_FP64_RATE;
        void *buf = nullptr;
        if (cudaMalloc(&buf, 8 * 1025) != cudaSuccess) { rc = CHM_ERR_NOMEM; break; }
        cudaMemset(buf, 0, 8 * 1025);
        const int grid = nsm * 8, block = 256, iters = f64 ? 2000 : 100000;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(a);
            if (f64) fma_rate<double><<<grid, block>>>(static_cast<double *>(buf), iters);
            else fma_rate<float><<<grid, block>>>(static_cast<float *>(buf), iters);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
        }
        const double fmas = (double)grid * block * iters * 8;
        out[0] = fmas / (time_ms(a, b) * 1e-3) / 1e12;  // T FMA/s (lane operations)
        out[1] = out[0] / nsm;
        cudaFree(buf);
        break;
    }
    case CHM_MB_FP64_WARP: {
        double *buf = nullptr;
        long long *cyc = nullptr;
        if (cudaMalloc(&buf, 8 * 64) != cudaSuccess || cudaMalloc(&cyc, 16) != cudaSuccess) { rc = CHM_ERR_NOMEM; break; }
        cudaMemset(buf, 0, 8 * 64);
        long long h = 0;
        const int iters = 4096;
        fp64_warp<<<1, 32>>>(buf, cyc, iters, 0);
        cudaMemcpy(&h, cyc, 8, cudaMemcpyDeviceToHost);
        out[0] = (double)h / (iters * 8.0);  // cycles per FP64 instruction, independent (issue)
        fp64_warp<<<1, 32>>>(buf, cyc, iters, 1);
        cudaMemcpy(&h, cyc, 8, cudaMemcpyDeviceToHost);
        out[1] = (double)h / iters;  // cycles per FP64 instruction, dependent (latency)
        cudaFree(buf);
        cudaFree(cyc);
        break;
    }
    case CHM_MB_FP64_LANES: {
        double *buf = nullptr;
        long long *cyc = nullptr;
        if (cudaMalloc(&buf, 8 * (1 + 128)) != cudaSuccess || cudaMalloc(&cyc, 4 * 8) != cudaSuccess) { rc = CHM_ERR_NOMEM; break; }
        cudaMemset(buf, 0, 8 * (1 + 128));
        long long h[4] = {0, 0, 0, 0};
        const int iters = 4096;
        fp64_lanes<<<1, 32>>>(buf, cyc, iters, 1);
        cudaMemcpy(h, cyc, 8, cudaMemcpyDeviceToHost);
        out[0] = (double)h[0] / iters;  // one warp, one active lane
        fp64_lanes<<<1, 128>>>(buf, cyc, iters, 32);
        cudaMemcpy(h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
        out[1] = (double)std::max(std::max(h[0], h[1]), std::max(h[2], h[3])) / iters;  // four warps, one SM
        cudaFree(buf);
        cudaFree(cyc);
        break;
    }
    case CHM_MB_SHFL_SPLIT: {
        long long *cyc = nullptr;
        int *ob = nullptr;
        if (cudaMalloc(&cyc, 16) != cudaSuccess || cudaMalloc(&ob, 128) != cudaSuccess) { rc = CHM_ERR_NOMEM; break; }
        shfl_after_wait<<<1, 64>>>(cyc, ob, 64);
        long long h[2] = {0, 0};
        cudaMemcpy(h, cyc, 16, cudaMemcpyDeviceToHost);
        out[0] = (double)h[0];  // cycles, 32-deep shuffle chain, converged warp
        out[1] = (double)h[1];  // the same after a wait run by lane 0 alone
        cudaFree(cyc);
        cudaFree(ob);
        break;
    }
    case CHM_MB_HBM_COPY: {
        const size_t bytes = (size_t)2 << 30;
        void *s = nullptr, *d = nullptr;
        if (cudaMalloc(&s, bytes) != cudaSuccess || cudaMalloc(&d, bytes) != cudaSuccess) {
            cudaFree(s);
            rc = CHM_ERR_NOMEM;
            break;
        }
        cudaMemset(s, 0, bytes);
        const size_t n = bytes / sizeof(double2);
        float best = 1e30f;
        for (int rep = 0; rep < 5; ++rep) {
            cudaEventRecord(a);
            copy_kernel<<<nsm * 8, 512>>>(static_cast<const double2 *>(s), static_cast<double2 *>(d), n);
            cudaEventRecord(b);
            cudaEventSynchronize(b);
            if (rep > 0 && time_ms(a, b) < best) best = time_ms(a, b);
        }
        out[0] = 2.0 * bytes / (best * 1e-3) / 1e9;  // GB/s, read + write
        out[1] = best;
        cudaFree(s);
        cudaFree(d);
        break;
    }
    case CHM_MB_FLAG_ROUND_TRIP: {
        int *flags = nullptr, *failed = nullptr;
        long long *ns = nullptr;
        if (cudaMalloc(&flags, 256) != cudaSuccess || cudaMalloc(&failed, 4) != cudaSuccess ||
            cudaMalloc(&ns, 8) != cudaSuccess) {
            rc = CHM_ERR_NOMEM;
            break;
        }
        cudaMemset(flags, 0, 256);
        cudaMemset(failed, 0, 4);
        const int rounds = 1000;
        ping_pong<<<2, 32>>>(flags, rounds, ns, failed);
        long long h = 0;
        int f = 0;
        cudaMemcpy(&h, ns, 8, cudaMemcpyDeviceToHost);
        cudaMemcpy(&f, failed, 4, cudaMemcpyDeviceToHost);
        out[0] = f ? -1.0 : (double)h / rounds / 1e3;  // microseconds per round trip
        out[1] = (double)f;
        cudaFree(flags);
        cudaFree(failed);
        cudaFree(ns);
        break;
    }
    default:
        rc = CHM_ERR_ARG;
    }
    if (rc == CHM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = CHM_ERR_CUDA;
    if (rc == CHM_OK && cudaGetLastError() != cudaSuccess) rc = CHM_ERR_CUDA;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    (void)clk_khz;
    return rc;
}
