// Device-side helpers shared by the up/downdate kernels: inter-block flags,
// bounded waits, the sticky status word, and the two steps of Algorithm 1
// (Compute and Apply) in the forms the kernels evaluate.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

namespace chm {

// Columns per column block == rows per published rotation panel.
constexpr int kW = 32;
// Update vectors handled by one launch (the k-column block of Sec. 4.1).
constexpr int kKB = 16;

// Device status codes (mirror chm_status in chm.h).
constexpr long long kStatusNotPD = -2;
constexpr long long kStatusTimeout = -3;

// Everything the blocks of one launch use to order themselves.
struct SyncArgs {
    int *flags;            // [npanels]: panel p is published when flags[p] == epoch
    int *ticket;           // column-block ticket counter, zero at launch
    int *abort_flag;       // non-zero once any block has recorded an error
    long long *status;     // sticky {status, info} of the (device, stream)
    long long *user_info;  // optional per-call {status, info}
    int epoch;
    long long timeout_ns;  // bound on any single wait
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First error wins; the winner also raises the abort flag so that every
// other block stops waiting.
__device__ __forceinline__ void record_error(const SyncArgs &s, long long code, long long info)
{
    unsigned long long *st = reinterpret_cast<unsigned long long *>(s.status);
    if (atomicCAS(st, 0ull, (unsigned long long)code) == 0ull)
        atomicExch(reinterpret_cast<unsigned long long *>(s.status + 1), (unsigned long long)info);
    if (s.user_info) {
        unsigned long long *ui = reinterpret_cast<unsigned long long *>(s.user_info);
        if (atomicCAS(ui, 0ull, (unsigned long long)code) == 0ull)
            atomicExch(ui + 1, (unsigned long long)info);
    }
    atomicExch(s.abort_flag, 1);
}

__device__ __forceinline__ bool aborted(const SyncArgs &s) { return ld_relaxed_gpu(s.abort_flag) != 0; }

// Wait (one thread) until panel p carries this launch's epoch.  Returns
// false if the launch is being aborted or the wait ran out of time (which
// is then recorded as CHM_ERR_TIMEOUT with info = the waiting block).
__device__ __noinline__ bool wait_panel(const SyncArgs &s, int p, int waiter)
{
    const long long t0 = global_ns();
    for (unsigned it = 1;; ++it) {
        if (ld_acquire_gpu(s.flags + p) == s.epoch) return true;
        if ((it & 63u) == 0u) {
            if (aborted(s)) return false;
            if (global_ns() - t0 > s.timeout_ns || it > (1u << 28)) {
                record_error(s, kStatusTimeout, waiter);
                return false;
            }
        }
        __nanosleep(20);
    }
}

// Rotation coefficients of one (row, vector) pair, in the type the Apply
// sweep computes in: c and s of Algorithm 1, a = 1/c and b = sigma*s/c.
template <typename T>
struct Coef {
    T c, s, a, b;
};

// Algorithm 1, "Compute", always in double: w = sqrt(l^2 + sigma v^2),
// c = w / l, s = v / l, l <- w; also a = 1/c = l/w and b = sigma s / c =
// sigma v / w, so that Apply needs no division.  Returns false when the
// modified matrix is not positive definite at this row (l <= 0, or
// l^2 + sigma v^2 <= 0, or a non-finite value).
__device__ __forceinline__ bool compute_rotation(double &l, double v, int sigma, double &c,
                                                 double &s, double &a, double &b)
{
    if (!(l > 0.0 && l <= DBL_MAX)) return false;
    const double t = fma((double)sigma * v, v, l * l);
    if (!(t > 0.0 && t <= DBL_MAX)) return false;
    const double w = sqrt(t);
    c = w / l;
    s = v / l;
    a = l / w;
    b = (double)sigma * v / w;
    l = w;
    return true;
}

// Algorithm 1, "Apply": L_ij <- (L_ij + sigma s V_j) / c = a L_ij + b V_j,
// then V_j <- c V_j - s L_ij with the NEW L_ij.
template <typename T>
__device__ __forceinline__ void apply_rotation(T &x, T &u, T c, T s, T a, T b)
{
    const T xn = fma(b, u, a * x);
    u = fma(-s, xn, c * u);
    x = xn;
}

}  // namespace chm
