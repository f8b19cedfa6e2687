// Device-side helpers shared by the up/downdate kernels: inter-block flags,
// bounded waits and the sticky status word.
#pragma once

#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

namespace chm {

// Device status codes (mirror chm_status in chm.h).
constexpr long long kStatusNotPD = -2;
constexpr long long kStatusTimeout = -3;
constexpr long long kStatusBounds = -8;

// What a waiting or failing thread needs: the launch's abort flag and
// status words, and the epoch that tags this launch's flags.
struct SyncArgs {
    int *abort_flag;       // non-zero once a block has timed out
    long long *status;     // sticky {status, info} of the scratch owner
    long long *user_info;  // optional {status, info} of the problem
    int epoch;             // distinguishes this launch's flags from older ones
    long long timeout_ns;  // bound on any single wait
    long long chk_cut;     // bounds-checked build: columns taken off a factor's declared extent
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long ld_acquire_gpu(const long long *p)
{
    long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_release_gpu(long long *p, long long v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(int *p, int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void st_relaxed_gpu(long long *p, long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Orders this thread's earlier loads and stores before its later ones at GPU scope.
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ int ld_relaxed_gpu(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long ld_relaxed_gpu(const long long *p)
{
    long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool aborted(const SyncArgs &s) { return ld_relaxed_gpu(s.abort_flag) != 0; }

// Record a device-side error.  The first code wins; for CHM_ERR_NOT_PD the
// smallest row wins, so that the reported row does not depend on the order
// in which blocks reach their rows.  A timeout also raises the abort flag;
// a failed Compute step does not (the run continues so that every row is
// examined, and the result is unspecified).
__device__ __forceinline__ void record_one(long long *w, long long code, long long info)
{
    unsigned long long *st = reinterpret_cast<unsigned long long *>(w);
    const unsigned long long prev = atomicCAS(st, 0ull, (unsigned long long)code);
    // info starts at -1, the largest value as unsigned, so the minimum over
    // recorded rows replaces it
    if (prev == 0ull || prev == (unsigned long long)code)
        atomicMin(reinterpret_cast<unsigned long long *>(w + 1), (unsigned long long)info);
}

__device__ __forceinline__ void record_error(const SyncArgs &s, long long code, long long info)
{
    record_one(s.status, code, info);
    if (s.user_info) record_one(s.user_info, code, info);
    if (code == kStatusTimeout || code == kStatusBounds) atomicExch(s.abort_flag, 1);
}

// Bounds checks.  A library built with -DCHM_CHECK passes every global
// access of the factor L, the update vectors V and the right-hand sides B
// through these predicates, and every workspace region a kernel derives
// through chk_region.  An index outside what the call's arguments declare
// (L: the upper triangle of the leading n x n block with leading dimension
// ld; V, B: the leading n rows of their k or nrhs columns) records
// CHM_ERR_BOUNDS with info = the element's offset from the array's base (for
// a region, the region's byte offset from its allocation), raises the abort
// flag so that every wait of the launch ends, and makes the caller skip the
// access: nothing traps and nothing outside the arrays is touched.
// chk_cut > 0 (a test setting) takes that many columns off the factor's
// declared extent, so that accesses to real, valid memory are reported.
// Without -DCHM_CHECK the predicates are the constant true.
#ifdef CHM_CHECK
static __device__ __noinline__ bool chk_fail(const SyncArgs &s, long long where)
{
    record_error(s, kStatusBounds, where < 0 ? 0x7fffffffffffffffll : where);
    return false;
}
// element `off` of an upper-triangular factor of order n, leading dimension ld
__device__ __forceinline__ bool chk_tri(const SyncArgs &s, long long off, long long n, long long ld)
{
    if (off >= 0 && ld > 0) {
        const long long j = off / ld, i = off - j * ld;
        if (i <= j && j < n - s.chk_cut) return true;
    }
    return chk_fail(s, off);
}
// element `off` of a column-major rows x cols array, leading dimension ld
__device__ __forceinline__ bool chk_rect(const SyncArgs &s, long long off, long long rows, long long cols,
                                         long long ld)
{
    if (off >= 0 && ld > 0) {
        const long long j = off / ld, i = off - j * ld;
        if (i < rows && j < cols) return true;
    }
    return chk_fail(s, off);
}
// bytes [p, p + bytes) inside the allocation [lo, lo + size)
__device__ __forceinline__ bool chk_region(const SyncArgs &s, const void *p, size_t bytes, const void *lo,
                                           size_t size)
{
    const char *a = static_cast<const char *>(p), *b = static_cast<const char *>(lo);
    if (a >= b && (size_t)(a - b) <= size && bytes <= size - (size_t)(a - b)) return true;
    return chk_fail(s, (long long)(a - b));
}
#define CHK_TRI(s, off, n, ld) ::chm::chk_tri((s), (off), (n), (ld))
#define CHK_RECT(s, off, rows, cols, ld) ::chm::chk_rect((s), (off), (rows), (cols), (ld))
#define CHK_REGION(s, p, bytes, lo, size) ::chm::chk_region((s), (p), (bytes), (lo), (size))
#else
#define CHK_TRI(s, off, n, ld) true
#define CHK_RECT(s, off, rows, cols, ld) true
#define CHK_REGION(s, p, bytes, lo, size) true
#endif

// One thread waits until ready() holds.  ready() polls with relaxed loads
// (cheap, no ordering) under exponential backoff up to max_ns between polls
// (the sleep is a hint the hardware may shorten); once it holds, acquire()
// performs the single acquiring load that orders this thread's later reads
// after the writer's release.  Returns false if the launch is being aborted
// or the wait ran out of time (then recorded as CHM_ERR_TIMEOUT, info = who).
template <typename F, typename A>
__device__ __forceinline__ bool bounded_wait(const SyncArgs &s, F ready, A acquire, long long who,
                                             unsigned max_ns = 256)
{
    if (ready()) {
        acquire();
        return true;
    }
    const long long t0 = global_ns();
    unsigned ns = 16;
    for (unsigned it = 1;; ++it) {
        __nanosleep(ns);
        if (ns < max_ns) ns <<= 1;
        if (ready()) {
            acquire();
            return true;
        }
        if ((it & 15u) == 0u) {
            if (aborted(s)) return false;
            if (global_ns() - t0 > s.timeout_ns || it > (1u << 26)) {
                record_error(s, kStatusTimeout, who);
                return false;
            }
        }
    }
}

// Wait helpers.
__device__ __forceinline__ bool wait_eq(const SyncArgs &s, const int *p, int want, long long who)
{
    return bounded_wait(s, [&] { return ld_acquire_gpu(p) == want; }, [] {}, who);
}
__device__ __forceinline__ bool wait_ge(const SyncArgs &s, const long long *p, long long want,
                                        long long who)
{
    return bounded_wait(s, [&] { return ld_acquire_gpu(p) >= want; }, [] {}, who);
}


// Reciprocal and reciprocal square root of a double to within 1 ulp (checked
// against IEEE division and square root over the whole exponent range by
// chm_selftest_reciprocals): the hardware's coarse approximations refined by
// one third-order Newton-Raphson (Householder) step,
//   1/x:       e = 1 - x y,    y' = y (1 + e + e^2),
//   1/sqrt(x): e = 1 - x y^2,  y' = y (1 + e/2 + 3 e^2 / 8).
// The PTX seeds exist only in a flush-to-zero form, which treats a subnormal
// input as zero (and would flush a subnormal result): outside
// [2^-1020, 2^1020] the IEEE quotient and square root are taken instead, so
// no input is flushed.  That branch is never taken by normal data.
__device__ __forceinline__ double rcp_refined(double x)
{
    const double ax = fabs(x);
    if (!(ax >= 0x1p-1020 && ax <= 0x1p1020)) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    const double t = fma(e, e, e);
    return fma(y, t, y);
}
__device__ __forceinline__ double rsqrt_refined(double x)
{
    if (!(x >= 0x1p-1020 && x <= 0x1p1020)) return 1.0 / sqrt(x);
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double xy = x * y;
    const double e = fma(-xy, y, 1.0);
    const double h = fma(0.375, e, 0.5);
    return fma(y * e, h, y);
}

// A double published as two tagged words, (epoch << 32) | high half and
// (epoch << 32) | low half: each 8-byte store is single-copy atomic, so a
// reader that sees both tags equal to the current epoch has the value, and
// the writer needs no fence or flag.
__device__ __forceinline__ void put_tagged(long long *w2, double v, long long ep64)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    __stcg(w2, ep64 | (long long)(u >> 32));
    __stcg(w2 + 1, ep64 | (long long)(u & 0xffffffffull));
}
// Read a tagged double: true (and *v) once both words carry `ep64`.
__device__ __forceinline__ bool get_tagged(const long long *w2, long long ep64, double *v)
{
    const long long h = ld_relaxed_gpu(w2), l = ld_relaxed_gpu(w2 + 1);
    if ((h & ~0xffffffffll) != ep64 || (l & ~0xffffffffll) != ep64) return false;
    *v = __longlong_as_double((long long)(((unsigned long long)h << 32) | ((unsigned long long)l & 0xffffffffull)));
    return true;
}

// The whole warp waits (bounded) until every lane's tagged double carries
// `ep64`; every exit is decided for the warp as a whole.  Returns false if
// the launch is being aborted or the wait ran out of time (recorded).
__device__ __forceinline__ bool warp_wait_tagged(const SyncArgs &s, const long long *w2, long long ep64,
                                                 long long who, double *v)
{
    const long long t0 = global_ns();
    unsigned ns = 16;
    for (unsigned it = 0;; ++it) {
        if (__all_sync(0xffffffffu, get_tagged(w2, ep64, v))) return true;
        if ((it & 15u) == 15u) {
            const int lane = threadIdx.x & 31;
            int stop = 0;
            if (lane == 0) {
                if (aborted(s)) {
                    stop = 1;
                } else if (global_ns() - t0 > s.timeout_ns || it > (1u << 26)) {
                    record_error(s, kStatusTimeout, who);
                    stop = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
    }
}

}  // namespace chm
