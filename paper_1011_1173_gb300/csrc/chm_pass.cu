// Host side of the pass path (chm_pass.cuh): the workspace of one pass, the
// launch sequence per block of update vectors, the choice between the pass
// path and the wave kernel, and the library-wide settings.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>

#include "chm.h"
#include "chm_internal.h"
#include "chm_pass.cuh"

namespace chm {

// ---------------------------------------------------------------- settings

namespace {
std::atomic<int> g_path{0};      // 0 automatic, 1 wave kernel, 2 pass kernels
std::atomic<int> g_pass_kb{0};   // vectors per pass (0: the largest, 16)
std::atomic<int> g_pass_d{0};    // lookahead of the substitution chain (0: per type)

int env_or(const char *name, int dflt)
{
    const char *e = getenv(name);
    return e ? atoi(e) : dflt;
}
}  // namespace

static int pass_kb_max()
{
    int v = g_pass_kb.load();
    if (v <= 0) v = env_or("CHM_PASS_KB", pass::kMaxKb);
    return std::max(1, std::min(pass::kMaxKb, v));
}

static int pass_d(int dtype)
{
    int v = g_pass_d.load();
    if (v <= 0) v = env_or("CHM_PASS_D", 0);
    if (v <= 0) v = dtype == CHM_F64 ? 4 : 10;
    // each instantiation clamps it further to what its shared memory holds
    return std::max(2, std::min(dtype == CHM_F64 ? 6 : 10, v));
}

int path_setting()
{
    int p = g_path.load();
    if (p == 0) p = env_or("CHM_PATH", 0);
    return p == 1 || p == 2 ? p : 0;
}

bool use_pass_path(long long n, long long k, int dtype, bool host_factor)
{
    const int p = path_setting();
    if (p == 1) return false;
    if (p == 2) return true;
    if (host_factor) return n >= 64;
    // automatic: the pass path once the factor is larger than about a
    // third of L2 (where the wave kernel's waves start to re-stream it); in
    // float64 only for few vectors, where the wave kernel's chain, not the
    // FP64 rate, bounds it
    const double bytes = (double)(dtype == CHM_F64 ? 8 : 4) * n * n / 2;
    if (dtype == CHM_F64) return bytes >= 256e6 && k <= 2;
    return bytes >= 32e6;
}

// ---------------------------------------------------------------- workspace

namespace {

struct PassLayout {
    size_t P, pflag, Ztag, Dinv, G, gram, H, coef, escale, dfac, ctl, bytes;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

PassLayout pass_layout(long long n, int elt)
{
    const size_t nb = (size_t)((n + pass::kB - 1) / pass::kB);
    const size_t rows = nb * pass::kB;
    const size_t KB = pass::kMaxKb;
    PassLayout l;
    size_t x = 0;
    // the tagged words and control words first: they are zeroed on
    // allocation (tag 0 matches no pass, whose epochs start at 1)
    const size_t words = elt / 4;
    l.pflag = x; x = al(x + nb * 4);
    l.Ztag = x; x = al(x + rows * KB * words * 8);
    l.ctl = x; x = al(x + pass::kCtlInts * 4);
    l.P = x; x = al(x + rows * KB * elt);
    l.Dinv = x; x = al(x + nb * 1024 * elt);
    l.G = x; x = al(x + (size_t)pass::kMaxCrit * nb * 1024 * elt);
    l.gram = x; x = al(x + nb * KB * KB * 8);
    l.H = x; x = al(x + nb * KB * KB * 8);
    l.coef = x; x = al(x + rows * 2 * KB * elt);
    l.escale = x; x = al(x + rows * elt);
    l.dfac = x; x = al(x + rows * 8);
    l.bytes = x;
    return l;
}

}  // namespace

size_t pass_workspace_bytes(long long n, int dtype)
{
    return pass_layout(n, dtype == CHM_F64 ? 8 : 4).bytes;
}

size_t pass_flag_bytes(long long n, int dtype)
{
    return pass_layout(n, dtype == CHM_F64 ? 8 : 4).P;  // the tagged and control words
}

// ---------------------------------------------------------------- launches

namespace {

int sm_of_current(int *nsm)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    *nsm = sm_count(dev);
    return *nsm > 0 ? CHM_OK : CHM_ERR_CUDA;
}

template <typename T, int KB>
size_t trsm_smem()
{
    const size_t chain = sizeof(pass::ChainSmem<T, KB>);
    using W = pass::WorkerCfg<T, KB>;
    const size_t workers = (size_t)W::warps * W::warp_bytes;
    return (std::max(chain, workers) + 127) & ~(size_t)127;
}

template <typename T, int KB>
size_t sweep_smem()
{
    return pass::SweepCfg<T, KB>::smem;
}

// One-time attributes and the sweep's resident blocks per SM, per device
// and instantiation (allocates nothing).
template <typename T, int KB>
int pass_setup(int dev, int *sweep_bps)
{
    static int bps[64] = {0};
    if (dev < 0 || dev >= 64) return CHM_ERR_ARG;
    if (!bps[dev]) {
        if (cudaFuncSetAttribute(pass::trsm_kernel<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)trsm_smem<T, KB>()) != cudaSuccess)
            return CHM_ERR_CUDA;
        if (cudaFuncSetAttribute(pass::sweep_kernel<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sweep_smem<T, KB>()) != cudaSuccess)
            return CHM_ERR_CUDA;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pass::sweep_kernel<T, KB>,
                                                          pass::SweepCfg<T, KB>::WARPS * 32, sweep_smem<T, KB>()) !=
                cudaSuccess ||
            b < 1)
            return CHM_ERR_CUDA;
        bps[dev] = b;
    }
    *sweep_bps = bps[dev];
    return CHM_OK;
}

template <typename T, int KB>
int launch_pass(pass::Args<T> A, cudaStream_t s)
{
    int dev = 0, nsm = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    int rc = sm_of_current(&nsm);
    if (rc != CHM_OK) return rc;
    if ((rc = pass_setup<T, KB>(dev, &bps)) != CHM_OK) return rc;
    const int nb = A.nb;
    A.d = std::min(A.d, pass::ChainCfg<T, KB>::DMAX);
    A.c = std::min(A.d, pass::ChainCfg<T, KB>::CMAX);
    if (cudaMemsetAsync(A.ctl, 0, pass::kCtlInts * sizeof(int), s) != cudaSuccess) return CHM_ERR_CUDA;
    pass::prep_kernel<T><<<std::min(nb, nsm * 16), 32, 0, s>>>(A);
    pass::trsm_kernel<T, KB><<<nsm, pass::kTrsmWarps * 32, trsm_smem<T, KB>(), s>>>(A);
    pass::gram_kernel<T, KB><<<std::min(nb, nsm * 16), 32, 0, s>>>(A);
    pass::scan_kernel<T, KB><<<(KB * KB + 31) / 32, 1024, 0, s>>>(A);
    pass::coef_kernel<T, KB><<<std::min(nb, nsm * 8), 32, pass::Packed<KB>::smem, s>>>(A);
    pass::sweep_kernel<T, KB><<<nsm * bps, pass::SweepCfg<T, KB>::WARPS * 32, sweep_smem<T, KB>(), s>>>(A);
    return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

template <typename T>
int launch_pass_kb(const pass::Args<T> &A, cudaStream_t s)
{
    const int kb = A.kb;
    if (kb <= 1) return launch_pass<T, 1>(A, s);
    if (kb <= 2) return launch_pass<T, 2>(A, s);
    if (kb <= 4) return launch_pass<T, 4>(A, s);
    if (kb <= 8) return launch_pass<T, 8>(A, s);
    return launch_pass<T, 16>(A, s);
}

template <typename T>
int enqueue_passes(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                   const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                   const Scratch &sc, PassSpace &ps)
{
    const PassLayout lay = pass_layout(n, sizeof(T));
    char *w = ps.buf;
    pass::Args<T> A;
    memset(&A, 0, sizeof(A));
    A.L = L;
    A.n = n;
    A.ld = ld;
    A.ldv = ldv;
    A.nb = (int)((n + pass::kB - 1) / pass::kB);
    A.d = pass_d(dtype);
    A.P = reinterpret_cast<T *>(w + lay.P);
    A.pflag = reinterpret_cast<int *>(w + lay.pflag);
    A.Ztag = reinterpret_cast<long long *>(w + lay.Ztag);
    A.Dinv = reinterpret_cast<T *>(w + lay.Dinv);
    A.G = reinterpret_cast<T *>(w + lay.G);
    A.gram = reinterpret_cast<double *>(w + lay.gram);
    A.H = reinterpret_cast<double *>(w + lay.H);
    A.coef = reinterpret_cast<T *>(w + lay.coef);
    A.escale = reinterpret_cast<T *>(w + lay.escale);
    A.dfac = reinterpret_cast<double *>(w + lay.dfac);
    A.ctl = reinterpret_cast<int *>(w + lay.ctl);
    A.status = sc.status;
    A.user_info = d_info;
    A.timeout_ns = timeout_ns();
    const int kbmax = pass_kb_max();
    for (long long q0 = 0; q0 < k; q0 += kbmax) {
        const int kb = (int)std::min<long long>(kbmax, k - q0);
        A.V = V + q0 * ldv;
        A.kb = kb;
        unsigned long long mask = 0;
        for (int q = 0; q < kb; ++q)
            if ((sigma ? sigma[q0 + q] : sign) < 0) mask |= 1ull << q;
        A.down_mask = mask;
        A.epoch = ++ps.epoch;
        A.trace = trace_buffer((size_t)A.nb * 16, stream);  // the last pass's, with CHM_TRACE=1
        const int rc = launch_pass_kb<T>(A, stream);
        if (rc != CHM_OK) return rc;
    }
    return CHM_OK;
}

}  // namespace

int pass_enqueue(void *L, long long n, long long ld, const void *V, long long ldv, long long k,
                 const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                 const Scratch &sc, PassSpace &ps)
{
    int rc = info_init(d_info, 1, stream);
    if (rc != CHM_OK) return rc;
    if (dtype == CHM_F64)
        return enqueue_passes<double>(static_cast<double *>(L), n, ld, static_cast<const double *>(V), ldv, k,
                                      sigma, sign, dtype, stream, d_info, sc, ps);
    return enqueue_passes<float>(static_cast<float *>(L), n, ld, static_cast<const float *>(V), ldv, k, sigma,
                                 sign, dtype, stream, d_info, sc, ps);
}

}  // namespace chm

extern "C" {

int chm_config_set(const char *key, int64_t value)
{
    if (!key) return CHM_ERR_ARG;
    if (!strcmp(key, "path")) {
        if (value < 0 || value > 2) return CHM_ERR_ARG;
        chm::g_path.store((int)value);
        return CHM_OK;
    }
    if (!strcmp(key, "pass_kb")) {
        if (value < 0 || value > chm::pass::kMaxKb) return CHM_ERR_ARG;
        chm::g_pass_kb.store((int)value);
        return CHM_OK;
    }
    if (!strcmp(key, "pass_d")) {
        if (value < 0 || value > 64) return CHM_ERR_ARG;
        chm::g_pass_d.store((int)value);
        return CHM_OK;
    }
    return CHM_ERR_ARG;
}

int chm_config_get(const char *key, int64_t *value)
{
    if (!key || !value) return CHM_ERR_ARG;
    if (!strcmp(key, "path")) *value = chm::g_path.load();
    else if (!strcmp(key, "pass_kb")) *value = chm::pass_kb_max();
    else if (!strcmp(key, "pass_d_f32")) *value = chm::pass_d(CHM_F32_MIXED);
    else if (!strcmp(key, "pass_d_f64")) *value = chm::pass_d(CHM_F64);
    else return CHM_ERR_ARG;
    return CHM_OK;
}

int chm_path_for(int64_t n, int64_t k, int dtype, int *path)
{
    if (!path || n < 0 || k < 0 || (dtype != CHM_F64 && dtype != CHM_F32_MIXED)) return CHM_ERR_ARG;
    *path = chm::use_pass_path(n, k, dtype, false) ? 2 : 1;
    return CHM_OK;
}

}  // extern "C"
