// C ABI of the rank-k Cholesky up/downdate (Walder 2010): argument checks,
// scratch carving, the launch of the wave kernel (chm_wave.cuh), the
// per-(device, stream) workspace of the plain entry points, the
// no-allocation variant and the device status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "chm.h"
#include "chm_internal.h"
#include "chm_wave.cuh"

namespace chm {

// ---------------------------------------------------------------- scratch carving

ScratchNeed scratch_need(const ProbShape *shapes, int count)
{
    ScratchNeed r;
    for (int i = 0; i < count; ++i) {
        const int nb = (int)((shapes[i].n + kW - 1) / kW);
        const int k = shapes[i].k;
        r.iflags += prob_iflags(nb, k);
        r.progress += prob_progress(nb, k);
        r.data += prob_data_bytes(nb, k);
        r.npairs += k + 1;  // its waves and the final pass
        r.nbmax = std::max(r.nbmax, nb);
    }
    return r;
}

std::vector<int> carve(const ProbShape *shapes, int count, const Scratch &sc, Prob *problems)
{
    std::vector<int> pair_prob;
    size_t fi = 0, fp = 0, fd = 0;
    int pair = 0;
    for (int i = 0; i < count; ++i) {
        const int nb = (int)((shapes[i].n + kW - 1) / kW);
        const int k = shapes[i].k;
        Prob &p = problems[i];
        p.nb = nb;
        p.k = k;
        p.pair0 = pair;
        p.iflags = sc.iflags + fi;
        p.progress = sc.progress + fp;
        p.data = sc.data + fd;
        fi += prob_iflags(nb, k);
        fp += prob_progress(nb, k);
        fd += prob_data_bytes(nb, k);
        pair_prob.insert(pair_prob.end(), (size_t)k + 1, i);
        pair += k + 1;
    }
    return pair_prob;
}

// ---------------------------------------------------------------- device facts

int sm_count(int dev)
{
    static int cache[64] = {0};
    if (dev < 0 || dev >= 64) return 1;
    if (!cache[dev]) cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev);
    return cache[dev];
}

long long timeout_ns()
{
    static long long v = [] {
        const char *e = getenv("CHM_TIMEOUT_NS");
        long long t = e ? atoll(e) : 0;
        return t > 0 ? t : 4000000000ll;
    }();
    return v;
}

static int env_int(const char *name)
{
    const char *e = getenv(name);
    return e ? atoi(e) : 0;
}

// One-time per-(device, type) set-up: the shared-memory attribute and the
// occupancy limit; allocates nothing.
template <typename T>
static int occupancy(int dev, int *bps_out)
{
    static int occ[2][64] = {{0}};
    if (dev < 0 || dev >= 64) return CHM_ERR_ARG;
    int &bps = occ[sizeof(T) == 8 ? 0 : 1][dev];
    if (!bps) {
        const size_t smem = kBlockSmemBytes;
        if (cudaFuncSetAttribute(wave_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return CHM_ERR_CUDA;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, wave_kernel<T>, 128, smem) != cudaSuccess ||
            b < 1)
            return CHM_ERR_CUDA;
        const int cap = env_int("CHM_MAX_CTAS_PER_SM");
        if (cap > 0 && cap < b) b = cap;
        bps = b;
    }
    *bps_out = bps;
    return CHM_OK;
}

int wave_occupancy(int dtype, int dev, int *ctas_per_sm)
{
    return dtype == CHM_F64 ? occupancy<double>(dev, ctas_per_sm) : occupancy<float>(dev, ctas_per_sm);
}

// Groups: one per concurrently running wave.  One problem: about seven sweep
// SMs per group (its waves share the sweep work of one factor), and up to
// nsm / 8 groups, so that a rank-16 modification runs all its waves and its
// final pass at once (measured at n = 5000, k = 16: 17 groups 1.88 ms, 16
// groups 1.99 ms, 12 groups 2.43 ms); many independent problems: two sweep
// SMs per group, since more chains in flight matter more than sweep
// capacity per chain (measured on the batched workload: 50 groups 31 ms,
// 16 groups 59 ms).
int default_groups(int npairs, int nsm, int nprobs)
{
    int g = env_int("CHM_GROUPS");
    if (g <= 0) g = std::max(1, nprobs > 1 ? nsm / 3 : nsm / 8);
    return std::max(1, std::min(std::min(g, npairs), std::min(kMaxGroups, nsm / 2)));
}

// ---------------------------------------------------------------- launch

template <typename T>
static int launch_t(const Prob *single, const Prob *d_probs, const int *d_pair_prob, int nprobs,
                    int npairs, int nbmax, const Scratch &sc, const LaunchCfg &cfg, long long *trace,
                    cudaStream_t stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    int bps = 0;
    int rc = occupancy<T>(dev, &bps);
    if (rc != CHM_OK) return rc;
    if (cfg.ctas_per_sm > 0) bps = std::min(bps, cfg.ctas_per_sm);
    const int nsm = sm_count(dev);
    if (nsm < 2 || nsm > kMaxSm || npairs < 1) return CHM_ERR_ARG;
    const int grid = cfg.grid > 0 ? std::max(2, std::min(cfg.grid, nsm * bps)) : nsm * bps;
    // SMs the launch can hold at the occupancy limit
    const int nsm_eff = std::max(2, std::min(nsm, grid / bps));
    int G = cfg.groups > 0 ? cfg.groups : default_groups(npairs, nsm_eff, nprobs);
    G = std::max(1, std::min(std::min(G, npairs), std::min(kMaxGroups, nsm_eff / 2)));
    Launch<T> P;
    memset(&P, 0, sizeof(P));
    P.probs = d_probs;
    if (single) P.prob0 = *single;
    P.pair_prob = d_pair_prob;
    P.nprobs = nprobs;
    P.npairs = npairs;
    P.ngroups = G;
    P.nbmax = nbmax;
    P.ctl = sc.ctl;
    P.status = sc.status;
    P.trace = trace;
    P.timeout_ns = timeout_ns();
    P.skip_publish = cfg.skip_publish;
    P.ws_data = sc.data;
    P.ws_data_bytes = sc.data_bytes;
    P.ws_iflags = sc.iflags;
    P.ws_iflags_n = sc.iflags_cap;
    P.ws_progress = sc.progress;
    P.ws_progress_n = sc.progress_cap;
    P.chk_cut = check_cut();
    wave_kernel<T><<<grid, 128, kBlockSmemBytes, stream>>>(P);
    return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

int launch_wave(int dtype, const Prob *single, const Prob *d_probs, const int *d_pair_prob, int nprobs,
                int npairs, int nbmax, const Scratch &sc, const LaunchCfg &cfg, long long *trace,
                cudaStream_t stream)
{
    if (dtype == CHM_F64)
        return launch_t<double>(single, d_probs, d_pair_prob, nprobs, npairs, nbmax, sc, cfg, trace, stream);
    return launch_t<float>(single, d_probs, d_pair_prob, nprobs, npairs, nbmax, sc, cfg, trace, stream);
}

__global__ void info_init_kernel(long long *info, int count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        info[2 * i] = 0;
        info[2 * i + 1] = -1;
    }
}

int info_init(long long *d_info, int count, cudaStream_t stream)
{
    if (!d_info || count <= 0) return CHM_OK;
    info_init_kernel<<<std::min(64, (count + 127) / 128), 128, 0, stream>>>(d_info, count);
    return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

static const long long kStatusInit[2] = {0, -1};

// Control words: zero, epoch 1 (flag regions are zero, so no flag matches
// until a launch of epoch >= 1 raises it).
static int ctl_init(int *ctl, long long *status)
{
    if (cudaMemset(ctl, 0, kCtlInts * sizeof(int)) != cudaSuccess) return CHM_ERR_CUDA;
    const int one = 1;
    if (cudaMemcpy(ctl + kCtlEpoch, &one, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
        return CHM_ERR_CUDA;
    if (cudaMemcpy(status, kStatusInit, sizeof(kStatusInit), cudaMemcpyHostToDevice) != cudaSuccess)
        return CHM_ERR_CUDA;
    return CHM_OK;
}

bool is_host_memory(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int check_reachable(const void *p)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    cudaPointerAttributes a{};
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? CHM_ERR_ARG : CHM_ERR_CUDA;
    }
    switch (a.type) {
    case cudaMemoryTypeDevice: return a.device == dev ? CHM_OK : CHM_ERR_ARG;
    case cudaMemoryTypeManaged: return CHM_OK;
    case cudaMemoryTypeHost: return a.devicePointer == p ? CHM_OK : CHM_ERR_ARG;
    default: return CHM_ERR_ARG;
    }
}

size_t single_workspace_bytes(long long n, long long k)
{
    if (n <= 0 || k <= 0) return 0;
    const ProbShape sh{n, (int)std::min<long long>(k, kMaxWaves)};
    const ScratchNeed need = scratch_need(&sh, 1);
    return kCtlInts * sizeof(int) + 2 * sizeof(long long) + std::max(need.iflags, (size_t)4096) * sizeof(int) +
           std::max(need.progress, (size_t)1024) * sizeof(long long) + need.data;
}

int scratch_alloc(Scratch *sc, size_t iflags, size_t progress, size_t data)
{
    if (!sc->ctl) {
        if (cudaMalloc(&sc->ctl, kCtlInts * sizeof(int)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&sc->status, 2 * sizeof(long long)) != cudaSuccess) return CHM_ERR_NOMEM;
        const int rc = ctl_init(sc->ctl, sc->status);
        if (rc != CHM_OK) return rc;
    }
    if (sc->iflags_cap < iflags) {
        cudaFree(sc->iflags);
        sc->iflags = nullptr;
        sc->iflags_cap = 0;
        const size_t cap = std::max(iflags, (size_t)4096);
        if (cudaMalloc(&sc->iflags, cap * sizeof(int)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(sc->iflags, 0, cap * sizeof(int)) != cudaSuccess) return CHM_ERR_CUDA;
        sc->iflags_cap = cap;
    }
    if (sc->progress_cap < progress) {
        cudaFree(sc->progress);
        sc->progress = nullptr;
        sc->progress_cap = 0;
        const size_t cap = std::max(progress, (size_t)1024);
        if (cudaMalloc(&sc->progress, cap * sizeof(long long)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(sc->progress, 0, cap * sizeof(long long)) != cudaSuccess) return CHM_ERR_CUDA;
        sc->progress_cap = cap;
    }
    if (sc->data_bytes < data) {
        cudaFree(sc->data);
        sc->data = nullptr;
        sc->data_bytes = 0;
        if (cudaMalloc(&sc->data, data) != cudaSuccess) return CHM_ERR_NOMEM;
        sc->data_bytes = data;
    }
    return CHM_OK;
}

void scratch_free(Scratch *sc)
{
    cudaFree(sc->ctl);
    cudaFree(sc->status);
    cudaFree(sc->iflags);
    cudaFree(sc->progress);
    cudaFree(sc->data);
    *sc = Scratch();
}

// ---------------------------------------------------------------- plain entry points

// Scratch of one (device, stream), grown on demand.
struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    Scratch sc;
    PassSpace ps;
};

static std::mutex g_mu;
static std::vector<Workspace *> g_ws;

// Diagnostics: with CHM_TRACE=1 in the environment every launch of the plain
// entry points records %globaltimer stamps per task; chm_trace_dump writes
// the last launch's.
static long long *g_trace = nullptr;
static size_t g_trace_words = 0, g_trace_cap = 0;
static bool trace_on()
{
    static int v = env_int("CHM_TRACE") > 0 ? 1 : 0;
    return v != 0;
}

long long *trace_buffer(size_t words, cudaStream_t stream)
{
    if (!trace_on() || words == 0) return nullptr;
    if (g_trace_cap < words) {
        cudaFree(g_trace);
        g_trace = nullptr;
        g_trace_cap = 0;
        if (cudaMalloc(&g_trace, words * sizeof(long long)) != cudaSuccess) return nullptr;
        g_trace_cap = words;
    }
    cudaMemsetAsync(g_trace, 0, words * sizeof(long long), stream);
    g_trace_words = words;
    return g_trace;
}

// Frees the workspace of (dev, s), if any (the caller has synchronised s).
void release_workspace(int dev, cudaStream_t s)
{
    std::lock_guard<std::mutex> lock(g_mu);
    for (size_t i = 0; i < g_ws.size(); ++i) {
        Workspace *w = g_ws[i];
        if (w->device == dev && w->stream == s) {
            scratch_free(&w->sc);
            cudaFree(w->ps.buf);
            delete w;
            g_ws.erase(g_ws.begin() + (long)i);
            return;
        }
    }
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

// Test hook for the bounded waits: CHM_TEST_SKIP_PUBLISH=b in the environment
// makes the next launch of the plain entry points leave block b's panel
// unreleased (once), so that the waits on it run out and the launch ends
// with CHM_ERR_TIMEOUT.  Nothing faults; the context stays usable.
static int take_test_skip()
{
    static int pending = [] {
        const char *e = getenv("CHM_TEST_SKIP_PUBLISH");
        return e ? atoi(e) : -1;
    }();
    const int v = pending;
    pending = -1;
    return v;
}

static unsigned long long down_mask(const int8_t *sigma, int sign, long long q0, int kw)
{
    unsigned long long mask = 0;
    for (int q = 0; q < kw; ++q) {
        const int sg = sigma ? sigma[q0 + q] : sign;
        if (sg < 0) mask |= 1ull << q;
    }
    return mask;
}

// Enqueue the launches of one modification, at most kw_max waves each, on
// scratch `sc` (already large enough for kw_max waves).
static int enqueue_single(void *L, long long n, long long ld, const void *V, long long ldv, long long k,
                          const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                          const Scratch &sc, int kw_max, bool allow_trace)
{
    const size_t elt = dtype == CHM_F64 ? 8 : 4;
    const int nb = (int)((n + kW - 1) / kW);
    int rc = info_init(d_info, 1, stream);
    if (rc != CHM_OK) return rc;
    for (long long q0 = 0; q0 < k; q0 += kw_max) {
        const int kw = (int)std::min<long long>(kw_max, k - q0);
        Prob pr;
        memset(&pr, 0, sizeof(pr));
        const ProbShape sh{n, kw};
        carve(&sh, 1, sc, &pr);
        pr.L = L;
        pr.V = static_cast<const char *>(V) + (size_t)q0 * ldv * elt;
        pr.n = n;
        pr.ld = ld;
        pr.ldv = ldv;
        pr.down_mask = down_mask(sigma, sign, q0, kw);
        pr.info = d_info;
        long long *trace = nullptr;
        if (allow_trace && trace_on()) {
            const size_t need = (size_t)2 * (kw + 1) * nb * kTracePoints;
            if (g_trace_cap < need) {
                cudaFree(g_trace);
                g_trace = nullptr;
                g_trace_cap = 0;
                if (cudaMalloc(&g_trace, need * sizeof(long long)) == cudaSuccess) g_trace_cap = need;
            }
            if (g_trace) {
                cudaMemsetAsync(g_trace, 0, need * sizeof(long long), stream);
                trace = g_trace;
                g_trace_words = need;
            }
        }
        LaunchCfg cfg;
        cfg.skip_publish = take_test_skip();
        rc = launch_wave(dtype, &pr, nullptr, nullptr, 1, kw + 1, nb, sc, cfg, trace, stream);
        if (rc != CHM_OK) return rc;
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
    if (n == 0 || k == 0) return info_init(d_info, 1, stream);
    if ((rc = check_reachable(L)) != CHM_OK || (rc = check_reachable(V)) != CHM_OK) return rc;
    const PassChoice ch = choose_path(n, k, dtype, is_host_memory(L));
    if (ch.path == 2) {
        return with_pass_workspace(stream, pass_workspace_bytes(n, dtype, ch.seg), n, dtype,
                                   [&](const Scratch &sc, PassSpace &ps) {
                                       return pass_enqueue(L, n, ld, V, ldv, k, sigma, sign, dtype, stream,
                                                           d_info, ch, sc, ps);
                                   });
    }
    const int kw_max = (int)std::min<long long>(k, kMaxWaves);
    const ProbShape sh{n, kw_max};
    const ScratchNeed need = scratch_need(&sh, 1);
    return with_stream_scratch(stream, need, [&](const Scratch &sc) {
        return enqueue_single(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info, sc, kw_max, true);
    });
}

// chm_modify_solve: the modification, then B <- (L~^T L~)^{-1} B.  On the
// pass kernels the forward half rides in the last pass (the substitution
// carries B's columns beside V's, and the recurrence task turns F^{-T} B
// into L~^{-T} B with the pass's rotations), so that it costs no crossing
// of the factor of its own; the back substitution follows.  On the wave
// kernel (factors that stay in L2) the modification and chm_solve follow
// each other on the stream.
static int modify_solve_dispatch(void *L, long long n, long long ld, const void *V, long long ldv, long long k,
                                 const int8_t *sigma, int sign, void *B, long long ldb, long long nrhs, int dtype,
                                 cudaStream_t stream, long long *d_info)
{
    int rc = check_args(L, n, ld, V, ldv, k, sigma, sign, dtype);
    if (rc != CHM_OK) return rc;
    const size_t elt = dtype == CHM_F64 ? 8 : 4;
    if (nrhs < 0 || ldb < std::max(1ll, n)) return CHM_ERR_ARG;
    if (n > 0 && nrhs > 0 && (!B || ((uintptr_t)B % elt))) return CHM_ERR_ARG;
    if (n == 0 || nrhs == 0) return modify_dispatch(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info);
    if (k == 0) {
        if ((rc = info_init(d_info, 1, stream)) != CHM_OK) return rc;
        return chm_solve(L, n, ld, B, ldb, nrhs, dtype, (chm_stream_t)stream);
    }
    if ((rc = check_reachable(L)) != CHM_OK || (rc = check_reachable(V)) != CHM_OK ||
        (rc = check_reachable(B)) != CHM_OK)
        return rc;
    const PassChoice ch = choose_path(n, k, dtype, is_host_memory(L));
    if (ch.path == 2) {
        // the solve's scratch first (the stream's workspace, grown under its
        // own hold of the lock), then the passes on the same workspace
        if ((rc = with_stream_scratch(stream, solve_need(n), [](const Scratch &) { return (int)CHM_OK; })) != CHM_OK)
            return rc;
        return with_pass_workspace(stream, pass_workspace_bytes(n, dtype, ch.seg), n, dtype,
                                   [&](const Scratch &sc, PassSpace &ps) {
                                       return pass_enqueue(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info,
                                                           ch, sc, ps, B, ldb, nrhs);
                                   });
    }
    if ((rc = modify_dispatch(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info)) != CHM_OK) return rc;
    return chm_solve(L, n, ld, B, ldb, nrhs, dtype, (chm_stream_t)stream);
}

int with_pass_workspace(cudaStream_t stream, size_t bytes, long long n, int dtype,
                        const std::function<int(const Scratch &, PassSpace &)> &fn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *w = find_workspace(dev, stream, true);
    if (!w->sc.ctl) {  // the control words and the stream's status word
        const int rc = scratch_alloc(&w->sc, 0, 0, 0);
        if (rc != CHM_OK) return rc;
    }
    if (w->ps.bytes < bytes) {
        // queued work on this stream may still use the old buffer
        if (cudaStreamSynchronize(stream) != cudaSuccess) return CHM_ERR_CUDA;
        cudaFree(w->ps.buf);
        w->ps.buf = nullptr;
        w->ps.bytes = 0;
        if (cudaMalloc(&w->ps.buf, bytes) != cudaSuccess) return CHM_ERR_NOMEM;
        // the flag and control words lead the buffer; zero flags match no epoch
        if (cudaMemset(w->ps.buf, 0, pass_flag_bytes(n, dtype)) != cudaSuccess) return CHM_ERR_CUDA;
        w->ps.bytes = bytes;
        w->ps.epoch = 0;
        w->ps.flag_n = n;
        w->ps.flag_dtype = dtype;
        w->ps.task_nb = -1;  // holds no sweep task table yet
    }
    // The flags' places move with the order and the element type: a call
    // whose layout differs from the last one's zeroes its flag region first
    // (in stream order), so that no word left there by another layout (a
    // data value, a control count) can pass for one of this pass's flags.
    // Within one layout the region only ever holds flags and tagged words of
    // earlier passes, whose epochs match no later pass.
    if (w->ps.flag_n != n || w->ps.flag_dtype != dtype) {
        if (cudaMemsetAsync(w->ps.buf, 0, pass_flag_bytes(n, dtype), stream) != cudaSuccess) return CHM_ERR_CUDA;
        w->ps.flag_n = n;
        w->ps.flag_dtype = dtype;
    }
    return fn(w->sc, w->ps);
}

int with_stream_scratch(cudaStream_t stream, const ScratchNeed &need, const std::function<int(const Scratch &)> &fn)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *w = find_workspace(dev, stream, true);
    if (w->sc.iflags_cap < need.iflags || w->sc.progress_cap < need.progress || w->sc.data_bytes < need.data ||
        !w->sc.ctl) {
        // queued work on this stream may still use the old regions
        if (cudaStreamSynchronize(stream) != cudaSuccess) return CHM_ERR_CUDA;
        const int rc = scratch_alloc(&w->sc, need.iflags, need.progress, need.data);
        if (rc != CHM_OK) return rc;
    }
    return fn(w->sc);
}

// ---------------------------------------------------------------- no-allocation variant

// chm_modify_noalloc serves callers that must not allocate device memory:
// its scratch is this array, one copy on every GPU that loads the library,
// held until the process exits.  Every call shares it.
constexpr size_t kNoAllocBytes = (size_t)16 << 20;
constexpr long long kNoAllocMaxN = 8192;
// control words, status word, int flags, progress words, data
constexpr size_t kNoAllocStatusOff = align256(kCtlInts * sizeof(int));
constexpr size_t kNoAllocIflagsOff = kNoAllocStatusOff + 256;
constexpr size_t kNoAllocIflags = 32768;  // ints
constexpr size_t kNoAllocProgressOff = kNoAllocIflagsOff + kNoAllocIflags * sizeof(int);
constexpr size_t kNoAllocProgress = 196608;  // tagged words (1.5 MiB)
constexpr size_t kNoAllocDataOff = kNoAllocProgressOff + kNoAllocProgress * sizeof(long long);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocState {
    bool ready = false;
    Scratch sc;
};
static NoAllocState g_noalloc[64];
static std::mutex g_noalloc_mu;

// First call on a device (with that device current): look up the array's
// device address, zero its control and flag words once and set the epoch.
static int noalloc_setup(int dev, NoAllocState **out)
{
    NoAllocState &st = g_noalloc[dev];
    if (!st.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CHM_ERR_CUDA;
        char *base = static_cast<char *>(p);
        if (cudaMemset(base, 0, kNoAllocDataOff) != cudaSuccess) return CHM_ERR_CUDA;
        Scratch sc;
        sc.ctl = reinterpret_cast<int *>(base);
        sc.status = reinterpret_cast<long long *>(base + kNoAllocStatusOff);
        sc.iflags = reinterpret_cast<int *>(base + kNoAllocIflagsOff);
        sc.iflags_cap = kNoAllocIflags;
        sc.progress = reinterpret_cast<long long *>(base + kNoAllocProgressOff);
        sc.progress_cap = kNoAllocProgress;
        sc.data = base + kNoAllocDataOff;
        sc.data_bytes = kNoAllocBytes - kNoAllocDataOff;
        const int rc = ctl_init(sc.ctl, sc.status);
        if (rc != CHM_OK) return rc;
        if (cudaDeviceSynchronize() != cudaSuccess) return CHM_ERR_CUDA;
        st.sc = sc;
        st.ready = true;
    }
    *out = &st;
    return CHM_OK;
}

// Waves per launch that fit the array for order n (0: none).
static int noalloc_waves(long long n)
{
    for (int kw = kMaxWaves; kw >= 1; --kw) {
        const ProbShape sh{n, kw};
        const ScratchNeed need = scratch_need(&sh, 1);
        if (need.iflags <= kNoAllocIflags && need.progress <= kNoAllocProgress &&
            need.data <= kNoAllocBytes - kNoAllocDataOff)
            return kw;
    }
    return 0;
}

static int modify_noalloc(void *L, long long n, long long ld, const void *V, long long ldv,
                          long long k, const int8_t *sigma, int sign, int dtype,
                          cudaStream_t stream, long long *d_info)
{
    int rc = check_args(L, n, ld, V, ldv, k, sigma, sign, dtype);
    if (rc != CHM_OK) return rc;
    // this variant's status word lives in the shared array, which
    // chm_status_sync does not read: without d_info an error would be lost
    if (n > 0 && k > 0 && !d_info) return CHM_ERR_ARG;
    if (n > kNoAllocMaxN) return CHM_ERR_BUDGET;
    if (n == 0 || k == 0) return info_init(d_info, 1, stream);
    if ((rc = check_reachable(L)) != CHM_OK || (rc = check_reachable(V)) != CHM_OK) return rc;
    const int kw_max = std::min<int>(noalloc_waves(n), (int)std::min<long long>(k, kMaxWaves));
    if (kw_max < 1) return CHM_ERR_BUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    if (dev < 0 || dev >= 64) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocState *st = nullptr;
    rc = noalloc_setup(dev, &st);
    if (rc != CHM_OK) return rc;
    return enqueue_single(L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info, st->sc, kw_max, false);
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

int chm_modify_solve(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k, const int8_t *sigma,
                     int sign, void *B, int64_t ldb, int64_t nrhs, int dtype, chm_stream_t stream, int64_t *d_info)
{
    return chm::modify_solve_dispatch(L, n, ld, V, ldv, k, sigma, sign, B, ldb, nrhs, dtype, (cudaStream_t)stream,
                                      reinterpret_cast<long long *>(d_info));
}

int chm_modify_noalloc(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k,
                       const int8_t *sigma, int sign, int dtype, chm_stream_t stream, int64_t *d_info)
{
    return chm::modify_noalloc(L, n, ld, V, ldv, k, sigma, sign, dtype, (cudaStream_t)stream,
                               reinterpret_cast<long long *>(d_info));
}

int chm_workspace_bytes(int64_t n, int64_t k, int dtype, size_t *bytes)
{
    if (!bytes || n < 0 || k < 0 || n > (1ll << 26)) return CHM_ERR_ARG;
    if (dtype != CHM_F64 && dtype != CHM_F32_MIXED) return CHM_ERR_ARG;
    const size_t wave = chm::single_workspace_bytes(n, k);
    const chm::PassChoice ch = chm::choose_path(n, k, dtype, false);
    const size_t pass = (n > 0 && k > 0) ? chm::kCtlInts * sizeof(int) + 2 * sizeof(long long) +
                                               chm::pass_workspace_bytes(n, dtype, ch.seg)
                                         : 0;
    // a forced path holds its own workspace; the automatic rule may take
    // either (a factor in host memory takes the pass kernels), so the larger
    const int path = chm::path_setting();
    *bytes = path == 1 ? wave : path == 2 ? pass : std::max(wave, pass);
    return CHM_OK;
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
        if (w && w->sc.status) {
            if (cudaMemcpy(h, w->sc.status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
                return CHM_ERR_CUDA;
            if (cudaMemcpy(w->sc.status, chm::kStatusInit, sizeof(chm::kStatusInit),
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
    case CHM_ERR_BOUNDS: return "CHM_ERR_BOUNDS: a kernel index outside its array (bounds-checked build)";
    default: return "unknown status";
    }
}

int chm_version(void) { return 200; }

int chm_trace_dump(const char *path)
{
    if (!path) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(chm::g_mu);
    if (!chm::g_trace || !chm::g_trace_words) return CHM_ERR_STATE;
    if (cudaDeviceSynchronize() != cudaSuccess) return CHM_ERR_CUDA;
    std::vector<long long> h(chm::g_trace_words);
    if (cudaMemcpy(h.data(), chm::g_trace, h.size() * sizeof(long long), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return CHM_ERR_CUDA;
    FILE *f = fopen(path, "wb");
    if (!f) return CHM_ERR_ARG;
    const size_t wrote = fwrite(h.data(), sizeof(long long), h.size(), f);
    fclose(f);
    return wrote == h.size() ? CHM_OK : CHM_ERR_ARG;
}

}  // extern "C"
