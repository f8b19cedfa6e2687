// C ABI of the rank-k Cholesky up/downdate (Walder 2010): argument checks,
// the per-(device, stream) workspace, launches of the wave kernel
// (chm_wave.cuh) and the device status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "chm.h"
#include "chm_wave.cuh"

namespace chm {

// ---------------------------------------------------------------- host side

// Device buffers of one (device, stream), grown on demand.
struct Workspace {
    int device = -1;
    cudaStream_t stream = nullptr;
    void *buf = nullptr;    // all per-launch arrays, carved by layout()
    size_t bytes = 0;
    int nb_cap = 0;         // blocks the flag arrays are laid out for
    int *misc = nullptr;    // ticket, abort, ndiag, smslot[kMaxSm], smrole[kMaxSm]
    long long *status = nullptr;
    int epoch = 0;
};

// Byte offsets of the per-launch arrays.  The flag and counter arrays come
// first, laid out for kMaxWaves waves and nb_cap blocks with fixed strides,
// so a flag word keeps one meaning for the life of the allocation and stale
// words from earlier launches (smaller epochs) never match; they are zeroed
// once when allocated.  The data arrays after them are written before they
// are read in every launch.
struct Layout {
    int nb_cap;
    size_t pflag, progress, zflag, cflag, dflag, rflag0, flags_end;
    size_t coef, chain, chain0, tend, zbuf, carry, rdiag, rtile, total;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t align_up_const(size_t x, size_t a) { return (x + a - 1) / a * a; }

static Layout layout(int nb_cap, int nw, int nb)
{
    Layout L;
    L.nb_cap = nb_cap;
    size_t o = 0;
    const size_t nflag = (size_t)kMaxWaves * nb_cap;
    const size_t rows = (size_t)nw * nb * kW;
    L.pflag = o;    o = align256(o + sizeof(int) * nflag);
    L.progress = o; o = align256(o + sizeof(long long) * nflag);
    L.zflag = o;    o = align256(o + sizeof(int) * nflag);
    L.cflag = o;    o = align256(o + sizeof(int) * nflag);
    L.dflag = o;    o = align256(o + sizeof(int) * nflag);
    L.rflag0 = o;   o = align256(o + sizeof(int) * (size_t)nb_cap);
    L.flags_end = o;
    L.coef = o;     o = align256(o + sizeof(CoefRow<double>) * rows);
    L.chain = o;    o = align256(o + sizeof(ChainRow) * rows);
    L.chain0 = o;   o = align256(o + sizeof(ChainRow) * (size_t)nb * kW);
    L.tend = o;     o = align256(o + sizeof(double) * (size_t)nw * nb);
    L.zbuf = o;     o = align256(o + sizeof(double) * rows);
    L.carry = o;    o = align256(o + sizeof(double) * rows);
    L.rdiag = o;    o = align256(o + sizeof(double) * rows * kW);
    L.rtile = o;    o = align256(o + sizeof(double) * rows * kW);
    L.total = o;
    return L;
}

static std::mutex g_mu;
static std::vector<Workspace *> g_ws;

// Diagnostics: with CHM_TRACE=1 in the environment every launch records
// per-task %globaltimer stamps; chm_trace_dump writes the last launch's.
static long long *g_trace = nullptr;
static size_t g_trace_tasks = 0, g_trace_cap = 0;
static bool trace_on()
{
    static int v = [] {
        const char *e = getenv("CHM_TRACE");
        return e && atoi(e) > 0 ? 1 : 0;
    }();
    return v != 0;
}

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
// Waves per launch: each takes one SM for its diagonal work.
constexpr int kWavesPerLaunch = 16;
// misc ints: [0] ticket, [32] abort, [64] ndiag, [128..] smslot, [128+kMaxSm..] smrole
constexpr int kMiscInts = 128 + 2 * kMaxSm;

static int alloc_workspace(Workspace *w, int nw, int nb, Layout *out)
{
    if (w->buf && w->nb_cap >= nb) {
        const Layout lay = layout(w->nb_cap, nw, nb);
        if (lay.total <= w->bytes && w->misc) {
            *out = lay;
            return CHM_OK;
        }
    }
    // Queued work on this stream may still use the old buffers.
    if (cudaStreamSynchronize(w->stream) != cudaSuccess) return CHM_ERR_CUDA;
    const int nb_cap = std::max(nb, w->nb_cap);
    const Layout lay = layout(nb_cap, std::max(nw, (int)std::min<long long>(kMaxWaves, 16)), nb_cap);
    cudaFree(w->buf);
    w->buf = nullptr;
    w->bytes = 0;
    w->nb_cap = 0;
    if (cudaMalloc(&w->buf, lay.total) != cudaSuccess) return CHM_ERR_NOMEM;
    if (cudaMemset(w->buf, 0, lay.flags_end) != cudaSuccess) return CHM_ERR_CUDA;
    w->bytes = lay.total;
    w->nb_cap = nb_cap;
    w->epoch = 0;
    if (!w->misc) {
        if (cudaMalloc(&w->misc, kMiscInts * sizeof(int)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&w->status, 2 * sizeof(long long)) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMemset(w->misc, 0, kMiscInts * sizeof(int)) != cudaSuccess) return CHM_ERR_CUDA;
        if (cudaMemcpy(w->status, kStatusInit, sizeof(kStatusInit), cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return CHM_ERR_CUDA;
    }
    *out = layout(nb_cap, nw, nb);
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

// Scratch memory of one launch sequence: the arrays of layout(), the misc
// words and the status word, and the epoch counter of that scratch.
struct Scratch {
    char *base;
    int nb_cap;
    int *misc;
    long long *status;
    int *epoch;
};

// One-time per-(device, type) kernel set-up; allocates nothing.
template <typename T>
static int kernel_setup(int dev, int *bps_out)
{
    static int occ[2][64] = {{0}};
    int &bps = occ[sizeof(T) == 8 ? 0 : 1][dev & 63];
    if (!bps) {
        const size_t smem = kBlockSmemBytes;
        if (cudaFuncSetAttribute(wave_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return CHM_ERR_CUDA;
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, wave_kernel<T>, 128, smem) != cudaSuccess ||
            b < 1)
            return CHM_ERR_CUDA;
        const char *cap = getenv("CHM_MAX_CTAS_PER_SM");
        if (cap && atoi(cap) > 0 && atoi(cap) < b) b = atoi(cap);
        bps = b;
    }
    *bps_out = bps;
    return CHM_OK;
}

// Enqueue the launches of one modification (up to nw_max waves each) on
// `stream` using scratch `sc`.  Tracing (which allocates) only if allowed.
template <typename T>
static int launch_waves(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                        const int8_t *sigma, int sign, cudaStream_t stream, long long *d_info,
                        const Scratch &sc, int nw_max, bool allow_trace)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    int bps = 0;
    int rc = kernel_setup<T>(dev, &bps);
    if (rc != CHM_OK) return rc;
    const int nb = (int)((n + kW - 1) / kW);
    const int nsm = sm_count(dev);
    if (d_info) {
        info_init_kernel<<<1, 1, 0, stream>>>(d_info);
        if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
    }
    const size_t smem = kBlockSmemBytes;
    // one SM per wave: keep most SMs for the sweep
    nw_max = std::max(1, std::min(nw_max, std::min(kWavesPerLaunch, nsm / 8)));
    for (long long q0 = 0; q0 < k; q0 += nw_max) {
        const int nw = (int)std::min<long long>(nw_max, k - q0);
        if (nw + 1 > nsm) return CHM_ERR_ARG;
        unsigned long long mask = 0;
        for (int q = 0; q < nw; ++q) {
            const int sg = sigma ? sigma[q0 + q] : sign;
            if (sg < 0) mask |= 1ull << q;
        }
        // ticket, abort flag and the start-up role registry are zero for every launch
        if (cudaMemsetAsync(sc.misc, 0, kMiscInts * sizeof(int), stream) != cudaSuccess)
            return CHM_ERR_CUDA;
        const Layout ly = layout(sc.nb_cap, nw, nb);
        char *base = sc.base;
        WaveParams<T> prm;
        prm.L = L;
        prm.n = n;
        prm.ld = ld;
        prm.V = V + q0 * ldv;
        prm.ldv = ldv;
        prm.nwaves = nw;
        prm.nblocks = nb;
        prm.fstride = sc.nb_cap;
        prm.down_mask = mask;
        prm.coef = reinterpret_cast<CoefRow<T> *>(base + ly.coef);
        prm.chain = reinterpret_cast<ChainRow *>(base + ly.chain);
        prm.chain0 = reinterpret_cast<ChainRow *>(base + ly.chain0);
        prm.tend = reinterpret_cast<double *>(base + ly.tend);
        prm.pflag = reinterpret_cast<int *>(base + ly.pflag);
        prm.progress = reinterpret_cast<long long *>(base + ly.progress);
        prm.zbuf = reinterpret_cast<double *>(base + ly.zbuf);
        prm.zflag = reinterpret_cast<int *>(base + ly.zflag);
        prm.cflag = reinterpret_cast<int *>(base + ly.cflag);
        prm.dflag = reinterpret_cast<int *>(base + ly.dflag);
        prm.carry = reinterpret_cast<double *>(base + ly.carry);
        prm.rdiag = reinterpret_cast<double *>(base + ly.rdiag);
        prm.rtile = reinterpret_cast<double *>(base + ly.rtile);
        prm.rflag0 = reinterpret_cast<int *>(base + ly.rflag0);
        prm.smslot = sc.misc + 128;
        prm.smrole = sc.misc + 128 + kMaxSm;
        prm.ndiag = sc.misc + 64;
        prm.trace = nullptr;
        if (allow_trace && trace_on()) {
            const size_t need = (size_t)2 * nw * nb * kTracePoints;
            if (g_trace_cap < need) {
                cudaFree(g_trace);
                g_trace = nullptr;
                g_trace_cap = 0;
                if (cudaMalloc(&g_trace, need * sizeof(long long)) == cudaSuccess) g_trace_cap = need;
            }
            if (g_trace) {
                cudaMemsetAsync(g_trace, 0, need * sizeof(long long), stream);
                prm.trace = g_trace;
                g_trace_tasks = (size_t)2 * nw * nb;
            }
        }
        prm.sync.ticket = sc.misc;
        prm.sync.abort_flag = sc.misc + 32;
        prm.sync.status = sc.status;
        prm.sync.user_info = d_info;
        prm.sync.epoch = ++*sc.epoch;
        prm.sync.timeout_ns = timeout_ns();
        wave_kernel<T><<<nsm * bps, 128, smem, stream>>>(prm);
        if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
    }
    return CHM_OK;
}

template <typename T>
static int launch_modify(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                         const int8_t *sigma, int sign, cudaStream_t stream, long long *d_info)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    const int nb = (int)((n + kW - 1) / kW);
    const int wmax = (int)std::min<long long>(k, kMaxWaves);
    std::lock_guard<std::mutex> lock(g_mu);
    Workspace *w = find_workspace(dev, stream, true);
    Layout lay0;
    int rc = alloc_workspace(w, wmax, nb, &lay0);
    if (rc != CHM_OK) return rc;
    const Scratch sc{static_cast<char *>(w->buf), w->nb_cap, w->misc, w->status, &w->epoch};
    return launch_waves<T>(L, n, ld, V, ldv, k, sigma, sign, stream, d_info, sc, kMaxWaves, true);
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

// ---------------------------------------------------------------- no-allocation variant

// chm_modify_noalloc serves callers that must not allocate device memory:
// its scratch is this array, one copy on every GPU that loads the library,
// held until the process exits.  Every call shares it.
constexpr size_t kNoAllocBytes = (size_t)16 << 20;
constexpr long long kNoAllocMaxN = 8192;
constexpr int kNoAllocNbCap = (int)((kNoAllocMaxN + kW - 1) / kW);
// misc words, then the status word, then the arrays of layout()
constexpr size_t kNoAllocStatusOff = align_up_const(kMiscInts * sizeof(int), 256);
constexpr size_t kNoAllocHeader = kNoAllocStatusOff + 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocState {
    bool ready = false;
    char *base = nullptr;  // device address of g_noalloc_scratch on this device
    int epoch = 0;
};
static NoAllocState g_noalloc[64];
static std::mutex g_noalloc_mu;

// First call on a device (with that device current): look up the array's
// device address and zero its flag words once; later launches only ever
// compare flags against larger epochs.
static int noalloc_setup(int dev, NoAllocState **out)
{
    NoAllocState &st = g_noalloc[dev];
    if (!st.ready) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CHM_ERR_CUDA;
        char *base = static_cast<char *>(p);
        const Layout lay = layout(kNoAllocNbCap, 1, 1);
        if (cudaMemset(base, 0, kNoAllocHeader + lay.flags_end) != cudaSuccess) return CHM_ERR_CUDA;
        if (cudaMemcpy(base + kNoAllocStatusOff, kStatusInit, sizeof(kStatusInit),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            return CHM_ERR_CUDA;
        if (cudaDeviceSynchronize() != cudaSuccess) return CHM_ERR_CUDA;
        st.base = base;
        st.ready = true;
    }
    *out = &st;
    return CHM_OK;
}

// Waves per launch that fit the array for nb column blocks (0: none).
static int noalloc_waves(int nb)
{
    for (int nw = kMaxWaves; nw >= 1; --nw)
        if (kNoAllocHeader + layout(kNoAllocNbCap, nw, nb).total <= kNoAllocBytes) return nw;
    return 0;
}

static int modify_noalloc(void *L, long long n, long long ld, const void *V, long long ldv,
                          long long k, const int8_t *sigma, int sign, int dtype,
                          cudaStream_t stream, long long *d_info)
{
    int rc = check_args(L, n, ld, V, ldv, k, sigma, sign, dtype);
    if (rc != CHM_OK) return rc;
    if (n > kNoAllocMaxN) return CHM_ERR_BUDGET;
    if (n == 0 || k == 0) {
        if (d_info) {
            info_init_kernel<<<1, 1, 0, stream>>>(d_info);
            if (cudaGetLastError() != cudaSuccess) return CHM_ERR_CUDA;
        }
        return CHM_OK;
    }
    const int nb = (int)((n + kW - 1) / kW);
    const int nw_max = noalloc_waves(nb);
    if (nw_max < 1) return CHM_ERR_BUDGET;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    if (dev < 0 || dev >= 64) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocState *st = nullptr;
    rc = noalloc_setup(dev, &st);
    if (rc != CHM_OK) return rc;
    const Scratch sc{st->base + kNoAllocHeader, kNoAllocNbCap, reinterpret_cast<int *>(st->base),
                     reinterpret_cast<long long *>(st->base + kNoAllocStatusOff), &st->epoch};
    if (dtype == CHM_F64)
        return launch_waves<double>(static_cast<double *>(L), n, ld, static_cast<const double *>(V), ldv,
                                    k, sigma, sign, stream, d_info, sc, nw_max, false);
    return launch_waves<float>(static_cast<float *>(L), n, ld, static_cast<const float *>(V), ldv, k,
                               sigma, sign, stream, d_info, sc, nw_max, false);
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

int chm_modify_noalloc(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k,
                       const int8_t *sigma, int sign, int dtype, chm_stream_t stream, int64_t *d_info)
{
    return chm::modify_noalloc(L, n, ld, V, ldv, k, sigma, sign, dtype, (cudaStream_t)stream,
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

int chm_trace_dump(const char *path)
{
    if (!path) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(chm::g_mu);
    if (!chm::g_trace || !chm::g_trace_tasks) return CHM_ERR_STATE;
    if (cudaDeviceSynchronize() != cudaSuccess) return CHM_ERR_CUDA;
    std::vector<long long> h(chm::g_trace_tasks * chm::kTracePoints);
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
