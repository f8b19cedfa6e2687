// Host side of the pass path (chm_pass.cuh): the workspace of one pass, the
// launch sequence per block of update vectors, the choice between the pass
// path and the wave kernel, and the library-wide settings.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <vector>
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
std::atomic<int> g_pass_seg{0};  // row blocks per sweep segment (0: by the order)
std::atomic<int> g_pass_fused{-1};  // 1 fused passes (up to 8 vectors), 0 the six-kernel pass (-1: default, 1)
std::atomic<long long> g_check_cut{0};  // bounds-checked build: columns taken off a factor's extent

int env_or(const char *name, int dflt)
{
    const char *e = getenv(name);
    return e ? atoi(e) : dflt;
}
}  // namespace

long long check_cut() { return g_check_cut.load(); }

// The explicit settings (library setting, else environment; 0: not set).
static int kb_setting()
{
    const int v = g_pass_kb.load();
    return v > 0 ? v : std::max(0, env_or("CHM_PASS_KB", 0));
}
static int d_setting()
{
    const int v = g_pass_d.load();
    return v > 0 ? v : std::max(0, env_or("CHM_PASS_D", 0));
}
static int seg_setting()
{
    const int v = g_pass_seg.load();
    return v > 0 ? v : std::max(0, env_or("CHM_PASS_SEG", 0));
}

static int fused_setting()
{
    const int v = g_pass_fused.load();
    if (v >= 0) return v;
    const char *e = getenv("CHM_PASS_FUSED");
    return e ? (atoi(e) != 0) : 1;
}

static int clamp_kb(int v) { return std::max(1, std::min(pass::kMaxKb, v)); }
// each instantiation clamps the lookahead further to what its shared memory holds
static int clamp_d(int v, int dtype) { return std::max(2, std::min(dtype == CHM_F64 ? 6 : 10, v)); }

// Vectors per pass by default: the largest block a fused pass takes in
// float (8); in double 4, where the chain block's FP64 issue rate, which
// grows with the vectors, sets a step's time (measured at n = 32768: a
// rank-16 modification takes 7.1 ms in float with 8 vectors per pass
// against 7.8 with 16 and 8.3 with 4; in double 50.1 ms with 4 or 8
// against 77 with 16).
static int default_kb(int dtype) { return dtype == CHM_F64 ? 4 : 8; }

static int pass_kb_of(int dtype) { return clamp_kb(kb_setting() > 0 ? kb_setting() : default_kb(dtype)); }

// Lookahead by default, by type and vectors per pass (measured at
// n = 32768, one modification: float with 1 vector 1.48 ms at d = 2..5
// against 1.64 at 10, the near warps' running sums then lagging the chain;
// 4 vectors 1.94 ms at d = 6; 8 vectors flat from d = 5 to 10; double
// 4.43 ms at d = 2..3 against 4.64 at 6).
static int default_d(int dtype, int kb)
{
    if (dtype == CHM_F64) return 3;
    return kb <= 2 ? 4 : kb <= 4 ? 6 : 10;
}

static int pass_d(int dtype) { return clamp_d(d_setting() > 0 ? d_setting() : default_d(dtype, default_kb(dtype)), dtype); }

// Row blocks per segment of the sweep's column tasks: a column block's
// tiles are split at multiples of this, each segment starting from the
// carry rebuilt from the substitution's partial residual, so that no task
// is longer than about this many tiles.  By default at most 16 boundaries,
// so that the residual snapshots stay O(n k).
static int pass_seg(int nb, int seg)
{
    return std::max(1, seg > 0 ? seg : std::max(64, (nb + 15) / 16));
}

int path_setting()
{
    int p = g_path.load();
    if (p == 0) p = env_or("CHM_PATH", 0);
    return p == 1 || p == 2 ? p : 0;
}

// The built-in rule: the pass path once the factor is larger than about a
// third of L2 (where the wave kernel's waves start to re-stream it); in
// float64 only up to 8 vectors: beyond that both paths run at the FP64 rate
// (n = 32768: 25.0 against 25.9 ms at k = 8, 50.1 against 50.1 at k = 16,
// the wave kernel ahead at k = 64); and for a factor in page-locked host
// memory with two or more vectors (the pass crosses the CPU-GPU link three
// times per block of vectors, the wave kernel twice per vector).
static bool rule_pass(long long n, long long k, int dtype, bool host_factor)
{
    if (host_factor) return n >= 64 && k >= 2;
    const double bytes = (double)(dtype == CHM_F64 ? 8 : 4) * n * n / 2;
    if (dtype == CHM_F64) return bytes >= 256e6 && k <= 8;
    return bytes >= 32e6;
}

PassChoice builtin_choice(long long n, long long k, int dtype, bool host_factor)
{
    // a factor in host memory: as many vectors per pass as the kernels take,
    // since every pass moves the factor across the CPU-GPU link three times
    // (n = 32768, rank 16: float64 291 ms with 4 vectors per pass)
    const int kb = host_factor ? pass::kMaxKb : default_kb(dtype);
    return PassChoice{rule_pass(n, k, dtype, host_factor) ? 2 : 1, kb,
                      default_d(dtype, (int)std::min<long long>(std::max(1ll, k), kb)), 0, 1};
}

PassChoice choose_path(long long n, long long k, int dtype, bool host_factor)
{
    // precedence: explicit settings, then the tuner's candidate while it
    // times one, then the tuning cache (device factors), then the defaults
    PassChoice base = builtin_choice(n, k, dtype, host_factor);
    PassChoice tuned;
    bool d_given = d_setting() > 0;
    if (const PassChoice *o = tune_override()) base = *o, d_given = true;
    else if (!host_factor && tune_lookup(dtype, n, k, &tuned)) base = tuned, d_given = true;
    PassChoice c = base;
    const int p = path_setting();
    if (p != 0) c.path = p;
    if (kb_setting() > 0) c.kb = kb_setting();
    // the default lookahead follows the vectors of the pass actually run
    if (!d_given) c.d = default_d(dtype, (int)std::min<long long>(std::max(1ll, k), clamp_kb(c.kb)));
    if (d_setting() > 0) c.d = d_setting();
    if (seg_setting() > 0) c.seg = seg_setting();
    c.kb = clamp_kb(c.kb);
    c.d = clamp_d(c.d, dtype);
    c.seg = std::max(0, c.seg);
    c.fused = fused_setting();
    return c;
}

bool use_pass_path(long long n, long long k, int dtype, bool host_factor)
{
    return choose_path(n, k, dtype, host_factor).path == 2;
}

// ---------------------------------------------------------------- workspace

namespace {

struct PassLayout {
    size_t P, Ptag, Htag, cflag, wprog, Ztag, Dinv, G, gram, H, coef, escale, dfac, snap, rst, tasks, post, ctl, bytes;
    int seg, nbound;  // row blocks per sweep segment; segment boundaries (the snapshots' count)
    size_t ntask_max;
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

PassLayout pass_layout(long long n, int elt, int seg)
{
    const size_t nb = (size_t)((n + pass::kB - 1) / pass::kB);
    const size_t rows = nb * pass::kB;
    const size_t KB = pass::kMaxKb;
    PassLayout l;
    size_t x = 0;
    // the tagged words and control words first: they are zeroed on
    // allocation (tag 0 matches no pass, whose epochs start at 1)
    const size_t words = elt / 4;
    l.Ptag = x; x = al(x + rows * KB * 2 * 8);
    l.Htag = x; x = al(x + nb * KB * KB * 2 * 8);
    l.cflag = x; x = al(x + nb * 4);
    l.wprog = x; x = al(x + nb * 8);
    l.Ztag = x; x = al(x + rows * KB * words * 8);
    l.ctl = x; x = al(x + pass::kCtlInts * 4);
    l.P = x; x = al(x + rows * KB * elt);
    l.Dinv = x; x = al(x + nb * 1024 * elt);
    // G^(j) for every lookahead offset: at most 10 in float, 6 in double (clamp_d)
    const size_t ng = elt == 8 ? 6 : pass::kMaxG;
    l.G = x; x = al(x + ng * nb * 1024 * elt);
    l.gram = x; x = al(x + nb * KB * KB * 8);
    l.H = x; x = al(x + nb * KB * KB * 8);
    l.coef = x; x = al(x + rows * 2 * KB * elt);
    l.escale = x; x = al(x + rows * elt);
    l.dfac = x; x = al(x + rows * 8);
    // sweep segments: boundaries at row blocks seg, 2 seg, ... below the last block
    l.seg = pass_seg((int)nb, seg);
    l.nbound = nb > 1 ? (int)((nb - 1) / (size_t)l.seg) : 0;
    l.snap = x; x = al(x + (size_t)l.nbound * rows * KB * elt);
    l.rst = x; x = al(x + (size_t)l.nbound * KB * (KB + 1) / 2 * 8);
    l.ntask_max = nb * (size_t)(1 + l.nbound);
    l.tasks = x; x = al(x + l.ntask_max * 8);
    l.post = x; x = al(x + (nb + l.ntask_max) * 8);
    l.bytes = x;
    return l;
}

}  // namespace

size_t pass_workspace_bytes(long long n, int dtype, int seg)
{
    return pass_layout(n, dtype == CHM_F64 ? 8 : 4, seg).bytes;
}

size_t pass_flag_bytes(long long n, int dtype)
{
    return pass_layout(n, dtype == CHM_F64 ? 8 : 4, 0).P;  // the tagged and control words (lead the buffer)
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

// The sweep's tasks, (column block, segment), longest first, in the
// workspace.  Column block b has 1 + floor((b - d - 1) / seg) segments (a
// boundary needs the residual snapshot the substitution's workers take,
// which covers row blocks below b - d); the last one ends at the diagonal
// tile.  The table is written when its place in the buffer (which moves
// with the element type and the order) or (nb, d, seg) differs from the one
// the workspace holds: the copy is ordered before this pass's kernels on
// the stream, and every earlier pass has read its table by then.
int sweep_tasks(PassSpace &ps, int nb, int d, int seg, int2 *dst, int2 *post, int *ntasks, int *npost,
                cudaStream_t s)
{
    if (!(ps.task_at == dst && ps.task_nb == nb && ps.task_d == d && ps.task_seg == seg)) {
        struct Item {
            int len, b, s, last;  // tiles, column block, segment, its last row block
        };
        std::vector<Item> items;
        for (int b = 0; b < nb; ++b) {
            const int ns = 1 + std::max(0, (b - d - 1) / seg);
            for (int q = 0; q < ns; ++q) {
                const int last_rb = q == ns - 1 ? b : (q + 1) * seg - 1;
                items.push_back(Item{last_rb - q * seg + 1, b, q, last_rb});
            }
        }
        std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) {
            return x.len != y.len ? x.len > y.len : x.b > y.b;
        });
        // the sweep kernel's table: longest first
        std::vector<int2> tab(items.size());
        for (size_t i = 0; i < items.size(); ++i) tab[i] = make_int2(items[i].b, items[i].s);
        // a fused pass's table: row block r's coefficients, then the segments
        // that end at r (longest first), for r = 0 .. nb - 1; each task's
        // inputs come from the chain, the far-sum workers or earlier tasks
        std::vector<std::vector<int2>> at(nb);
        for (const Item &it : items) at[it.last].push_back(make_int2(it.b, it.s));
        std::vector<int2> pt;
        pt.reserve(items.size() + nb);
        for (int r = 0; r < nb; ++r) {
            pt.push_back(make_int2(-1, r));
            pt.insert(pt.end(), at[r].begin(), at[r].end());
        }
        // pageable sources: each call returns once the data is staged, so the
        // vectors may go out of scope afterwards
        ps.task_nb = -1;
        if (cudaMemcpyAsync(dst, tab.data(), tab.size() * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(post, pt.data(), pt.size() * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return CHM_ERR_CUDA;
        ps.task_at = dst;
        ps.task_nb = nb;
        ps.task_d = d;
        ps.task_seg = seg;
        ps.task_count = (int)tab.size();
        ps.post_count = (int)pt.size();
    }
    *ntasks = ps.task_count;
    *npost = ps.post_count;
    return CHM_OK;
}

template <typename T, int KB>
int launch_pass(pass::Args<T> A, PassSpace &ps, cudaStream_t s)
{
    int dev = 0, nsm = 0, bps = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    int rc = sm_of_current(&nsm);
    if (rc != CHM_OK) return rc;
    if ((rc = pass_setup<T, KB>(dev, &bps)) != CHM_OK) return rc;
    const int nb = A.nb;
    A.d = std::min(A.d, pass::ChainCfg<T, KB>::DMAX);
    A.c = std::min(A.d, pass::ChainCfg<T, KB>::CMAX);
    // a fused pass (up to 8 vectors per pass); a pass that rotates nothing
    // (right-hand sides only) is the substitution alone
    A.fused = A.fused && pass::FusedCfg<T, KB>::ok && A.kr > 0;
    if ((rc = sweep_tasks(ps, A.nb, A.d, A.seg, const_cast<int2 *>(A.tasks), const_cast<int2 *>(A.post), &A.ntasks,
                          &A.npost, s)) != CHM_OK)
        return rc;
    if (cudaMemsetAsync(A.ctl, 0, pass::kCtlInts * sizeof(int), s) != cudaSuccess) return CHM_ERR_CUDA;
    pass::prep_kernel<T><<<std::min(nb, nsm * 16), 32, 0, s>>>(A);
    pass::trsm_kernel<T, KB><<<nsm, pass::kTrsmWarps * 32, trsm_smem<T, KB>(), s>>>(A);
    if (A.fused || A.kr == 0) return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
    pass::gram_kernel<T, KB><<<std::min(nb, nsm * 16), 32, 0, s>>>(A);
    pass::scan_kernel<T, KB><<<(KB * KB + 31) / 32, 1024, 0, s>>>(A);
    pass::coef_kernel<T, KB><<<std::min(nb, nsm * 8), 32, pass::Packed<KB>::smem, s>>>(A);
    pass::sweep_kernel<T, KB><<<nsm * bps, pass::SweepCfg<T, KB>::WARPS * 32, sweep_smem<T, KB>(), s>>>(A);
    return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

template <typename T>
int launch_pass_kb(const pass::Args<T> &A, PassSpace &ps, cudaStream_t s)
{
    const int kb = A.kb;
    if (kb <= 1) return launch_pass<T, 1>(A, ps, s);
    if (kb <= 2) return launch_pass<T, 2>(A, ps, s);
    if (kb <= 4) return launch_pass<T, 4>(A, ps, s);
    if (kb <= 8) return launch_pass<T, 8>(A, ps, s);
    return launch_pass<T, 16>(A, ps, s);
}

// The kernels' instantiation for kb vectors: the next power of two (P's row stride).
int kb_instance(int kb) { return kb <= 1 ? 1 : kb <= 2 ? 2 : kb <= 4 ? 4 : kb <= 8 ? 8 : 16; }

template <typename T>
int enqueue_passes(T *L, long long n, long long ld, const T *V, long long ldv, long long k,
                   const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                   const PassChoice &ch, const Scratch &sc, PassSpace &ps, T *B, long long ldb, long long nrhs)
{
    const PassLayout lay = pass_layout(n, sizeof(T), ch.seg);
    char *w = ps.buf;
    pass::Args<T> A;
    memset(&A, 0, sizeof(A));
    A.L = L;
    A.n = n;
    A.ld = ld;
    A.ldv = ldv;
    A.nb = (int)((n + pass::kB - 1) / pass::kB);
    A.d = ch.d;
    A.P = reinterpret_cast<T *>(w + lay.P);
    A.Ptag = reinterpret_cast<long long *>(w + lay.Ptag);
    A.Htag = reinterpret_cast<long long *>(w + lay.Htag);
    A.Ztag = reinterpret_cast<long long *>(w + lay.Ztag);
    A.Dinv = reinterpret_cast<T *>(w + lay.Dinv);
    A.G = reinterpret_cast<T *>(w + lay.G);
    A.gram = reinterpret_cast<double *>(w + lay.gram);
    A.H = reinterpret_cast<double *>(w + lay.H);
    A.coef = reinterpret_cast<T *>(w + lay.coef);
    A.escale = reinterpret_cast<T *>(w + lay.escale);
    A.dfac = reinterpret_cast<double *>(w + lay.dfac);
    A.ctl = reinterpret_cast<int *>(w + lay.ctl);
    A.snap = reinterpret_cast<T *>(w + lay.snap);
    A.rst = reinterpret_cast<double *>(w + lay.rst);
    A.tasks = reinterpret_cast<const int2 *>(w + lay.tasks);
    A.post = reinterpret_cast<const int2 *>(w + lay.post);
    A.cflag = reinterpret_cast<int *>(w + lay.cflag);
    A.wprog = reinterpret_cast<long long *>(w + lay.wprog);
    A.fused = ch.fused;
    A.seg = lay.seg;
    A.ws = w;
    A.ws_bytes = ps.bytes;
    A.chk_cut = check_cut();
    A.status = sc.status;
    A.user_info = d_info;
    A.timeout_ns = timeout_ns();
    A.ldb = ldb;
    const int kbmax = ch.kb;
    // right-hand sides the last pass carries.  In float as many as keep it
    // a fused pass of at most 8 vectors (its recurrence task then follows
    // the chain).  In double only those that fill the instantiation's unused
    // columns: the chain block's step there is bound by its FP64 issue,
    // which grows with the kernels' vector count (at n = 32768, k = 1, one
    // carried right-hand side took the pass from 4.4 to about 10 ms, more
    // than chm_solve's whole forward half, whose tasks spread over the SMs).
    const int kr_last = k > 0 ? (int)(k - ((k - 1) / kbmax) * kbmax) : 0;
    const bool dbl = sizeof(T) == 8;
    const int room = dbl ? kb_instance(kr_last) - kr_last : std::max(0, 8 - kr_last);
    const long long nr1 = (nrhs > 0 && k > 0 && ch.fused) ? std::min<long long>(nrhs, room) : 0;
    for (long long q0 = 0; q0 < k; q0 += kbmax) {
        const int kr = (int)std::min<long long>(kbmax, k - q0);
        const int nr = q0 + kbmax >= k ? (int)nr1 : 0;
        A.V = V + q0 * ldv;
        A.kr = kr;
        A.kb = kr + nr;
        A.B = nr > 0 ? B : nullptr;
        unsigned long long mask = 0;
        for (int q = 0; q < kr; ++q)
            if ((sigma ? sigma[q0 + q] : sign) < 0) mask |= 1ull << q;
        A.down_mask = mask;
        A.epoch = ++ps.epoch;
        A.trace = trace_buffer((size_t)A.nb * 16, stream);  // the last pass's, with CHM_TRACE=1
        int rc = launch_pass_kb<T>(A, ps, stream);
        // the carried right-hand sides: L~^{-T} B stands in P's columns kr ..
        if (rc == CHM_OK && nr > 0)
            rc = solve_back_enqueue(L, n, ld, B, ldb, nr, A.P + kr, kb_instance(A.kb), 1, dtype, sc, stream);
        if (rc != CHM_OK) return rc;
    }
    // the other right-hand sides: in double chm_solve's forward and back
    // substitution with the new factor; in float, up to 16 at a time, the
    // substitution (a pass that rotates nothing, one chain step about
    // 1.3 us against chm_solve's 2 to 3) then the back substitution
    if (dbl && nr1 < nrhs) return solve_enqueue(L, n, ld, B + nr1 * ldb, ldb, nrhs - nr1, dtype, sc, stream);
    for (long long r0 = nr1; r0 < nrhs; r0 += pass::kMaxKb) {
        const int nr = (int)std::min<long long>(pass::kMaxKb, nrhs - r0);
        A.V = nullptr;
        A.kr = 0;
        A.kb = nr;
        A.B = B + r0 * ldb;
        A.down_mask = 0;
        A.epoch = ++ps.epoch;
        A.trace = nullptr;
        int rc = launch_pass_kb<T>(A, ps, stream);
        if (rc == CHM_OK) rc = solve_back_enqueue(L, n, ld, B + r0 * ldb, ldb, nr, A.P, kb_instance(nr), 1, dtype, sc, stream);
        if (rc != CHM_OK) return rc;
    }
    return CHM_OK;
}

}  // namespace

int pass_enqueue(void *L, long long n, long long ld, const void *V, long long ldv, long long k,
                 const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                 const PassChoice &ch, const Scratch &sc, PassSpace &ps, void *B, long long ldb, long long nrhs)
{
    int rc = info_init(d_info, 1, stream);
    if (rc != CHM_OK) return rc;
    if (dtype == CHM_F64)
        return enqueue_passes<double>(static_cast<double *>(L), n, ld, static_cast<const double *>(V), ldv, k,
                                      sigma, sign, dtype, stream, d_info, ch, sc, ps, static_cast<double *>(B), ldb,
                                      nrhs);
    return enqueue_passes<float>(static_cast<float *>(L), n, ld, static_cast<const float *>(V), ldv, k, sigma,
                                 sign, dtype, stream, d_info, ch, sc, ps, static_cast<float *>(B), ldb, nrhs);
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
    if (!strcmp(key, "pass_seg")) {
        if (value < 0 || value > (1 << 24)) return CHM_ERR_ARG;
        chm::g_pass_seg.store((int)value);
        return CHM_OK;
    }
    if (!strcmp(key, "pass_fused")) {
        if (value < 0 || value > 1) return CHM_ERR_ARG;
        chm::g_pass_fused.store((int)value);
        return CHM_OK;
    }
#ifdef CHM_CHECK
    if (!strcmp(key, "check_cut")) {
        if (value < 0) return CHM_ERR_ARG;
        chm::g_check_cut.store((long long)value);
        return CHM_OK;
    }
#endif
    return CHM_ERR_ARG;
}

int chm_config_get(const char *key, int64_t *value)
{
    if (!key || !value) return CHM_ERR_ARG;
    if (!strcmp(key, "path")) *value = chm::g_path.load();
    else if (!strcmp(key, "pass_kb")) *value = chm::kb_setting();  // 0: by type
    else if (!strcmp(key, "pass_kb_f32")) *value = chm::pass_kb_of(CHM_F32_MIXED);
    else if (!strcmp(key, "pass_kb_f64")) *value = chm::pass_kb_of(CHM_F64);
    else if (!strcmp(key, "pass_d_f32")) *value = chm::pass_d(CHM_F32_MIXED);
    else if (!strcmp(key, "pass_d_f64")) *value = chm::pass_d(CHM_F64);
    else if (!strcmp(key, "pass_seg")) *value = chm::seg_setting();
    else if (!strcmp(key, "pass_fused")) *value = chm::fused_setting();
#ifdef CHM_CHECK
    else if (!strcmp(key, "checked")) *value = 1;
    else if (!strcmp(key, "check_cut")) *value = chm::check_cut();
#else
    else if (!strcmp(key, "checked")) *value = 0;
#endif
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
