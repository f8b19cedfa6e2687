// Batched up/downdate: many independent factors in one launch of the wave
// kernel, replayed from a CUDA graph, with a launch configuration chosen by
// an autotuner that times candidate configurations on synthetic factors of
// the plan's shapes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "chm.h"
#include "chm_internal.h"

namespace chm {

namespace {

constexpr int kStaging = 2;  // host staging buffers (and graphs) used in turn

struct Plan {
    int device = -1;
    int dtype = CHM_F64;
    int count = 0;
    std::vector<long long> n, ld;
    std::vector<int> k;
    std::vector<int8_t> sign;
    // problems with work, in launch order: order[p] = caller's factor index
    std::vector<int> order;
    bool lpt = true;  // launch order: largest work first (else caller's order)
    int npairs = 0, nbmax = 0;
    std::vector<Prob> tmpl;  // carved records without L and V
    Scratch sc;
    Prob *d_probs = nullptr;
    int *d_pair_prob = nullptr;
    long long *d_info = nullptr;  // [count][2], caller's order
    Prob *h_probs[kStaging] = {nullptr, nullptr};
    cudaGraphExec_t exec[kStaging] = {nullptr, nullptr};
    cudaEvent_t used[kStaging] = {nullptr, nullptr};  // last launch that read staging buffer i
    bool pending[kStaging] = {false, false};
    cudaEvent_t last = nullptr;  // last execution of the plan
    bool any_exec = false;
    int next = 0;
    LaunchCfg cfg;
};

size_t elt_size(int dtype) { return dtype == CHM_F64 ? 8 : 4; }

// Launch order and carved records for the plan's current ordering.
int relayout(Plan *p)
{
    std::vector<int> act;
    for (int i = 0; i < p->count; ++i)
        if (p->n[i] > 0 && p->k[i] > 0) act.push_back(i);
    if (p->lpt) {
        std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
            return (double)p->n[a] * p->n[a] * p->k[a] > (double)p->n[b] * p->n[b] * p->k[b];
        });
    }
    p->order = act;
    std::vector<ProbShape> shapes;
    for (int i : act) shapes.push_back(ProbShape{p->n[i], p->k[i]});
    const ScratchNeed need = scratch_need(shapes.data(), (int)shapes.size());
    p->npairs = need.npairs;
    p->nbmax = need.nbmax;
    p->tmpl.assign(act.size(), Prob());
    for (Prob &pr : p->tmpl) memset(&pr, 0, sizeof(pr));
    if (act.empty()) return CHM_OK;
    const std::vector<int> pair_prob = carve(shapes.data(), (int)shapes.size(), p->sc, p->tmpl.data());
    for (size_t q = 0; q < act.size(); ++q) {
        const int i = act[q];
        Prob &pr = p->tmpl[q];
        pr.n = p->n[i];
        pr.ld = p->ld[i];
        pr.ldv = std::max(1ll, p->n[i]);
        pr.down_mask = p->sign[i] < 0 ? (p->k[i] >= 64 ? ~0ull : ((1ull << p->k[i]) - 1)) : 0ull;
        pr.info = p->d_info + 2 * (size_t)i;
    }
    if (cudaMemcpy(p->d_pair_prob, pair_prob.data(), pair_prob.size() * sizeof(int), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return CHM_ERR_CUDA;
    return CHM_OK;
}

void drop_graphs(Plan *p)
{
    for (int s = 0; s < kStaging; ++s) {
        if (p->pending[s]) cudaEventSynchronize(p->used[s]);
        p->pending[s] = false;
        if (p->exec[s]) cudaGraphExecDestroy(p->exec[s]);
        p->exec[s] = nullptr;
    }
}

void destroy(Plan *p)
{
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (p->device >= 0) cudaSetDevice(p->device);
    drop_graphs(p);
    if (p->any_exec) cudaEventSynchronize(p->last);
    for (int s = 0; s < kStaging; ++s) {
        if (p->used[s]) cudaEventDestroy(p->used[s]);
        if (p->h_probs[s]) cudaFreeHost(p->h_probs[s]);
    }
    if (p->last) cudaEventDestroy(p->last);
    cudaFree(p->d_probs);
    cudaFree(p->d_pair_prob);
    cudaFree(p->d_info);
    scratch_free(&p->sc);
    if (cur >= 0) cudaSetDevice(cur);
    delete p;
}

// The graph of one execution reading staging buffer s: the problem table,
// the status words, the launch.
int capture(Plan *p, int s)
{
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return CHM_ERR_CUDA;
    int rc = CHM_OK;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return CHM_ERR_CUDA;
    }
    const size_t np = p->order.size();
    if (cudaMemcpyAsync(p->d_probs, p->h_probs[s], np * sizeof(Prob), cudaMemcpyHostToDevice, cs) != cudaSuccess)
        rc = CHM_ERR_CUDA;
    if (rc == CHM_OK) rc = info_init(p->d_info, p->count, cs);
    if (rc == CHM_OK)
        rc = launch_wave(p->dtype, nullptr, p->d_probs, p->d_pair_prob, (int)np, p->npairs, p->nbmax, p->sc,
                         p->cfg, nullptr, cs);
    const cudaError_t ec = cudaStreamEndCapture(cs, &g);
    if (rc == CHM_OK && ec != cudaSuccess) rc = CHM_ERR_CUDA;
    if (rc == CHM_OK && cudaGraphInstantiate(&p->exec[s], g, 0) != cudaSuccess) rc = CHM_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    return rc;
}

int execute(Plan *p, void *const *L, const void *const *V, cudaStream_t stream)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CHM_ERR_CUDA;
    if (cur != p->device) return CHM_ERR_STATE;
    const size_t np = p->order.size();
    if (np == 0) return info_init(p->d_info, p->count, stream);
    if (!L || !V) return CHM_ERR_ARG;
    const size_t elt = elt_size(p->dtype);
    const int s = p->next;
    // the graph that last read this staging buffer must have copied it
    if (p->pending[s] && cudaEventSynchronize(p->used[s]) != cudaSuccess) return CHM_ERR_CUDA;
    p->pending[s] = false;
    for (size_t q = 0; q < np; ++q) {
        const int i = p->order[q];
        if (!L[i] || !V[i] || (uintptr_t)L[i] % elt || (uintptr_t)V[i] % elt) return CHM_ERR_ARG;
        int rc = check_reachable(L[i]);
        if (rc == CHM_OK) rc = check_reachable(V[i]);
        if (rc != CHM_OK) return rc;
        Prob pr = p->tmpl[q];
        pr.L = L[i];
        pr.V = V[i];
        p->h_probs[s][q] = pr;
    }
    if (!p->exec[s]) {
        const int rc = capture(p, s);
        if (rc != CHM_OK) return rc;
    }
    // executions of one plan share its scratch: keep them in order
    if (p->any_exec && cudaStreamWaitEvent(stream, p->last, 0) != cudaSuccess) return CHM_ERR_CUDA;
    if (cudaGraphLaunch(p->exec[s], stream) != cudaSuccess) return CHM_ERR_CUDA;
    if (cudaEventRecord(p->used[s], stream) != cudaSuccess) return CHM_ERR_CUDA;
    if (cudaEventRecord(p->last, stream) != cudaSuccess) return CHM_ERR_CUDA;
    p->pending[s] = true;
    p->any_exec = true;
    p->next = (s + 1) % kStaging;
    return CHM_OK;
}

// Synthetic factors of the plan's shapes for timing: L = I, V = 1e-3 (the
// kernel's work and waits do not depend on the values).
struct Synthetic {
    std::vector<void *> L, V;
    ~Synthetic()
    {
        for (void *x : L) cudaFree(x);
        for (void *x : V) cudaFree(x);
    }
};

__global__ void fill_identity(void *L, long long n, long long ld, int f64)
{
    const long long total = n * ld;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e % ld, j = e / ld;
        const double v = (i == j) ? 1.0 : 0.0;
        if (f64) static_cast<double *>(L)[e] = v;
        else static_cast<float *>(L)[e] = (float)v;
    }
}

__global__ void fill_const(void *V, long long count, int f64)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
        if (f64) static_cast<double *>(V)[e] = 1e-3;
        else static_cast<float *>(V)[e] = 1e-3f;
    }
}

int make_synthetic(const Plan *p, Synthetic *syn)
{
    const size_t elt = elt_size(p->dtype);
    syn->L.assign(p->count, nullptr);
    syn->V.assign(p->count, nullptr);
    for (int i = 0; i < p->count; ++i) {
        if (p->n[i] <= 0 || p->k[i] <= 0) continue;
        const long long n = p->n[i];
        if (cudaMalloc(&syn->L[i], (size_t)n * n * elt) != cudaSuccess) return CHM_ERR_NOMEM;
        if (cudaMalloc(&syn->V[i], (size_t)n * p->k[i] * elt) != cudaSuccess) return CHM_ERR_NOMEM;
        fill_identity<<<256, 256>>>(syn->L[i], n, n, p->dtype == CHM_F64);
        fill_const<<<64, 256>>>(syn->V[i], n * (long long)p->k[i], p->dtype == CHM_F64);
    }
    return cudaDeviceSynchronize() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

// Time one configuration: one untimed execution, then the best of `reps`.
int time_config(Plan *p, const Synthetic &syn, cudaStream_t stream, int reps, float *ms)
{
    // synthetic factors are square (ld = n)
    std::vector<long long> ld_save = p->ld;
    for (int i = 0; i < p->count; ++i) p->ld[i] = std::max(1ll, p->n[i]);
    int rc = relayout(p);
    p->ld = ld_save;
    if (rc != CHM_OK) return rc;
    drop_graphs(p);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r <= reps && rc == CHM_OK; ++r) {
        cudaEventRecord(a, stream);
        rc = execute(p, syn.L.data(), syn.V.data(), stream);
        cudaEventRecord(b, stream);
        if (rc == CHM_OK && cudaEventSynchronize(b) != cudaSuccess) rc = CHM_ERR_CUDA;
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        if (r > 0) best = std::min(best, t);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *ms = best;
    return rc;
}

int autotune(Plan *p, cudaStream_t stream)
{
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CHM_ERR_CUDA;
    if (cur != p->device) return CHM_ERR_STATE;
    if (p->order.empty()) return CHM_OK;
    Synthetic syn;
    int rc = make_synthetic(p, &syn);
    if (rc != CHM_OK) return rc;
    const int nsm = sm_count(p->device);
    int occ = 0;
    rc = wave_occupancy(p->dtype, p->device, &occ);
    if (rc != CHM_OK) return rc;
    std::vector<int> groups;
    for (int d : {16, 12, 9, 7, 6, 5, 4, 3, 2}) {
        const int g = std::max(1, std::min(std::min(p->npairs, kMaxGroups), nsm / d));
        if (std::find(groups.begin(), groups.end(), g) == groups.end()) groups.push_back(g);
    }
    const LaunchCfg keep = p->cfg;
    const bool keep_lpt = p->lpt;
    float best = 1e30f;
    LaunchCfg best_cfg = keep;
    bool best_lpt = keep_lpt;
    for (int lpt = 1; lpt >= 0; --lpt) {
        for (int g : groups) {
            for (int c = occ; c >= std::max(1, occ - 1); --c) {
                p->lpt = lpt != 0;
                p->cfg.groups = g;
                p->cfg.ctas_per_sm = c;
                float t = 0.f;
                rc = time_config(p, syn, stream, 2, &t);
                if (rc != CHM_OK) break;
                if (t < best) {
                    best = t;
                    best_cfg = p->cfg;
                    best_lpt = p->lpt;
                }
            }
            if (rc != CHM_OK) break;
        }
        if (rc != CHM_OK) break;
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess && rc == CHM_OK) rc = CHM_ERR_CUDA;
    p->cfg = rc == CHM_OK ? best_cfg : keep;
    p->lpt = rc == CHM_OK ? best_lpt : keep_lpt;
    drop_graphs(p);
    const int rc2 = relayout(p);
    return rc != CHM_OK ? rc : rc2;
}

}  // namespace

}  // namespace chm

extern "C" {

int chm_batch_plan_create(int count, const int64_t *n, const int64_t *ld, const int64_t *k,
                          const int8_t *sigma, int dtype, void **plan)
{
    using namespace chm;
    if (!plan) return CHM_ERR_ARG;
    *plan = nullptr;
    if (count < 0 || (count > 0 && (!n || !ld || !k))) return CHM_ERR_ARG;
    if (dtype != CHM_F64 && dtype != CHM_F32_MIXED) return CHM_ERR_ARG;
    for (int i = 0; i < count; ++i) {
        if (n[i] < 0 || n[i] > (1ll << 26) || ld[i] < std::max<int64_t>(1, n[i])) return CHM_ERR_ARG;
        if (k[i] < 0 || k[i] > kMaxWaves) return CHM_ERR_ARG;
        if (sigma && sigma[i] != 1 && sigma[i] != -1) return CHM_ERR_ARG;
    }
    Plan *p = new Plan();
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return CHM_ERR_CUDA;
    }
    p->dtype = dtype;
    p->count = count;
    p->n.assign(n, n + count);
    p->ld.assign(ld, ld + count);
    p->k.resize(count);
    p->sign.resize(count);
    std::vector<ProbShape> shapes;
    for (int i = 0; i < count; ++i) {
        p->k[i] = (int)k[i];
        p->sign[i] = sigma ? sigma[i] : 1;
        if (n[i] > 0 && k[i] > 0) shapes.push_back(ProbShape{n[i], (int)k[i]});
    }
    const ScratchNeed need = scratch_need(shapes.data(), (int)shapes.size());
    int rc = CHM_OK;
    if (cudaMalloc(&p->d_info, 2 * sizeof(long long) * std::max(1, count)) != cudaSuccess) rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && cudaMalloc(&p->d_probs, sizeof(Prob) * std::max<size_t>(1, shapes.size())) != cudaSuccess)
        rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && cudaMalloc(&p->d_pair_prob, sizeof(int) * std::max(1, need.npairs)) != cudaSuccess)
        rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK) rc = scratch_alloc(&p->sc, need.iflags, need.progress, std::max<size_t>(need.data, 256));
    for (int s = 0; s < kStaging && rc == CHM_OK; ++s) {
        if (cudaMallocHost(&p->h_probs[s], sizeof(Prob) * std::max<size_t>(1, shapes.size())) != cudaSuccess)
            rc = CHM_ERR_NOMEM;
        else if (cudaEventCreateWithFlags(&p->used[s], cudaEventDisableTiming) != cudaSuccess)
            rc = CHM_ERR_CUDA;
    }
    if (rc == CHM_OK && cudaEventCreateWithFlags(&p->last, cudaEventDisableTiming) != cudaSuccess) rc = CHM_ERR_CUDA;
    if (rc == CHM_OK) rc = relayout(p);
    // the kernel's one-time set-up happens here, outside any stream capture
    int occ = 0;
    if (rc == CHM_OK) rc = wave_occupancy(dtype, p->device, &occ);
    if (rc == CHM_OK) rc = info_init(p->d_info, count, nullptr);
    if (rc == CHM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = CHM_ERR_CUDA;
    if (rc != CHM_OK) {
        destroy(p);
        return rc;
    }
    *plan = p;
    return CHM_OK;
}

int chm_batch_autotune(void *plan, chm_stream_t stream)
{
    if (!plan) return CHM_ERR_ARG;
    return chm::autotune(static_cast<chm::Plan *>(plan), (cudaStream_t)stream);
}

int chm_batch_config(void *plan, int *groups, int *ctas_per_sm, int *largest_first)
{
    if (!plan) return CHM_ERR_ARG;
    const chm::Plan *p = static_cast<const chm::Plan *>(plan);
    if (groups) *groups = p->cfg.groups;
    if (ctas_per_sm) *ctas_per_sm = p->cfg.ctas_per_sm;
    if (largest_first) *largest_first = p->lpt ? 1 : 0;
    return CHM_OK;
}

int chm_batch_execute(void *plan, void *const *L, const void *const *V, chm_stream_t stream)
{
    if (!plan) return CHM_ERR_ARG;
    return chm::execute(static_cast<chm::Plan *>(plan), L, V, (cudaStream_t)stream);
}

int chm_batch_status(void *plan, int64_t *info)
{
    if (!plan || !info) return CHM_ERR_ARG;
    chm::Plan *p = static_cast<chm::Plan *>(plan);
    if (p->any_exec && cudaEventSynchronize(p->last) != cudaSuccess) return CHM_ERR_CUDA;
    if (p->count == 0) return CHM_OK;
    std::vector<long long> h(2 * (size_t)p->count);
    if (cudaMemcpy(h.data(), p->d_info, h.size() * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CHM_ERR_CUDA;
    int first = CHM_OK;
    for (int i = 0; i < p->count; ++i) {
        info[2 * i] = h[2 * i];
        info[2 * i + 1] = h[2 * i + 1];
        if (first == CHM_OK && h[2 * i] != 0) first = (int)h[2 * i];
    }
    return first;
}

int chm_batch_plan_destroy(void *plan)
{
    if (!plan) return CHM_ERR_ARG;
    chm::destroy(static_cast<chm::Plan *>(plan));
    return CHM_OK;
}

}  // extern "C"
