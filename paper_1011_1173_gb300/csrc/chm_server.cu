// Serving loop for many device-resident factors (chm_server_*): a host
// worker thread admits up/downdate requests against an HBM budget, keeps
// them in per-factor FIFOs and runs continuous batching: whenever one of its
// launch slots is free it packs the oldest ready request of every idle
// factor into one launch of the wave kernel.  Slots launch on their own
// streams with a share of the GPU's resident blocks each, so a launch
// formed from requests that arrived while another was running overlaps it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "chm.h"
#include "chm_internal.h"

namespace chm {

namespace {

constexpr int kMaxSlots = 4;
constexpr int kMaxProbsPerLaunch = 512;

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    long long id = 0;
    long long fid = 0;
    void *V = nullptr;  // server copy, n x k
    int k = 0;
    int sigma = 1;
    size_t bytes = 0;
    double t_arrival = 0.0;
    cudaEvent_t v_ready = nullptr;
};

struct Factor {
    void *L = nullptr;
    long long n = 0;
    size_t bytes = 0;
    std::deque<Request *> fifo;
    bool busy = false;   // a request of it is in a launch
    bool valid = true;   // false after a failed modification
};

struct Done {
    long long id;
    int status;
    double latency;
};

struct Slot {
    cudaStream_t stream = nullptr;
    Scratch sc;
    size_t scratch_bytes = 0;
    Prob *h_probs = nullptr;
    int *h_pair = nullptr;
    long long *h_info = nullptr;
    Prob *d_probs = nullptr;
    int *d_pair = nullptr;
    long long *d_info = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Request *> reqs;
    bool busy = false;
};

struct Server {
    int device = -1;
    int dtype = CHM_F64;
    size_t budget = 0, used = 0;
    int nslots = 2;
    int grid = 0;  // blocks per launch
    cudaStream_t copy_stream = nullptr;
    Slot slots[kMaxSlots];
    std::vector<Factor> factors;
    long long next_req = 1;
    long long outstanding = 0;  // submitted, not yet completed
    std::deque<Done> done;
    std::mutex mu;
    std::condition_variable cv;       // wakes the worker
    std::condition_variable cv_done;  // wakes waiters on completions
    std::thread worker;
    bool stop = false;
    int error = CHM_OK;  // sticky CUDA failure of the worker
    // statistics
    long long launches = 0, launched_requests = 0, completed = 0;
    int max_concurrent = 0;
};

size_t elt_size(int dtype) { return dtype == CHM_F64 ? 8 : 4; }

// Scratch of one launch for one request.
ScratchNeed need_of(long long n, int k)
{
    const ProbShape sh{n, k};
    return scratch_need(&sh, 1);
}

// Complete the launch of a slot (its event has fired); called with the lock held.
void complete_slot(Server *s, Slot &sl)
{
    const double t = now_s();
    for (size_t i = 0; i < sl.reqs.size(); ++i) {
        Request *r = sl.reqs[i];
        Factor &f = s->factors[r->fid];
        const int st = (int)sl.h_info[2 * i];
        if (st != CHM_OK) f.valid = false;
        f.busy = false;
        s->done.push_back(Done{r->id, st, t - r->t_arrival});
        ++s->completed;
        cudaFreeAsync(r->V, sl.stream);
        cudaEventDestroy(r->v_ready);
        s->used -= r->bytes;
        --s->outstanding;
        delete r;
    }
    sl.reqs.clear();
    sl.busy = false;
}

// Requests of factors already marked invalid complete at once with CHM_ERR_STATE.
void drain_invalid(Server *s)
{
    const double t = now_s();
    for (Factor &f : s->factors) {
        if (f.valid || f.busy) continue;
        while (!f.fifo.empty()) {
            Request *r = f.fifo.front();
            f.fifo.pop_front();
            s->done.push_back(Done{r->id, CHM_ERR_STATE, t - r->t_arrival});
            ++s->completed;
            cudaFreeAsync(r->V, s->copy_stream);
            cudaEventDestroy(r->v_ready);
            s->used -= r->bytes;
            --s->outstanding;
            delete r;
        }
    }
}

// Pack ready requests into slot sl and enqueue its launch; lock held.
int launch_slot(Server *s, Slot &sl)
{
    // the oldest ready head of every idle factor, oldest first
    std::vector<Factor *> ready;
    for (Factor &f : s->factors)
        if (!f.busy && f.valid && !f.fifo.empty()) ready.push_back(&f);
    if (ready.empty()) return CHM_OK;
    std::sort(ready.begin(), ready.end(),
              [](const Factor *a, const Factor *b) { return a->fifo.front()->t_arrival < b->fifo.front()->t_arrival; });
    std::vector<ProbShape> shapes;
    size_t fi = 0, fp = 0, fd = 0;
    for (Factor *f : ready) {
        if ((int)sl.reqs.size() >= kMaxProbsPerLaunch) break;
        Request *r = f->fifo.front();
        const ScratchNeed nd = need_of(f->n, r->k);
        if (fi + nd.iflags > sl.sc.iflags_cap || fp + nd.progress > sl.sc.progress_cap ||
            fd + nd.data > sl.sc.data_bytes)
            continue;
        fi += nd.iflags;
        fp += nd.progress;
        fd += nd.data;
        f->fifo.pop_front();
        f->busy = true;
        sl.reqs.push_back(r);
        shapes.push_back(ProbShape{f->n, r->k});
    }
    if (sl.reqs.empty()) return CHM_OK;
    const int np = (int)sl.reqs.size();
    std::vector<Prob> probs(np);
    for (Prob &p : probs) memset(&p, 0, sizeof(p));
    const std::vector<int> pair_prob = carve(shapes.data(), np, sl.sc, probs.data());
    int nbmax = 0;
    for (int i = 0; i < np; ++i) {
        Request *r = sl.reqs[i];
        const Factor &f = s->factors[r->fid];
        Prob &p = probs[i];
        p.L = f.L;
        p.V = r->V;
        p.n = f.n;
        p.ld = f.n;
        p.ldv = f.n;
        p.down_mask = r->sigma < 0 ? (r->k >= 64 ? ~0ull : ((1ull << r->k) - 1)) : 0ull;
        p.info = sl.d_info + 2 * (size_t)i;
        nbmax = std::max(nbmax, p.nb);
        sl.h_probs[i] = p;
    }
    memcpy(sl.h_pair, pair_prob.data(), pair_prob.size() * sizeof(int));
    for (Request *r : sl.reqs)
        if (cudaStreamWaitEvent(sl.stream, r->v_ready, 0) != cudaSuccess) return CHM_ERR_CUDA;
    if (cudaMemcpyAsync(sl.d_probs, sl.h_probs, np * sizeof(Prob), cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return CHM_ERR_CUDA;
    if (cudaMemcpyAsync(sl.d_pair, sl.h_pair, pair_prob.size() * sizeof(int), cudaMemcpyHostToDevice, sl.stream) !=
        cudaSuccess)
        return CHM_ERR_CUDA;
    int rc = info_init(sl.d_info, np, sl.stream);
    if (rc != CHM_OK) return rc;
    LaunchCfg cfg;
    cfg.grid = s->grid;
    rc = launch_wave(s->dtype, nullptr, sl.d_probs, sl.d_pair, np, (int)pair_prob.size(), nbmax, sl.sc, cfg,
                     nullptr, sl.stream);
    if (rc != CHM_OK) return rc;
    if (cudaMemcpyAsync(sl.h_info, sl.d_info, 2 * np * sizeof(long long), cudaMemcpyDeviceToHost, sl.stream) !=
        cudaSuccess)
        return CHM_ERR_CUDA;
    if (cudaEventRecord(sl.done, sl.stream) != cudaSuccess) return CHM_ERR_CUDA;
    sl.busy = true;
    ++s->launches;
    s->launched_requests += np;
    int busy = 0;
    for (int i = 0; i < s->nslots; ++i) busy += s->slots[i].busy ? 1 : 0;
    s->max_concurrent = std::max(s->max_concurrent, busy);
    return CHM_OK;
}

void worker_main(Server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (!s->stop) {
        bool any_busy = false, progressed = false;
        for (int i = 0; i < s->nslots; ++i) {
            Slot &sl = s->slots[i];
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) {
                complete_slot(s, sl);
                progressed = true;
            } else if (q == cudaErrorNotReady) {
                any_busy = true;
            } else {
                s->error = CHM_ERR_CUDA;
                s->stop = true;
            }
        }
        drain_invalid(s);
        if (progressed) s->cv_done.notify_all();
        for (int i = 0; i < s->nslots && !s->stop; ++i) {
            Slot &sl = s->slots[i];
            if (sl.busy) continue;
            const int rc = launch_slot(s, sl);
            if (rc != CHM_OK) {
                s->error = rc;
                s->stop = true;
            }
            if (sl.busy) any_busy = true;
        }
        if (s->stop) break;
        // poll launches in flight closely; otherwise sleep until a submission
        if (any_busy)
            s->cv.wait_for(lock, std::chrono::microseconds(20));
        else
            s->cv.wait_for(lock, std::chrono::milliseconds(5));
    }
    s->cv_done.notify_all();
}

void destroy(Server *s)
{
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < kMaxSlots; ++i) {
        Slot &sl = s->slots[i];
        for (Request *r : sl.reqs) {
            cudaFreeAsync(r->V, nullptr);
            if (r->v_ready) cudaEventDestroy(r->v_ready);
            delete r;
        }
        scratch_free(&sl.sc);
        cudaFreeHost(sl.h_probs);
        cudaFreeHost(sl.h_pair);
        cudaFreeHost(sl.h_info);
        cudaFree(sl.d_probs);
        cudaFree(sl.d_pair);
        cudaFree(sl.d_info);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    for (Factor &f : s->factors) {
        for (Request *r : f.fifo) {
            cudaFreeAsync(r->V, nullptr);
            if (r->v_ready) cudaEventDestroy(r->v_ready);
            delete r;
        }
        cudaFree(f.L);
    }
    cudaDeviceSynchronize();
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
}

int create(size_t budget, int dtype, int max_inflight, Server **out)
{
    Server *s = new Server();
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return CHM_ERR_CUDA;
    }
    s->dtype = dtype;
    s->budget = budget;
    s->nslots = std::max(1, std::min(kMaxSlots, max_inflight <= 0 ? 2 : max_inflight));
    int occ = 0;
    int rc = wave_occupancy(dtype, s->device, &occ);
    if (rc != CHM_OK) {
        delete s;
        return rc;
    }
    s->grid = std::max(2, sm_count(s->device) * occ / s->nslots);
    // scratch per slot: a sixteenth of the budget each, 256 MiB .. 8 GiB
    const size_t per = std::min<size_t>((size_t)8 << 30, std::max<size_t>((size_t)256 << 20, budget / 16));
    if (per * s->nslots >= budget) {
        delete s;
        return CHM_ERR_BUDGET;
    }
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) rc = CHM_ERR_CUDA;
    for (int i = 0; i < s->nslots && rc == CHM_OK; ++i) {
        Slot &sl = s->slots[i];
        // flag and tagged-word regions in proportion to the data region: per
        // 32 columns and wave, ~18 KB of data against 3 int flags and 129 tags
        const size_t iflags = per / 4096, progress = per / 128;
        const size_t data = per - iflags * sizeof(int) - progress * sizeof(long long);
        rc = scratch_alloc(&sl.sc, iflags, progress, data);
        sl.scratch_bytes = per;
        if (rc != CHM_OK) break;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&sl.h_probs, kMaxProbsPerLaunch * sizeof(Prob)) != cudaSuccess ||
            cudaMallocHost(&sl.h_pair, kMaxProbsPerLaunch * (kMaxWaves + 1) * sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&sl.h_info, 2 * kMaxProbsPerLaunch * sizeof(long long)) != cudaSuccess ||
            cudaMalloc(&sl.d_probs, kMaxProbsPerLaunch * sizeof(Prob)) != cudaSuccess ||
            cudaMalloc(&sl.d_pair, kMaxProbsPerLaunch * (kMaxWaves + 1) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&sl.d_info, 2 * kMaxProbsPerLaunch * sizeof(long long)) != cudaSuccess)
            rc = CHM_ERR_NOMEM;
    }
    if (rc == CHM_OK) {
        s->used = per * s->nslots;
        s->worker = std::thread(worker_main, s);
        *out = s;
        return CHM_OK;
    }
    destroy(s);
    return rc;
}

int add_factor(Server *s, const void *L, long long n, long long ld, long long *fid)
{
    if (!L || n <= 0 || ld < n || !fid) return CHM_ERR_ARG;
    const size_t elt = elt_size(s->dtype);
    const size_t bytes = (size_t)n * n * elt;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return CHM_ERR_CUDA;
    if (cur != s->device) return CHM_ERR_STATE;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->error != CHM_OK) return s->error;
        if (s->used + bytes > s->budget) return CHM_ERR_BUDGET;
        s->used += bytes;
    }
    void *d = nullptr;
    int rc = CHM_OK;
    if (cudaMalloc(&d, bytes) != cudaSuccess) rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && cudaMemcpy2D(d, n * elt, L, ld * elt, n * elt, n, cudaMemcpyDefault) != cudaSuccess)
        rc = CHM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(s->mu);
    if (rc != CHM_OK) {
        cudaFree(d);
        s->used -= bytes;
        return rc;
    }
    Factor f;
    f.L = d;
    f.n = n;
    f.bytes = bytes;
    s->factors.push_back(f);
    *fid = (long long)s->factors.size() - 1;
    return CHM_OK;
}

int submit(Server *s, long long fid, const void *V, long long k, int sigma, long long *req_id)
{
    if (!V || k < 1 || k > kMaxWaves || (sigma != 1 && sigma != -1) || !req_id) return CHM_ERR_ARG;
    const double t = now_s();
    const size_t elt = elt_size(s->dtype);
    long long n = 0;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (s->error != CHM_OK) return s->error;
        if (fid < 0 || fid >= (long long)s->factors.size()) return CHM_ERR_ARG;
        n = s->factors[fid].n;
        const ScratchNeed nd = need_of(n, (int)k);
        const Slot &sl = s->slots[0];
        if (nd.iflags > sl.sc.iflags_cap || nd.progress > sl.sc.progress_cap || nd.data > sl.sc.data_bytes)
            return CHM_ERR_BUDGET;
        const size_t bytes = (size_t)n * k * elt;
        if (s->used + bytes > s->budget) return CHM_ERR_BUDGET;
        s->used += bytes;
    }
    Request *r = new Request();
    r->fid = fid;
    r->k = (int)k;
    r->sigma = sigma;
    r->bytes = (size_t)n * k * elt;
    r->t_arrival = t;
    int rc = CHM_OK;
    if (cudaMallocAsync(&r->V, r->bytes, s->copy_stream) != cudaSuccess) rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && cudaMemcpyAsync(r->V, V, r->bytes, cudaMemcpyDefault, s->copy_stream) != cudaSuccess)
        rc = CHM_ERR_CUDA;
    if (rc == CHM_OK && (cudaEventCreateWithFlags(&r->v_ready, cudaEventDisableTiming) != cudaSuccess ||
                         cudaEventRecord(r->v_ready, s->copy_stream) != cudaSuccess))
        rc = CHM_ERR_CUDA;
    // the caller may reuse or free V once this returns, so the copy must have
    // read it: wait for it (it runs on the server's own copy stream, behind no
    // other work, so this is the copy's own time)
    if (rc == CHM_OK && cudaEventSynchronize(r->v_ready) != cudaSuccess) rc = CHM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(s->mu);
    if (rc != CHM_OK) {
        if (r->V) cudaFreeAsync(r->V, s->copy_stream);
        if (r->v_ready) cudaEventDestroy(r->v_ready);
        s->used -= r->bytes;
        delete r;
        return rc;
    }
    r->id = s->next_req++;
    *req_id = r->id;
    s->factors[fid].fifo.push_back(r);
    ++s->outstanding;
    s->cv.notify_all();
    return CHM_OK;
}

int poll(Server *s, long long *ids, int *status, double *latency, int max, int *got)
{
    if (!got || max < 0 || (max > 0 && !ids)) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(s->mu);
    int g = 0;
    while (g < max && !s->done.empty()) {
        const Done d = s->done.front();
        s->done.pop_front();
        ids[g] = d.id;
        if (status) status[g] = d.status;
        if (latency) latency[g] = d.latency;
        ++g;
    }
    *got = g;
    return s->error;
}

int drain(Server *s, double timeout_s)
{
    std::unique_lock<std::mutex> lock(s->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (s->outstanding > 0 && s->error == CHM_OK && !s->stop) {
        if (s->cv_done.wait_until(lock, until) == std::cv_status::timeout && s->outstanding > 0)
            return CHM_ERR_TIMEOUT;
    }
    return s->error;
}

int get_factor(Server *s, long long fid, void *out, long long ld)
{
    std::unique_lock<std::mutex> lock(s->mu);
    if (fid < 0 || fid >= (long long)s->factors.size() || !out) return CHM_ERR_ARG;
    Factor &f = s->factors[fid];
    if (ld < f.n) return CHM_ERR_ARG;
    // wait until the factor has no queued or running request
    while ((f.busy || !f.fifo.empty()) && s->error == CHM_OK && !s->stop)
        s->cv_done.wait_for(lock, std::chrono::milliseconds(1));
    if (s->error != CHM_OK) return s->error;
    const size_t elt = elt_size(s->dtype);
    const int valid = f.valid;
    const void *src = f.L;
    const long long n = f.n;
    lock.unlock();
    if (cudaMemcpy2D(out, ld * elt, src, n * elt, n * elt, n, cudaMemcpyDefault) != cudaSuccess) return CHM_ERR_CUDA;
    return valid ? CHM_OK : CHM_ERR_NOT_PD;
}

int stats(Server *s, long long *out)
{
    std::lock_guard<std::mutex> lock(s->mu);
    out[0] = s->launches;
    out[1] = s->launched_requests;
    out[2] = s->completed;
    out[3] = s->max_concurrent;
    out[4] = (long long)s->used;
    out[5] = s->outstanding;
    return s->error;
}

}  // namespace

}  // namespace chm

extern "C" {

int chm_server_create(size_t hbm_budget_bytes, int dtype, int max_inflight, void **srv)
{
    if (!srv) return CHM_ERR_ARG;
    *srv = nullptr;
    if (dtype != CHM_F64 && dtype != CHM_F32_MIXED) return CHM_ERR_ARG;
    chm::Server *s = nullptr;
    const int rc = chm::create(hbm_budget_bytes, dtype, max_inflight, &s);
    if (rc == CHM_OK) *srv = s;
    return rc;
}

int chm_server_add_factor(void *srv, const void *L, int64_t n, int64_t ld, int64_t *fid)
{
    if (!srv) return CHM_ERR_ARG;
    return chm::add_factor(static_cast<chm::Server *>(srv), L, n, ld, reinterpret_cast<long long *>(fid));
}

int chm_server_submit(void *srv, int64_t fid, const void *V, int64_t k, int sigma, int64_t *req_id)
{
    if (!srv) return CHM_ERR_ARG;
    return chm::submit(static_cast<chm::Server *>(srv), fid, V, k, sigma, reinterpret_cast<long long *>(req_id));
}

int chm_server_poll(void *srv, int64_t *req_ids, int *status, double *latency_s, int max, int *got)
{
    if (!srv) return CHM_ERR_ARG;
    return chm::poll(static_cast<chm::Server *>(srv), reinterpret_cast<long long *>(req_ids), status, latency_s,
                     max, got);
}

int chm_server_drain(void *srv, double timeout_s)
{
    if (!srv || !(timeout_s >= 0.0)) return CHM_ERR_ARG;
    return chm::drain(static_cast<chm::Server *>(srv), timeout_s);
}

int chm_server_get_factor(void *srv, int64_t fid, void *out, int64_t ld)
{
    if (!srv) return CHM_ERR_ARG;
    return chm::get_factor(static_cast<chm::Server *>(srv), fid, out, ld);
}

int chm_server_stats(void *srv, int64_t *out)
{
    if (!srv || !out) return CHM_ERR_ARG;
    return chm::stats(static_cast<chm::Server *>(srv), reinterpret_cast<long long *>(out));
}

int chm_server_destroy(void *srv)
{
    if (!srv) return CHM_ERR_ARG;
    chm::destroy(static_cast<chm::Server *>(srv));
    return CHM_OK;
}

}  // extern "C"
