// Autotuning of the single-factor entry points.
//
// The paper fixes its kernels' parameters (Sec. 4.1: blocks per kernel,
// threads per block, elements per thread) for its GPU.  Here they are
// measured: chm_tune times, for one shape, the wave kernel and the pass
// kernels over the vectors per pass, the substitution's lookahead and the
// sweep's segment length, and keeps the fastest in a cache keyed on
// (dtype, floor(log2 n), ceil(log2 k)); later modifications of any shape in
// that bucket take the cached configuration unless a library setting forces
// a parameter.  The cache can be saved to and loaded from a text file.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "chm.h"
#include "chm_internal.h"

namespace chm {

namespace {

struct TuneEntry {
    PassChoice ch;
    long long ns;  // time of one modification when tuned
};

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneEntry> g_tune;
thread_local const PassChoice *t_override = nullptr;

int n_bucket(long long n)
{
    int b = 0;
    while ((2ll << b) <= n) ++b;  // floor(log2 n), n >= 1
    return b;
}
int k_bucket(long long k)
{
    int b = 0;
    while ((1ll << b) < k) ++b;  // ceil(log2 k), k >= 1
    return b;
}

bool valid(const PassChoice &c)
{
    return (c.path == 1 || c.path == 2) && c.kb >= 1 && c.kb <= 16 && c.d >= 2 && c.d <= 10 && c.seg >= 0 &&
           c.seg <= (1 << 24);
}

// A factor of order n with diagonal 1 + u and strictly upper entries
// uniform with variance 1 / n (an upper triangle with positive diagonal is
// the Cholesky factor of L^T L), and V with entries of variance 1 / (4 n k):
// an update by V followed by the downdate by V stays well inside the
// positive definite range.  splitmix64 of the element index and the seed.
__device__ __forceinline__ double unit_of(unsigned long long x)
{
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    x ^= x >> 31;
    return (double)(x >> 11) * 0x1p-53;  // [0, 1)
}
template <typename T>
__global__ void tune_fill(T *L, long long n, T *V, long long k)
{
    const long long tot = n * n, totv = n * k;
    const double s = sqrt(3.0 / (double)n), sv = 0.5 * sqrt(3.0 / ((double)n * (double)k));
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot + totv;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < tot) {
            const long long j = e / n, i = e - j * n;  // column j, row i
            const double u = unit_of((unsigned long long)e);
            L[e] = (T)(i < j ? (2.0 * u - 1.0) * s : i == j ? 1.0 + u : 0.0);
        } else {
            V[e - tot] = (T)((2.0 * unit_of((unsigned long long)e) - 1.0) * sv);
        }
    }
}

}  // namespace

bool tune_lookup(int dtype, long long n, long long k, PassChoice *out)
{
    if (n < 1 || k < 1) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto it = g_tune.find(std::make_tuple(dtype, n_bucket(n), k_bucket(k)));
    if (it == g_tune.end()) return false;
    *out = it->second.ch;
    return true;
}

const PassChoice *tune_override() { return t_override; }

namespace {

// Median time of one modification under `c` (update and downdate pairs),
// or a negative value if a call failed.
double time_choice(const PassChoice &c, void *L, long long n, const void *V, long long k, int dtype,
                   cudaStream_t s, long long *d_info, cudaEvent_t e0, cudaEvent_t e1)
{
    t_override = &c;
    std::vector<float> ts;
    bool ok = true;
    for (int rep = 0; rep < 4 && ok; ++rep) {
        if (cudaEventRecord(e0, s) != cudaSuccess) ok = false;
        for (int sg = 1; sg >= -1 && ok; sg -= 2)
            ok = chm_modify_ex(L, n, n, V, n, k, nullptr, sg, dtype, (chm_stream_t)s, (int64_t *)d_info) == CHM_OK;
        if (ok && cudaEventRecord(e1, s) != cudaSuccess) ok = false;
        if (ok && cudaEventSynchronize(e1) != cudaSuccess) ok = false;
        float ms = 0.f;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ok = false;
        if (ok && rep > 0) ts.push_back(ms / 2.f);  // the first pair warms up
    }
    t_override = nullptr;
    long long h[2] = {0, -1};
    if (!ok || cudaMemcpy(h, d_info, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess || h[0] != 0) return -1.0;
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

template <typename T>
int tune_t(long long n, long long k, int dtype, int64_t *result)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CHM_ERR_CUDA;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return CHM_ERR_CUDA;
    T *L = nullptr, *V = nullptr;
    long long *d_info = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CHM_OK;
    if (cudaMalloc(&L, sizeof(T) * (size_t)n * n) != cudaSuccess || cudaMalloc(&V, sizeof(T) * (size_t)n * k) != cudaSuccess ||
        cudaMalloc(&d_info, 2 * sizeof(long long)) != cudaSuccess)
        rc = CHM_ERR_NOMEM;
    if (rc == CHM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = CHM_ERR_CUDA;
    if (rc == CHM_OK) {
        tune_fill<T><<<1024, 256, 0, s>>>(L, n, V, k);
        if (cudaGetLastError() != cudaSuccess) rc = CHM_ERR_CUDA;
    }
    PassChoice def{1, 16, dtype == CHM_F64 ? 4 : 10, 0, 1};
    PassChoice best{};
    double best_ms = -1.0, def_ms = -1.0;
    auto consider = [&](const PassChoice &c) {
        if (rc != CHM_OK) return -1.0;
        const double ms = time_choice(c, L, n, V, k, dtype, s, d_info, e0, e1);
        if (ms < 0.0) {
            rc = CHM_ERR_CUDA;
            return -1.0;
        }
        if (best_ms < 0.0 || ms < best_ms) {
            best_ms = ms;
            best = c;
        }
        return ms;
    };
    if (rc == CHM_OK) {
        // the built-in choice for this shape, without the cache
        def = builtin_choice(n, k, dtype, false);
        def.kb = (int)std::min<long long>(k, def.kb);
        def_ms = consider(def);
        if (def.path == 2) consider(PassChoice{1, 16, def.d, 0, 1});
        // vectors per pass: min(k, 16) and the two powers of two below it
        const int kb0 = (int)std::min<long long>(k, 16);
        std::vector<int> kbs{kb0};
        int p2 = 1;
        while (p2 * 2 < kb0) p2 *= 2;
        for (; p2 >= 1 && kbs.size() < 3; p2 /= 2)
            if (p2 < kb0) kbs.push_back(p2);
        const std::vector<int> ds = dtype == CHM_F64 ? std::vector<int>{2, 3, 4, 6} : std::vector<int>{4, 6, 8, 10};
        PassChoice bp{2, 16, def.d, 0};
        double bp_ms = -1.0;
        for (int kb : kbs)
            for (int d : ds) {
                const PassChoice c{2, kb, d, 0};
                if (c.kb == def.kb && c.d == def.d && def.path == 2) continue;  // timed as the default
                const double ms = consider(c);
                if (ms >= 0.0 && (bp_ms < 0.0 || ms < bp_ms)) {
                    bp_ms = ms;
                    bp = c;
                }
            }
        if (def.path == 2 && (bp_ms < 0.0 || def_ms < bp_ms)) {
            bp = def;
            bp_ms = def_ms;
        }
        // the sweep's segment length around the default
        const long long nb = (n + 31) / 32;
        for (int seg : {32, 128})
            if (seg < nb) consider(PassChoice{2, bp.kb, bp.d, seg});
    }
    if (rc == CHM_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = CHM_ERR_CUDA;
    release_workspace(dev, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_info);
    cudaFree(V);
    cudaFree(L);
    cudaStreamDestroy(s);
    if (rc != CHM_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[std::make_tuple(dtype, n_bucket(n), k_bucket(k))] = TuneEntry{best, (long long)llround(best_ms * 1e6)};
    }
    if (result) {
        result[0] = best.path;
        result[1] = best.kb;
        result[2] = best.d;
        result[3] = best.seg;
        result[4] = (int64_t)llround(best_ms * 1e6);
        result[5] = (int64_t)llround(def_ms * 1e6);
    }
    return CHM_OK;
}

}  // namespace
}  // namespace chm

extern "C" {

int chm_tune(int64_t n, int64_t k, int dtype, int64_t *result)
{
    if (n < 1 || k < 1 || n > (1ll << 20) || k > 4096 || (dtype != CHM_F64 && dtype != CHM_F32_MIXED))
        return CHM_ERR_ARG;
    return dtype == CHM_F64 ? chm::tune_t<double>(n, k, dtype, result) : chm::tune_t<float>(n, k, dtype, result);
}

int chm_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(chm::g_tune_mu);
    chm::g_tune.clear();
    return CHM_OK;
}

int chm_tune_save(const char *path)
{
    if (!path) return CHM_ERR_ARG;
    FILE *f = fopen(path, "w");
    if (!f) return CHM_ERR_ARG;
    std::lock_guard<std::mutex> lock(chm::g_tune_mu);
    fprintf(f, "chm-tune 1\n");
    for (const auto &kv : chm::g_tune) {
        const chm::PassChoice &c = kv.second.ch;
        fprintf(f, "%d %d %d %d %d %d %d %lld\n", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                c.path, c.kb, c.d, c.seg, kv.second.ns);
    }
    const bool ok = fclose(f) == 0;
    return ok ? CHM_OK : CHM_ERR_ARG;
}

int chm_tune_load(const char *path)
{
    if (!path) return CHM_ERR_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return CHM_ERR_ARG;
    char head[32] = {0};
    std::map<std::tuple<int, int, int>, chm::TuneEntry> got;
    bool ok = fgets(head, sizeof(head), f) && !strcmp(head, "chm-tune 1\n");
    while (ok) {
        int dt, nb, kb, p, q, d, seg;
        long long ns;
        const int m = fscanf(f, "%d %d %d %d %d %d %d %lld", &dt, &nb, &kb, &p, &q, &d, &seg, &ns);
        if (m == EOF) break;
        const chm::PassChoice c{p, q, d, seg};
        if (m != 8 || (dt != CHM_F64 && dt != CHM_F32_MIXED) || nb < 0 || nb > 62 || kb < 0 || kb > 62 ||
            !chm::valid(c) || ns < 0) {
            ok = false;
            break;
        }
        got[std::make_tuple(dt, nb, kb)] = chm::TuneEntry{c, ns};
    }
    fclose(f);
    if (!ok) return CHM_ERR_ARG;  // the cache is left as it was
    std::lock_guard<std::mutex> lock(chm::g_tune_mu);
    for (const auto &kv : got) chm::g_tune[kv.first] = kv.second;
    return CHM_OK;
}

}  // extern "C"
