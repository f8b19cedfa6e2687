// Host-side interface between the translation units of the library: the
// scratch regions a launch of the wave kernel uses, the carving of problems
// into them, and the launch itself (chm_modify.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "chm_layout.h"

namespace chm {

// Scratch of one owner (a stream's workspace, a batch plan, a server, the
// no-allocation array).  The three regions are typed: a word of `iflags`
// only ever holds an int flag and a word of `progress` only a progress
// word, so stale words from earlier launches hold smaller epochs and never
// match.  `ctl` holds kCtlInts control words whose epoch starts at 1.
struct Scratch {
    int *ctl = nullptr;
    long long *status = nullptr;  // {status, row}, sticky
    int *iflags = nullptr;
    size_t iflags_cap = 0;        // ints
    long long *progress = nullptr;
    size_t progress_cap = 0;      // words
    char *data = nullptr;
    size_t data_bytes = 0;
};

// Shape of one problem as the scheduler sees it.
struct ProbShape {
    long long n;
    int k;  // waves in the launch (1 .. kMaxWaves)
};

// Scratch needed by a list of problems laid out one after another.
struct ScratchNeed {
    size_t iflags = 0, progress = 0, data = 0;
    int npairs = 0, nbmax = 0;
};
ScratchNeed scratch_need(const ProbShape *shapes, int count);

// Fill the scratch pointers, nb, k and pair0 of problems[0..count) for the
// layout of scratch_need(); the caller sets L, V, n, ld, ldv, down_mask and
// info.  Returns the pair -> problem map.
std::vector<int> carve(const ProbShape *shapes, int count, const Scratch &sc, Prob *problems);

// Launch configuration.
struct LaunchCfg {
    int groups = 0;       // SM groups (0: automatic)
    int ctas_per_sm = 0;  // resident blocks per SM (0: the occupancy limit)
    int grid = 0;         // blocks of the launch (0: every SM x ctas_per_sm); a
                          // smaller grid leaves room for concurrent launches
    int skip_publish = -1;  // test hook: no wave releases this block's panel, so
                            // its consumers' bounded waits run out (-1: none)
};

// Number of SMs of a device and the occupancy limit of the wave kernel.
int sm_count(int dev);
int wave_occupancy(int dtype, int dev, int *ctas_per_sm);
long long timeout_ns();
int default_groups(int npairs, int nsm, int nprobs);

// Enqueue one launch of the wave kernel on `stream`.  Either one problem
// (`single`, no device tables) or `nprobs` problems whose records are in
// device memory `d_probs` with pair map `d_pair_prob`.  `trace` is null or
// a device array of 2 * npairs * nbmax * kTracePoints words.
int launch_wave(int dtype, const Prob *single, const Prob *d_probs, const int *d_pair_prob,
                int nprobs, int npairs, int nbmax, const Scratch &sc, const LaunchCfg &cfg,
                long long *trace, cudaStream_t stream);

// Set count {status, row} words to {0, -1} on `stream`.
int info_init(long long *d_info, int count, cudaStream_t stream);

// Allocate (and zero) a scratch with at least the given capacities.
int scratch_alloc(Scratch *sc, size_t iflags, size_t progress, size_t data);
// CHM_OK if the current device can dereference p at that address (its own
// device memory, managed memory, or page-locked host memory mapped at the
// same address); CHM_ERR_ARG otherwise (pageable host memory, another
// device's memory, an unknown address).
int check_reachable(const void *p);
// Device bytes the single-factor entry points hold for order n, k vectors.
size_t single_workspace_bytes(long long n, long long k);
// Runs fn on the current device's workspace for `stream` (the one the plain
// entry points use, whose status word chm_status_sync reads), grown first to
// at least `need`, under the workspaces' lock.
int with_stream_scratch(cudaStream_t stream, const ScratchNeed &need, const std::function<int(const Scratch &)> &fn);
void scratch_free(Scratch *sc);

// ---------------------------------------------------------------- pass path

// Workspace of the pass kernels (chm_pass.cuh) of one (device, stream): one
// buffer, carved per pass, whose flag words are zeroed when it is allocated,
// and the epoch that tags each pass's flags (earlier passes' flags hold
// smaller epochs, so no flag needs clearing between passes).
struct PassSpace {
    char *buf = nullptr;
    size_t bytes = 0;
    int epoch = 0;
    long long flag_n = -1;  // the order and element type whose flag layout the buffer holds
    int flag_dtype = -1;
    // the sweep task table the buffer holds: where it is (its offset depends
    // on the element type and the order), the (nb, d, seg) it was built for
    // (nb < 0: none; reset whenever the buffer is allocated) and its length
    const void *task_at = nullptr;
    int task_nb = -1, task_d = -1, task_seg = -1, task_count = 0, post_count = 0;
};
// What a single-factor modification runs: the path and the pass kernels' parameters.
struct PassChoice {
    int path;  // 1 the wave kernel, 2 the pass kernels
    int kb;    // vectors per pass, 1 .. 16
    int d;     // lookahead of the substitution chain (each instantiation clamps it further)
    int seg;   // row blocks per sweep segment (0: by the order)
    int fused; // 1: the substitution kernel's workers also form the coefficients and sweep (up to 8 vectors per pass)
};
// The choice for a modification of this shape: explicit settings, else the
// tuner's candidate while it times one, else the tuning cache (device
// factors), else the built-in rule and defaults.
PassChoice choose_path(long long n, long long k, int dtype, bool host_factor);
// The built-in rule and defaults alone (no settings, no tuning cache).
PassChoice builtin_choice(long long n, long long k, int dtype, bool host_factor);
// The tuning cache (chm_tune.cu): the entry for (dtype, floor(log2 n), ceil(log2 k)).
bool tune_lookup(int dtype, long long n, long long k, PassChoice *out);
// The configuration the tuner is timing on this thread (null outside chm_tune).
const PassChoice *tune_override();
size_t pass_workspace_bytes(long long n, int dtype, int seg);
// Frees the workspace the library keeps for (device, stream), if any; the
// caller has synchronised the stream.
void release_workspace(int dev, cudaStream_t s);
size_t pass_flag_bytes(long long n, int dtype);
// True if a single-factor modification of this shape runs on the pass
// kernels (the library setting "path", else the size rule; a factor in
// page-locked host memory takes the pass kernels, which cross the CPU-GPU
// link three times per pass instead of once per vector).
bool use_pass_path(long long n, long long k, int dtype, bool host_factor);
bool is_host_memory(const void *p);
// The "path" setting in effect (0 automatic, 1 wave kernel, 2 pass kernels).
int path_setting();
// Bounds-checked builds: columns taken off each factor's declared extent by the checks (a test setting; 0 otherwise).
long long check_cut();
// Runs fn on the stream's status word and pass workspace, grown first to
// at least `bytes`, under the workspaces' lock.
int with_pass_workspace(cudaStream_t stream, size_t bytes, long long n, int dtype,
                        const std::function<int(const Scratch &, PassSpace &)> &fn);
// Diagnostics: with CHM_TRACE=1 in the environment, a zeroed device buffer
// of `words` timestamps that chm_trace_dump writes out (null otherwise).
// Called under the workspaces' lock.
long long *trace_buffer(size_t words, cudaStream_t stream);
// Enqueue the passes of one modification (kb <= 16 vectors each).  With
// right-hand sides (B, nrhs > 0; chm_modify_solve) B is then overwritten by
// (L~^T L~)^{-1} B: when passes are fused the last pass's substitution
// carries some of them (float: up to 8 - its update vectors; double: as
// many as fill its kernels' unused vector columns) and its recurrence task
// turns them into L~^{-T} B, then a back substitution; the rest take, in
// float, a substitution of their own with the new factor and a back
// substitution, in double chm_solve's two substitutions (chm_solve.cu).
// `sc` must hold the solve's scratch (solve_need) when nrhs > 0.
int pass_enqueue(void *L, long long n, long long ld, const void *V, long long ldv, long long k,
                 const int8_t *sigma, int sign, int dtype, cudaStream_t stream, long long *d_info,
                 const PassChoice &ch, const Scratch &sc, PassSpace &ps, void *B = nullptr, long long ldb = 0,
                 long long nrhs = 0);
// The solve's scratch for a factor of order n (chm_solve.cu).
ScratchNeed solve_need(long long n);
// chm_solve's forward and back substitution on `sc` (which holds solve_need).
int solve_enqueue(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs, int dtype,
                  const Scratch &sc, cudaStream_t stream);
// Back substitution with the upper factor L: B <- L^{-1} Y, row i of
// right-hand side c of Y at Y[i * ys + c * cs] (element type of dtype).
int solve_back_enqueue(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs,
                       const void *Y, long long ys, long long cs, int dtype, const Scratch &sc, cudaStream_t stream);

}  // namespace chm
