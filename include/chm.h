/*
 * chm.h - C ABI of the GB300 rank-k Cholesky up/downdate library.
 *
 * Operation (Walder 2010, Sec. 1): given an upper-triangular factor L of
 * order n with positive diagonal, A = L^T L, and V in R^{n x k}, overwrite L
 * with the factor Lt such that
 *
 *     Lt^T Lt = A + V diag(sigma) V^T,      sigma_p in {+1 (update), -1 (downdate)}
 *
 * by the hyperbolic rotations of Algorithm 1 (Compute / Apply), in O(k n^2)
 * work.  The k columns of V are processed in ascending order, which yields
 * the same factor as k successive rank-1 modifications.
 *
 * Conventions shared by every entry point:
 *   - Layout.  L is column-major upper triangular with leading dimension ld
 *     (LAPACK uplo = 'U', Matlab's chol convention): element (i, j), i <= j,
 *     is at L[i + j*ld].  Only the upper triangle including the diagonal is
 *     read or written; the strictly lower part and the rows n..ld-1 of each
 *     column are left bit-for-bit unchanged.  V is column-major n x k with
 *     leading dimension ldv (ldv = n in the short forms); column p is the
 *     p-th update vector.  V is read only.
 *   - Pointers.  L, V and d_info are pointers the current device can
 *     dereference, owned by the caller (the library never frees them):
 *     device memory of the current device, managed memory, or page-locked
 *     host memory (cudaHostAlloc, cudaHostRegister) mapped at the same
 *     address, which every unified-addressing system provides.  Pageable
 *     host memory and other devices' memory are rejected with CHM_ERR_ARG
 *     before any work is enqueued.  With L in page-locked host memory the
 *     kernel reads and writes the factor in place across the CPU-GPU link
 *     and the device holds only the O(n k) workspace of chm_workspace_bytes:
 *     the paper's property that device memory grows as O(n), not O(n^2)
 *     (abstract, Sec. 5), so a factor may be as large as host memory.
 *     L and V must be aligned to their element size.  sigma arrays are HOST
 *     pointers.
 *   - Precision.  CHM_F64: L and V are double; all arithmetic in double.
 *     CHM_F32_MIXED: L and V are float; the Apply sweep runs in float while
 *     every Compute step runs in double on the promoted float values.  The
 *     vectors are taken in groups (those of one launch of the wave kernel,
 *     or one pass of the pass kernels): within a group each diagonal entry
 *     is carried in double from vector to vector and rounded to float once,
 *     after the group's last vector; the ratios that enter Apply (c and s,
 *     or the pass kernels' sweep coefficients) are rounded to float.  The
 *     result differs from that of the serial Algorithm 1 in the same split
 *     by float rounding only: its column-scaled error is bounded by
 *     8 u_f sqrt(n k) with u_f = 2^-24.
 *   - Streams.  Work is enqueued on `stream` (a cudaStream_t; NULL means the
 *     legacy default stream of the current device) and the call returns
 *     without synchronising.  L is modified in place in stream order.
 *   - Errors.  A call returns synchronously only argument errors
 *     (CHM_ERR_ARG), allocation failures (CHM_ERR_NOMEM) and launch errors
 *     (CHM_ERR_CUDA).  Conditions found on the device are recorded in a
 *     per-(device, stream) status word that stays set until read by
 *     chm_status_sync: CHM_ERR_NOT_PD (a Compute step found L_ii <= 0 or
 *     L_ii^2 + sigma V_i^2 <= 0 or a non-finite value; info = the 0-based
 *     row) and CHM_ERR_TIMEOUT (a wait between thread blocks exceeded its
 *     bound; info = the column block whose wait ran out, or a negative code
 *     for the launch's other waits, -5 for a problem of a batch or server
 *     launch that stopped because another problem's wait ran out).  After
 *     either, L is unspecified.
 *   - Bounds-checked build.  The same sources compiled with -DCHM_CHECK
 *     (libchm_check.so, built beside libchm.so) check every global index
 *     the kernels form: each element of L against the upper triangle of its
 *     leading n x n block with leading dimension ld, each element of V and
 *     of a solve's B against their leading n rows and k (nrhs) columns, and
 *     every workspace region against its allocation.  A failed check skips
 *     the access, records CHM_ERR_BOUNDS (info = the element's offset from
 *     the array's base, or the region's byte offset from its allocation)
 *     and ends the launch's waits; nothing traps.  chm_config_get("checked")
 *     says which build is loaded (1 checked, 0 not).
 *   - Memory.  The library keeps a workspace per (device, stream): per
 *     vector of a launch (at most 64 per launch) rotation panels, ratio
 *     tiles and flags of about 19 KB per 32 rows, and the status word
 *     (chm_workspace_bytes gives the total).  It is allocated on the first
 *     call that needs a larger one; later calls of the same or smaller size
 *     allocate nothing.
 *
 * Thread safety: entry points may be called from several host threads; calls
 * on the same stream from different threads must be ordered by the caller.
 */
#ifndef CHM_H
#define CHM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so that this header needs no CUDA header. */
typedef struct CUstream_st *chm_stream_t;

typedef enum {
    CHM_F64 = 0,       /* double storage, double arithmetic */
    CHM_F32_MIXED = 1  /* float storage and Apply, double Compute */
} chm_dtype;

typedef enum {
    CHM_OK = 0,
    CHM_ERR_ARG = -1,
    CHM_ERR_NOT_PD = -2,
    CHM_ERR_TIMEOUT = -3,
    CHM_ERR_CUDA = -4,
    CHM_ERR_NOMEM = -5,
    CHM_ERR_BUDGET = -6,
    CHM_ERR_STATE = -7,
    CHM_ERR_BOUNDS = -8  /* bounds-checked build only: a kernel index outside its array */
} chm_status;

/*
 * Rank-k update (sigma = +1 for every column): L <- Lt with
 * Lt^T Lt = L^T L + V V^T.  Algorithm 1 with sigma = +1 (Sec. 2); the
 * k-column blocking follows Sec. 4.1.
 *   L      device, n x n upper factor, leading dimension ld (in/out)
 *   n      order, n >= 0 (n == 0 is a no-op)
 *   ld     leading dimension of L, ld >= max(1, n)
 *   V      device, n x k, leading dimension n (read only)
 *   k      number of update vectors, k >= 0 (k == 0 is a no-op)
 *   dtype  CHM_F64 or CHM_F32_MIXED (element type of L and V)
 *   stream CUDA stream
 * Returns CHM_OK or CHM_ERR_ARG / CHM_ERR_NOMEM / CHM_ERR_CUDA.
 */
int chm_update(void *L, int64_t n, int64_t ld, const void *V, int64_t k, int dtype,
               chm_stream_t stream);

/*
 * Rank-k downdate (sigma = -1 for every column): Lt^T Lt = L^T L - V V^T.
 * Same arguments and errors as chm_update.  If L^T L - V V^T is not
 * positive definite, the stream's status word records CHM_ERR_NOT_PD.
 */
int chm_downdate(void *L, int64_t n, int64_t ld, const void *V, int64_t k, int dtype,
                 chm_stream_t stream);

/*
 * General form: per-column signs and an explicit leading dimension for V.
 *   ldv    leading dimension of V, ldv >= max(1, n)
 *   sigma  HOST array of k entries, each +1 or -1; if NULL every column uses `sign`
 *   sign   +1 or -1, used when sigma == NULL
 *   d_info optional DEVICE int64[2]; if non-NULL the library sets it to
 *          {CHM_OK, -1} on the stream before the work and the device writes
 *          {status, info} there if this call hits CHM_ERR_NOT_PD or
 *          CHM_ERR_TIMEOUT (the per-stream status word is written as well)
 * Each column uses its own sign in both Compute and Apply (a generalisation
 * of Algorithm 1, where sigma is one scalar).
 */
int chm_modify_ex(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k,
                  const int8_t *sigma, int sign, int dtype, chm_stream_t stream,
                  int64_t *d_info);

/*
 * Same operation and arguments as chm_modify_ex, for callers that cannot
 * allocate device memory: code that must not call cudaMalloc, such as a
 * real-time or memory-budgeted host thread whose process has handed all
 * device memory to its own allocator, or an application whose allocator
 * forbids allocations outside its own pool (cudaMalloc can block, fail under
 * the budget, or synchronise the device).  It calls no cudaMalloc, cudaFree
 * or allocating library routine.  The paper has no
 * counterpart; this is a deployment variant of the same computation.
 *
 * Scratch: a file-scope device array of 16 MiB that every GPU which loads
 * the library holds until the process exits.  It limits the order to
 * n <= 8192 (larger n returns CHM_ERR_BUDGET before any work is enqueued) and
 * the vectors per launch (more vectors are processed in several launches).
 * The first call on a device (with that device current) looks up the array's
 * device address and clears its flag words; make that first call before any
 * stream capture.  All calls share the array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU (different streams, or
 * different host threads without ordering) race and give wrong results.
 * Device-side errors (CHM_ERR_NOT_PD, CHM_ERR_TIMEOUT) are reported only
 * through d_info; chm_status_sync does not see this variant's status, so
 * d_info is required here whenever n > 0 and k > 0 (NULL returns
 * CHM_ERR_ARG).
 * Returns CHM_OK or CHM_ERR_ARG / CHM_ERR_BUDGET / CHM_ERR_CUDA.
 */
int chm_modify_noalloc(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k,
                       const int8_t *sigma, int sign, int dtype, chm_stream_t stream,
                       int64_t *d_info);

/*
 * Batched up/downdate of many independent factors (a systems form of the
 * method; Sec. 4.1's rank-k blocking applied to each factor).  A plan fixes
 * the shapes; each execution takes the factors' and update blocks' device
 * addresses and runs every factor in ONE launch of the wave kernel, replayed
 * from a CUDA graph captured by the plan (a copy of the problem table from
 * pinned host memory, a reset of the per-factor status words, the launch).
 *
 * chm_batch_plan_create
 *   count   number of factors, >= 0
 *   n, ld   HOST arrays [count]: order and leading dimension of factor i
 *   k       HOST array [count]: update vectors of factor i, 0 <= k_i <= 64
 *   sigma   HOST array [count] of +1 (update) / -1 (downdate) per factor,
 *           or NULL for all updates
 *   dtype   CHM_F64 or CHM_F32_MIXED
 *   plan    receives the plan
 * Factors with n_i == 0 or k_i == 0 are no-ops.  V_i is n_i x k_i
 * column-major with leading dimension n_i.  The plan owns all device scratch
 * (about n_i * 19 KB per vector of every factor) and pinned staging memory;
 * nothing is allocated by chm_batch_execute.  The current device at creation
 * is the plan's device.  Returns CHM_OK, CHM_ERR_ARG, CHM_ERR_NOMEM or
 * CHM_ERR_CUDA.
 *
 * chm_batch_autotune: times candidate launch configurations (SM groups,
 * blocks per SM, largest-work-first or caller order) on synthetic factors of
 * the plan's shapes (L = I, V = 1e-3, allocated for the duration of the call)
 * and keeps the fastest.  Synchronises `stream`.  The plan's status words
 * are reset.  Returns CHM_OK, CHM_ERR_NOMEM (no room for the synthetic
 * factors; the plan keeps its configuration), CHM_ERR_STATE (another device
 * is current) or CHM_ERR_CUDA.
 *
 * chm_batch_config: the configuration in use (groups 0 = automatic,
 * ctas_per_sm 0 = occupancy limit, largest_first 1/0); any pointer may be NULL.
 *
 * chm_batch_execute
 *   L, V    HOST arrays [count] of DEVICE pointers (entries of no-op factors
 *           are ignored); L[i] is modified in place, V[i] is read only
 * Enqueues the execution on `stream` and returns.  Executions of one plan
 * run in the order they are enqueued, on any streams; a plan must not be
 * used from several host threads at once.  Returns CHM_OK, CHM_ERR_ARG
 * (null or misaligned pointer), CHM_ERR_STATE (wrong device) or CHM_ERR_CUDA.
 *
 * chm_batch_status: waits for the plan's last execution and copies the
 * per-factor {status, row} words into the HOST array info[2 * count]
 * ({CHM_OK, -1} for factors without a device-side error).  Returns the first
 * non-OK status in factor order, else CHM_OK.
 *
 * chm_batch_plan_destroy: waits for the plan's work and frees it.
 */
int chm_batch_plan_create(int count, const int64_t *n, const int64_t *ld, const int64_t *k,
                          const int8_t *sigma, int dtype, void **plan);
int chm_batch_autotune(void *plan, chm_stream_t stream);
int chm_batch_config(void *plan, int *groups, int *ctas_per_sm, int *largest_first);
int chm_batch_execute(void *plan, void *const *L, const void *const *V, chm_stream_t stream);
int chm_batch_status(void *plan, int64_t *info);
int chm_batch_plan_destroy(void *plan);

/*
 * Serving: many factors resident in device memory, up/downdate requests
 * admitted against a memory budget and run by continuous batching (a
 * systems form of the method; each request is Algorithm 1 with its own V
 * and sign).  A worker thread keeps one FIFO per factor; whenever one of
 * its launch slots is free it packs the oldest ready request of every idle
 * factor into one launch of the wave kernel on that slot's stream.  Each
 * slot launches with 1/max_inflight of the GPU's resident blocks, so a
 * launch formed from requests that arrived while another was running
 * overlaps it on the device.  Requests on one factor run one after another
 * in submission order, each in its own launch; a factor's result is
 * bit-identical to applying the same requests alone with chm_modify_ex.
 *
 * chm_server_create
 *   hbm_budget_bytes  device memory the server may hold: factors (n^2
 *                     elements each), queued update blocks and the launch
 *                     slots' scratch (a sixteenth of the budget per slot,
 *                     between 256 MiB and 8 GiB)
 *   dtype             CHM_F64 or CHM_F32_MIXED for every factor
 *   max_inflight      launch slots (concurrent launches), 1..4; <= 0 means 2
 *   srv               receives the server
 *   Returns CHM_OK, CHM_ERR_ARG, CHM_ERR_BUDGET (budget below the slots'
 *   scratch), CHM_ERR_NOMEM or CHM_ERR_CUDA.  The current device is the
 *   server's device.
 * chm_server_add_factor: copies the upper factor L (n x n, leading dimension
 *   ld, HOST or DEVICE memory) into the server; fid receives its id (0, 1,
 *   ...).  Synchronous.  CHM_ERR_BUDGET if it does not fit the budget.
 * chm_server_submit: queues L_fid <- modification by V (n x k column-major,
 *   leading dimension n, HOST or DEVICE memory, 1 <= k <= 64) with sign
 *   sigma = +1 or -1.  V must hold its final values when the call is made:
 *   the server copies it on a stream of its own, which is not ordered after
 *   the caller's streams, so a V written by GPU work must have that work
 *   synchronised first.  The call returns once the copy has read V (the
 *   caller may then reuse or free it); it does not wait for the modification
 *   or for other GPU work.  req_id receives the request id (1, 2, ...).
 *   CHM_ERR_BUDGET if the block does not fit the budget or a launch slot's
 *   scratch.
 * chm_server_poll: moves up to `max` completed requests into req_ids[],
 *   status[] (CHM_OK, CHM_ERR_NOT_PD, CHM_ERR_TIMEOUT, or CHM_ERR_STATE for a
 *   request on a factor invalidated by an earlier failure) and latency_s[]
 *   (seconds from submission to the worker seeing the launch complete);
 *   status and latency_s may be NULL.  *got receives the count.  Does not
 *   block.  Returns CHM_OK or the worker's sticky CUDA error.
 * chm_server_drain: waits until every submitted request has completed or
 *   timeout_s has passed (CHM_ERR_TIMEOUT).
 * chm_server_get_factor: waits until factor fid has no queued or running
 *   request, then copies it to `out` (HOST or DEVICE, leading dimension ld,
 *   n x n with the strictly lower part as stored).  Returns CHM_ERR_NOT_PD
 *   (after copying) if a modification of this factor failed.  Submissions
 *   on fid during the copy race with it.
 * chm_server_stats: out[6] = {launches, requests launched, requests
 *   completed, largest number of launches seen in flight at once, device
 *   bytes held, requests outstanding}.
 * chm_server_destroy: stops the worker, waits for the device and frees
 *   everything; requests still queued are dropped.
 * A server may be used from several host threads.
 */
int chm_server_create(size_t hbm_budget_bytes, int dtype, int max_inflight, void **srv);
int chm_server_add_factor(void *srv, const void *L, int64_t n, int64_t ld, int64_t *fid);
int chm_server_submit(void *srv, int64_t fid, const void *V, int64_t k, int sigma, int64_t *req_id);
int chm_server_poll(void *srv, int64_t *req_ids, int *status, double *latency_s, int max, int *got);
int chm_server_drain(void *srv, double timeout_s);
int chm_server_get_factor(void *srv, int64_t fid, void *out, int64_t ld);
int chm_server_stats(void *srv, int64_t *out);
int chm_server_destroy(void *srv);

/*
 * Solve with a factor: B <- X = (L^T L)^{-1} B, the use a maintained
 * Cholesky factor serves (Sec. 1: the factor of A is kept so that systems
 * with A, here the modified matrix, can be solved).  A forward substitution
 * with L^T followed by a back substitution with L.
 *   L      upper factor as for chm_update (read only; device memory or
 *          page-locked host memory), leading dimension ld >= max(1, n)
 *   n      order, n >= 0 (n == 0 is a no-op)
 *   B      n x nrhs column-major, leading dimension ldb >= max(1, n),
 *          overwritten with X (same memory kinds as L); rows n..ldb-1 are
 *          left unchanged
 *   nrhs   number of right-hand sides, nrhs >= 0 (0 is a no-op)
 *   dtype  CHM_F64: double L and B, double arithmetic.  CHM_F32_MIXED: float
 *          L and B, every product and sum in double, X rounded to float once
 * Stream-ordered like chm_update (enqueue it after a modification on the
 * same stream to solve with the modified factor).  Each 32 x 32 diagonal
 * block is applied through its explicit inverse.  If some L_ii <= 0 or is
 * not finite, the stream's status word records CHM_ERR_NOT_PD with that row
 * and X is unspecified.  Uses the stream's workspace (O(n) bytes).
 * Returns CHM_OK, CHM_ERR_ARG, CHM_ERR_NOMEM or CHM_ERR_CUDA.
 */
int chm_solve(const void *L, int64_t n, int64_t ld, void *B, int64_t ldb, int64_t nrhs, int dtype,
              chm_stream_t stream);

/*
 * Modify, then solve with the modified factor (Sec. 1: the factor is kept
 * up to date in order to solve with the modified matrix): L <- L~ as
 * chm_modify_ex does, then B <- (L~^T L~)^{-1} B as chm_solve does.
 *   L, n, ld, V, ldv, k, sigma, sign, dtype, stream, d_info  as for
 *          chm_modify_ex
 *   B, ldb, nrhs  as for chm_solve (B must not overlap L or V)
 * Where the modification runs on the pass kernels (large factors, see
 * chm_config_set), the forward half of the solve is fused into its last
 * pass: appending L^{-T} B to the factor as extra columns (the factor of
 * [[A, B], [B^T, c]]), the last pass's substitution carries B's columns
 * beside V's and a recurrence task applies the pass's rotations to them,
 * which leaves L~^{-T} B without another crossing of the factor, and the
 * back substitution follows.  In float up to 8 - (vectors of the last pass)
 * right-hand sides ride that way and the others take a substitution with the
 * new factor of their own; in double only as many as fill the last pass's
 * unused vector columns (its chain is bound by the FP64 rate), the others
 * take chm_solve's two substitutions.  Otherwise the two calls follow each
 * other on the stream.  Precision: CHM_F64 in double; CHM_F32_MIXED as each part of
 * the pair: a carried right-hand side's forward half in float like the
 * pass's Apply, the back substitution with double arithmetic on float data.
 * d_info receives the modification's status; a failure of the solve part
 * (a diagonal entry not positive) goes to the stream's status word
 * (chm_status_sync).  k == 0 is chm_solve alone, nrhs == 0 chm_modify_ex
 * alone.  Returns CHM_OK, CHM_ERR_ARG, CHM_ERR_NOMEM or CHM_ERR_CUDA.
 */
int chm_modify_solve(void *L, int64_t n, int64_t ld, const void *V, int64_t ldv, int64_t k, const int8_t *sigma,
                     int sign, void *B, int64_t ldb, int64_t nrhs, int dtype, chm_stream_t stream, int64_t *d_info);

/*
 * Device memory that chm_update / chm_downdate / chm_modify_ex hold for one
 * factor of order n modified by k vectors (the per-stream workspace; the
 * factor and V themselves are the caller's), for the path the "path"
 * setting forces, or under the automatic rule the larger of the two paths'
 * (the wave kernel's grows as O(n min(k, 64)), the pass kernels' as O(n)).
 * Either way it is O(n min(k, 64)):
 * with L in page-locked host memory this is all the device memory a
 * modification needs (abstract, Sec. 5: O(n) device memory).  Host only.
 *   bytes  receives the size
 * Returns CHM_OK or CHM_ERR_ARG (n or k negative or n > 2^26, bad dtype,
 * bytes NULL).
 */
int chm_workspace_bytes(int64_t n, int64_t k, int dtype, size_t *bytes);

/*
 * Synchronises `stream`, then reads and clears the status word of the
 * current device and that stream.
 *   info   optional HOST int64[2] receiving {status, info}
 * Returns the recorded status (CHM_OK if no call since the last read hit a
 * device-side error), or CHM_ERR_CUDA if the synchronisation failed.
 */
int chm_status_sync(chm_stream_t stream, int64_t *info);

/* Human-readable name of a status code (static string). */
const char *chm_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int chm_version(void);

/*
 * Microbenchmarks of the hardware facts the kernel is designed around
 * (diagnostics; the up/downdate entry points never call them).  Runs on the
 * current device, allocates and frees its own buffers, synchronises.
 *   which   one of chm_microbench_kind
 *   out     HOST array of at least 2 doubles:
 *     CHM_MB_FP64_RATE / CHM_MB_FP32_RATE  {T FMA/s for the GPU, per SM}
 *     CHM_MB_FP64_WARP       {cycles per FP64 FMA of one warp issuing
 *                             independent FMAs, cycles per dependent FMA}
 *     CHM_MB_FP64_LANES      {cycles per dependent FP64 FMA of one warp with
 *                             one active lane, the same for each of four
 *                             warps of one block with all lanes active}
 *     CHM_MB_SHFL_SPLIT      {cycles of 32 dependent shuffles in a converged
 *                             warp, the same after a wait run by lane 0 alone}
 *     CHM_MB_HBM_COPY        {GB/s of a 2 GiB device copy (read + write), ms}
 *     CHM_MB_FLAG_ROUND_TRIP {microseconds per release/acquire round trip
 *                             between two thread blocks, 1 if a wait gave up}
 * Returns CHM_OK, CHM_ERR_ARG, CHM_ERR_NOMEM or CHM_ERR_CUDA.
 */
typedef enum {
    CHM_MB_FP64_RATE = 0,
    CHM_MB_FP32_RATE = 1,
    CHM_MB_FP64_WARP = 2,
    CHM_MB_SHFL_SPLIT = 3,
    CHM_MB_HBM_COPY = 4,
    CHM_MB_FLAG_ROUND_TRIP = 5,
    CHM_MB_FP64_LANES = 6
} chm_microbench_kind;
int chm_microbench(int which, double *out, int nout);

/*
 * Library-wide settings of the single-factor entry points (chm_update,
 * chm_downdate, chm_modify_ex), for tuning and tests; they take effect on
 * the next call and may be changed at any time from one thread.
 *   "path"     0 automatic (default), 1 the wave kernel, 2 the pass kernels
 *   "pass_kb"  update vectors per pass of the pass kernels, 1..16 (0: by
 *              type, 8 float, 4 double)
 *   "pass_d"   lookahead of the pass kernels' forward-substitution chain in
 *              row blocks, clamped to 2..10 (float) or 2..6 (double) and
 *              further by what the chain block's shared memory holds for
 *              the pass's vectors; 0 is the default by type and vectors
 *              per pass (float: 4 up to 2 vectors, 6 up to 4, 10 beyond;
 *              double: 3)
 *   "pass_seg" row blocks per segment of the pass kernels' sweep tasks
 *              (0: max(64, row blocks / 16))
 *   "pass_fused" 1 (default): up to 8 vectors per pass, the substitution
 *              kernel's worker warps also form the coefficients and sweep,
 *              each segment as soon as its inputs are out; 0: the sweep
 *              and the Compute kernels run after the substitution
 * The two paths compute the same factor by the same method (Algorithm 1's
 * rotations, restated exactly) with different work splits:
 *   wave  one persistent launch per 64 vectors; each vector is a wave that
 *         sweeps the factor, its forward-substitution chain driven by the
 *         sweep's carries.  Fastest while the factor stays in L2.
 *   pass  per block of up to 16 vectors (Sec. 4.1's blocking): a forward
 *         substitution P = L^{-T} V run by one chain block with lookahead,
 *         every rotation's coefficients from prefix Grams of P (the Compute,
 *         in double), and one sweep that reads and writes each tile of the
 *         factor once for the whole block of vectors.
 * The automatic rule takes the pass kernels when the factor's upper
 * triangle is at least 32 MB (float) or 256 MB with k <= 8 (double), and
 * for a factor of order >= 64 in page-locked host memory modified by two or
 * more vectors (it then crosses the CPU-GPU link three times per pass of up
 * to 16 vectors; the wave kernel twice per vector).
 * chm_config_get also answers "pass_d_f32", "pass_d_f64", "pass_kb_f32"
 * and "pass_kb_f64" (the values in effect, tuning cache aside) and
 * "checked" (1 in the bounds-checked build).  The bounds-checked
 * build also takes "check_cut" (>= 0, default 0): its checks treat each
 * factor as that many columns narrower than declared, so that they report
 * accesses to real, valid memory (a test of the checks themselves; the
 * access is skipped).  Host only.  Returns CHM_OK or CHM_ERR_ARG (unknown
 * key or value out of range).
 */
int chm_config_set(const char *key, int64_t value);
int chm_config_get(const char *key, int64_t *value);

/*
 * The path (1 wave kernel, 2 pass kernels) a single-factor modification of
 * order n by k vectors takes under the current settings and tuning cache.
 * Host only.  Returns CHM_OK or CHM_ERR_ARG.
 */
int chm_path_for(int64_t n, int64_t k, int dtype, int *path);

/*
 * Autotuning of the single-factor entry points.  The paper fixes its
 * kernels' parameters for its GPU (Sec. 4.1: blocks per kernel, threads per
 * block, elements per thread); here they are measured.  chm_tune times, on
 * the current device, a modification of order n by k vectors in dtype
 * under candidate configurations: the wave kernel, and the pass kernels
 * over vectors per pass (min(k, 16) and the two powers of two below it),
 * the substitution's lookahead d ({4, 6, 8, 10} float, {2, 3, 4, 6}
 * double) and the sweep's segment length (the default, 32, 128 row blocks).
 * Each candidate runs an update and downdate by the same V four times on a
 * scratch factor it generates (diagonal 1 + U[0,1), strictly upper entries
 * of variance 1/n; V of variance 1/(4nk)); the median of the last three is
 * its time.  The fastest configuration is stored in the library's tuning
 * cache under (dtype, floor(log2 n), ceil(log2 k)); from then on every
 * single-factor modification of a device factor whose shape falls in that
 * bucket takes it, except for the parameters a library setting ("path",
 * "pass_kb", "pass_d", "pass_seg") forces.  The result is the same factor
 * up to rounding whichever configuration runs.
 *   result  HOST array of 6 (may be NULL): path, vectors per pass,
 *           lookahead, segment length (0: by the order), the tuned time of
 *           one modification in ns, and the time of the built-in default
 *           configuration in ns.
 * Synchronous; allocates n*n + n*k elements and a workspace on its own
 * stream and frees them before returning.  Returns CHM_OK, CHM_ERR_ARG
 * (n < 1, k < 1, n > 2^20, k > 4096, bad dtype), CHM_ERR_NOMEM or
 * CHM_ERR_CUDA (a launch failed, or a candidate's modification reported an
 * error; the cache is then unchanged).
 */
int chm_tune(int64_t n, int64_t k, int dtype, int64_t *result);
/* Empties the tuning cache.  Host only; returns CHM_OK. */
int chm_tune_clear(void);
/*
 * Writes the tuning cache to a text file: the line "chm-tune 1", then one
 * line per entry, "dtype nbucket kbucket path kb d seg ns".  Host only;
 * returns CHM_OK or CHM_ERR_ARG (NULL path, file not writable).
 */
int chm_tune_save(const char *path);
/*
 * Merges a file written by chm_tune_save into the tuning cache (its entries
 * replace those with the same key).  A file that is not in that format, or
 * holds an out-of-range value, changes nothing and returns CHM_ERR_ARG.
 * Host only.
 */
int chm_tune_load(const char *path);

/*
 * Self-test of the reciprocal and reciprocal square root the kernels use in
 * double precision (a hardware approximation refined by one third-order
 * Newton-Raphson step, with IEEE division and square root outside
 * [2^-1020, 2^1020] so that no input or result is flushed to zero).  For
 * each x[i] it evaluates, on the current device,
 *   out[4i] = the library's 1/x,  out[4i+1] = the library's 1/sqrt(x),
 *   out[4i+2] = CUDA's 1.0/x,     out[4i+3] = CUDA's 1.0/sqrt(x)
 * (the last two correctly rounded).  x and out are HOST arrays of count and
 * 4 count doubles.  Allocates and frees its own device buffers,
 * synchronises.  Diagnostics; returns CHM_OK, CHM_ERR_ARG, CHM_ERR_NOMEM or
 * CHM_ERR_CUDA.
 */
int chm_selftest_reciprocals(const double *x, int64_t count, double *out);

/*
 * Diagnostics.  When the environment variable CHM_TRACE is set to 1 before
 * the first call, every launch of the plain entry points records 16 int64
 * stamps of the device's %globaltimer (ns) at fixed points per (wave, column
 * block): first the sweep tasks' records, then the wave blocks'
 * ([2][waves][blocks][16]).  chm_trace_dump synchronises the device and
 * writes the last launch's records (native endianness) to the file `path`.
 * Returns CHM_OK, CHM_ERR_STATE if tracing is off, CHM_ERR_ARG if the file
 * cannot be written, or CHM_ERR_CUDA.  Not for production use.
 *
 * Environment read once per process:
 *   CHM_TIMEOUT_NS         bound on any single wait between thread blocks
 *                          (default 4e9); a wait that runs out ends the
 *                          launch with CHM_ERR_TIMEOUT and the context stays
 *                          usable
 *   CHM_GROUPS             SM groups (concurrent waves) of a launch
 *   CHM_MAX_CTAS_PER_SM    cap on resident blocks per SM
 *   CHM_TEST_SKIP_PUBLISH  test hook: the next launch of the plain entry
 *                          points leaves the given block's rotation panel
 *                          unreleased, so the waits on it run out
 */
int chm_trace_dump(const char *path);

#ifdef __cplusplus
}
#endif

#endif /* CHM_H */
