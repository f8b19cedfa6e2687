// Solve with a factor: B <- (L^T L)^{-1} B, the use a maintained Cholesky
// factor serves (Sec. 1).  A forward substitution with L^T (lower) followed
// by a back substitution with L (upper), both blocked by kW = 32 rows, in
// one persistent launch per group of up to four right-hand sides.
//
// Tasks, taken in order from a launch-wide counter by blocks of four warps:
//   t <  nb: forward task for block b = t:  y_b = D_b^{-T} (b_b - sum_{p<b} L_{p,b}^T y_p)
//   t >= nb: backward task for b = 2nb-1-t: x_b = D_b^{-1} (y_b - sum_{q>b} L_{b,q} x_q)
// where D_b is the diagonal block and L_{p,b} the 32 x 32 tile in row block
// p and column block b.  A task waits only on tasks taken before it, so the
// launch cannot deadlock whatever the number of resident blocks.
//
// Each forward task inverts its diagonal block (U_b = D_b^{-1}, one column
// per lane) and forms G_b = U_b^T L_{b-1,b}^T while its warps accumulate the
// tiles whose y is already published, and z_b = U_b^T (b_b - sum over
// p <= b-2) once y_{b-2} is in; then y_b = z_b - G_b y_{b-1}.  The backward
// task reuses U_b and forms H_b = U_b L_{b,b+1}: x_b = z'_b - H_b x_{b+1}.
// Between one block's result and the next block's there is one 32 x 32
// product (eight FMAs per warp), one barrier and a four-way sum.  Results
// pass between blocks as epoch-tagged doubles (no fence, no flag).
#include <float.h>

#include <algorithm>

#include "chm.h"
#include "chm_device.cuh"
#include "chm_internal.h"
#include "chm_layout.h"

namespace chm {
namespace {

constexpr int kSolveThreads = 128;
constexpr int kSolveWarps = kSolveThreads / 32;
constexpr int kSolveRhs = 4;                       // right-hand sides per launch (largest)
constexpr int kRowsPerWarp = kW / kSolveWarps;     // rows (or columns) of a split tile per warp
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
struct SolveArgs {
    const T *L;
    long long n, ld;
    T *B;
    long long ldb;
    int nb;           // blocks of kW rows
    int nr;           // right-hand sides of this launch (1 .. R)
    // back substitution only: y = L^{-T} b is given, row i of right-hand
    // side r at Y[i * ys + r * cs] (chm_modify_solve's pass forms it)
    const T *Y;
    long long ys, cs;
    int back_only;
    double *inv;      // [nb][kW][kW]: U_b = D_b^{-1}, row i at i * kW
    int *yflag;       // [nb]: y_b and U_b published (== epoch)
    long long *ytag;  // [nb][kW][R][2]: y_b as tagged doubles
    long long *xtag;  // [nb][kW][R][2]: x_b as tagged doubles
    int *ctl;
    long long *status;
    long long timeout_ns;
    // the workspace allocations inv, yflag and ytag / xtag are carved from (bounds-checked builds)
    const char *ws_data;
    size_t ws_data_bytes;
    const int *ws_iflags;
    size_t ws_iflags_n;
    const long long *ws_progress;
    size_t ws_progress_n;
    long long chk_cut;
};

template <int R>
struct SolveSmem {
    double D[kW][kW + 1];  // diagonal block (row, column); identity beyond the order
    double U[kW][kW + 1];  // its inverse
    double T[kW][kW + 1];  // the tile next to the diagonal block (see the tasks)
    double part[2][kSolveWarps][R][kW];
    double rd[kW];         // 1 / D_ii
};

template <int R>
__device__ __forceinline__ size_t tag_at(int blk, int i, int r)
{
    return (((size_t)blk * kW + i) * R + r) * 2;
}

// The whole warp waits for the R tagged values of block `blk` (lane i gets
// row i).  `next_step` marks the wait on the previous block's result, the
// one step of the chain: it polls at short fixed intervals (only the next
// block's four warps wait on a fresh result, and each step gains the time a
// longer sleep would add); every other wait backs off up to 256 ns, since
// hundreds of warps may be waiting on older results at once.  A wait that
// gives up (recorded as a timeout, or the launch is aborted) yields zeros,
// so that every warp still reaches the block's barriers; the result is then
// unspecified and the status says so.
template <int R>
__device__ __forceinline__ void wait_block(const SyncArgs &sy, const long long *tags, long long ep64, int blk,
                                           long long who, double *v, bool next_step = false)
{
    const int lane = threadIdx.x & 31;
    const long long *w = tags + tag_at<R>(blk, lane, 0);
    const long long t0 = global_ns();
    unsigned ns = next_step ? 32 : 16;
    for (unsigned it = 0;; ++it) {
        bool ok = true;
#pragma unroll
        for (int r = 0; r < R; ++r) ok = get_tagged(w + 2 * r, ep64, &v[r]) && ok;
        if (__all_sync(kFull, ok)) return;
        if ((it & 15u) == 15u) {
            int stop = 0;
            if (lane == 0) {
                if (aborted(sy)) {
                    stop = 1;
                } else if (global_ns() - t0 > sy.timeout_ns || it > (1u << 28)) {
                    record_error(sy, kStatusTimeout, who);
                    stop = 1;
                }
            }
            if (__shfl_sync(kFull, stop, 0)) {
#pragma unroll
                for (int r = 0; r < R; ++r) v[r] = 0.0;
                return;
            }
        }
        __nanosleep(ns);
        if (!next_step && ns < 256) ns <<= 1;
    }
}

// Sum of the four warps' partial products of row `lane`, for each r.
template <int R>
__device__ __forceinline__ double part_sum(const SolveSmem<R> &S, int buf, int r, int lane)
{
    return (S.part[buf][0][r][lane] + S.part[buf][1][r][lane]) + (S.part[buf][2][r][lane] + S.part[buf][3][r][lane]);
}

template <typename T, int R>
__device__ void forward_task(const SolveArgs<T> &a, const SyncArgs &sy, long long ep64, int b, SolveSmem<R> &S)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long ld = a.ld;
    const long long c0 = (long long)b * kW;
    const int nc = (int)min((long long)kW, a.n - c0);
    const bool active = lane < nc;
    const long long who = b;

    // the diagonal block (identity beyond the order) and the tile above it,
    // S.T[j][m] = L[(b-1) kW + j, c0 + m]
    for (int e = threadIdx.x; e < kW * kW; e += kSolveThreads) {
        const int i = e & (kW - 1), j = e / kW;
        double v = 0.0;
        if (j < nc) {
            if (i <= j && CHK_TRI(sy, c0 + i + (c0 + j) * ld, a.n, ld)) v = (double)__ldg(a.L + c0 + i + (c0 + j) * ld);
        } else if (i == j) {
            v = 1.0;
        }
        S.D[i][j] = v;
        if (b >= 1)
            S.T[i][j] = (j < nc && CHK_TRI(sy, c0 - kW + i + (c0 + j) * ld, a.n, ld))
                            ? (double)__ldg(a.L + c0 - kW + i + (c0 + j) * ld) : 0.0;
    }
    double rhs[R];
    if (a.back_only) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            rhs[r] = (active && r < a.nr) ? (double)__ldcg(a.Y + (c0 + lane) * a.ys + r * a.cs) : 0.0;
    } else {
#pragma unroll
        for (int r = 0; r < R; ++r)
            rhs[r] = (active && r < a.nr && CHK_RECT(sy, c0 + lane + r * a.ldb, a.n, a.nr, a.ldb))
                         ? (double)a.B[c0 + lane + r * a.ldb] : 0.0;
    }
    __syncthreads();

    if (warp == 0) {
        double d = S.D[lane][lane];
        if (!(d > 0.0 && d <= DBL_MAX)) {  // not a Cholesky factor
            record_error(sy, kStatusNotPD, c0 + lane);
            d = 1.0;
        }
        S.rd[lane] = 1.0 / d;
        __syncwarp();
        // column `lane` of U = D^{-1}: back substitution on D u = e_lane
        double u[kW];
#pragma unroll
        for (int i = kW - 1; i >= 0; --i) {
            double s = (i == lane) ? 1.0 : 0.0;
#pragma unroll
            for (int m = i + 1; m < kW; ++m) s = fma(-S.D[i][m], u[m], s);
            u[i] = s * S.rd[i];
        }
        double *inv = a.inv + (size_t)b * kW * kW;
#pragma unroll
        for (int i = 0; i < kW; ++i) {
            S.U[i][lane] = u[i];
            __stcg(inv + i * kW + lane, u[i]);
        }
    }

    __syncthreads();  // U in shared memory

    if (a.back_only) {
        // y_b is given: publish it with U_b for this block's backward task
        if (warp == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) put_tagged(a.ytag + tag_at<R>(b, lane, r), rhs[r], ep64);
            __syncwarp();
            if (lane == 0) st_release_gpu(a.yflag + b, sy.epoch);
        }
        return;
    }

    // G = U^T S.T^T, the rows j of S.T split over the warps:
    // g[jj] = G[lane][warp * 8 + jj] = sum_m U[m][lane] S.T[warp * 8 + jj][m]
    double g[kRowsPerWarp];
#pragma unroll
    for (int jj = 0; jj < kRowsPerWarp; ++jj) g[jj] = 0.0;
    if (b >= 1) {
#pragma unroll
        for (int m = 0; m < kW; ++m) {
            const double um = S.U[m][lane];
#pragma unroll
            for (int jj = 0; jj < kRowsPerWarp; ++jj) g[jj] = fma(um, S.T[warp * kRowsPerWarp + jj][m], g[jj]);
        }
    }
    // tiles p <= b - 3 of column block b, dealt round-robin to the warps (a
    // fixed order of the sums: results do not depend on timing); lane =
    // column of the block, the tile's 32 rows read down the column
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    const long long colo = (c0 + (active ? lane : 0)) * ld;
    const T *col = a.L + colo;
    for (int p = warp; p <= b - 3; p += kSolveWarps) {
        const T *src = col + (long long)p * kW;
        double t[kW];
#pragma unroll
        for (int j = 0; j < kW; ++j)
            t[j] = (active && CHK_TRI(sy, colo + (long long)p * kW + j, a.n, ld)) ? (double)__ldg(src + j) : 0.0;
        double yv[R];
        wait_block<R>(sy, a.ytag, ep64, p, who, yv);
#pragma unroll
        for (int j = 0; j < kW; ++j)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(t[j], __shfl_sync(kFull, yv[r], j), acc[r]);
    }
    // tile b - 2: its rows split over the warps
    if (b >= 2) {
        const T *src = col + (long long)(b - 2) * kW + warp * kRowsPerWarp;
        double t[kRowsPerWarp];
#pragma unroll
        for (int jj = 0; jj < kRowsPerWarp; ++jj) t[jj] = active ? (double)__ldg(src + jj) : 0.0;
        double yv[R];
        wait_block<R>(sy, a.ytag, ep64, b - 2, who, yv);
#pragma unroll
        for (int jj = 0; jj < kRowsPerWarp; ++jj)
#pragma unroll
            for (int r = 0; r < R; ++r)
                acc[r] = fma(t[jj], __shfl_sync(kFull, yv[r], warp * kRowsPerWarp + jj), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[0][warp][r][lane] = acc[r];
    __syncthreads();
    double rv[R];  // b_b - sum_{p <= b-2} L_{p,b}^T y_p, row `lane`
#pragma unroll
    for (int r = 0; r < R; ++r) rv[r] = rhs[r] - part_sum(S, 0, r, lane);
    // z_b = U^T r: z_i = sum_{j <= i} U_ji r_j, the j split over the warps
    double pz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) pz[r] = 0.0;
#pragma unroll
    for (int jj = 0; jj < kRowsPerWarp; ++jj) {
        const int j = warp * kRowsPerWarp + jj;
        const double uji = S.U[j][lane];
#pragma unroll
        for (int r = 0; r < R; ++r) pz[r] = fma(uji, __shfl_sync(kFull, rv[r], j), pz[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[1][warp][r][lane] = pz[r];
    __syncthreads();
    double z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) z[r] = part_sum(S, 1, r, lane);
    __syncthreads();  // part[0] free again
    // y_b = z_b - G_b y_{b-1}: the step that waits on the previous block
    double py[R];
#pragma unroll
    for (int r = 0; r < R; ++r) py[r] = 0.0;
    if (b >= 1) {
        double yv[R];
        wait_block<R>(sy, a.ytag, ep64, b - 1, who, yv, true);
#pragma unroll
        for (int jj = 0; jj < kRowsPerWarp; ++jj)
#pragma unroll
            for (int r = 0; r < R; ++r)
                py[r] = fma(g[jj], __shfl_sync(kFull, yv[r], warp * kRowsPerWarp + jj), py[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[0][warp][r][lane] = py[r];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) put_tagged(a.ytag + tag_at<R>(b, lane, r), z[r] - part_sum(S, 0, r, lane), ep64);
        __syncwarp();
        // U_b and y_b for this block's backward task
        if (lane == 0) st_release_gpu(a.yflag + b, sy.epoch);
    }
}

template <typename T, int R>
__device__ void backward_task(const SolveArgs<T> &a, const SyncArgs &sy, long long ep64, int b,
                              SolveSmem<R> &S)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n = a.n, ld = a.ld;
    const long long c0 = (long long)b * kW;
    const int nc = (int)min((long long)kW, n - c0);
    const bool active = lane < nc;
    const long long who = b;
    const bool has_next = b + 1 < a.nb;

    (void)__all_sync(kFull, wait_eq(sy, a.yflag + b, sy.epoch, who));
    __syncwarp();
    // U_b, and the tile to its right, S.T[m][j] = L[c0 + m, (b+1) kW + j]
    const double *inv = a.inv + (size_t)b * kW * kW;
    const long long q1 = (long long)(b + 1) * kW;
    const int nc1 = has_next ? (int)min((long long)kW, n - q1) : 0;
    for (int e = threadIdx.x; e < kW * kW; e += kSolveThreads) {
        const int i = e / kW, j = e & (kW - 1);
        S.U[i][j] = __ldcg(inv + e);
        S.T[j][i] = (has_next && j < nc && i < nc1 && CHK_TRI(sy, c0 + j + (q1 + i) * ld, n, ld))
                        ? (double)__ldg(a.L + c0 + j + (q1 + i) * ld) : 0.0;
    }
    double yv[R];
    wait_block<R>(sy, a.ytag, ep64, b, who, yv);
    __syncthreads();

    // H = U S.T, the columns j of S.T split over the warps:
    // h[jj] = H[lane][warp * 8 + jj] = sum_m U[lane][m] S.T[m][warp * 8 + jj]
    double h[kRowsPerWarp];
#pragma unroll
    for (int jj = 0; jj < kRowsPerWarp; ++jj) h[jj] = 0.0;
    if (has_next) {
#pragma unroll
        for (int m = 0; m < kW; ++m) {
            const double um = S.U[lane][m];
#pragma unroll
            for (int jj = 0; jj < kRowsPerWarp; ++jj) h[jj] = fma(um, S.T[m][warp * kRowsPerWarp + jj], h[jj]);
        }
    }

    // tiles q >= b + 3 of row block b, from the last one up, dealt
    // round-robin to the warps; lane = row of the block, so each column of a
    // tile is one coalesced read
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    const long long rowo = c0 + (active ? lane : 0);
    const T *row = a.L + rowo;
    for (int q = a.nb - 1 - warp; q >= b + 3; q -= kSolveWarps) {
        const long long q0 = (long long)q * kW;
        const int ncq = (int)min((long long)kW, n - q0);
        double t[kW];
#pragma unroll
        for (int c = 0; c < kW; ++c)
            t[c] = (active && c < ncq && CHK_TRI(sy, rowo + (q0 + c) * ld, n, ld)) ? (double)__ldg(row + (q0 + c) * ld) : 0.0;
        double xv[R];
        wait_block<R>(sy, a.xtag, ep64, q, who, xv);
#pragma unroll
        for (int c = 0; c < kW; ++c)
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = fma(t[c], __shfl_sync(kFull, xv[r], c), acc[r]);
    }
    // tile b + 2: its columns split over the warps
    if (b + 2 < a.nb) {
        const long long q0 = (long long)(b + 2) * kW;
        const int ncq = (int)min((long long)kW, n - q0);
        double t[kRowsPerWarp];
#pragma unroll
        for (int cc = 0; cc < kRowsPerWarp; ++cc) {
            const int c = warp * kRowsPerWarp + cc;
            t[cc] = (active && c < ncq && CHK_TRI(sy, rowo + (q0 + c) * ld, n, ld)) ? (double)__ldg(row + (q0 + c) * ld) : 0.0;
        }
        double xv[R];
        wait_block<R>(sy, a.xtag, ep64, b + 2, who, xv);
#pragma unroll
        for (int cc = 0; cc < kRowsPerWarp; ++cc)
#pragma unroll
            for (int r = 0; r < R; ++r)
                acc[r] = fma(t[cc], __shfl_sync(kFull, xv[r], warp * kRowsPerWarp + cc), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[0][warp][r][lane] = acc[r];
    __syncthreads();
    double rv[R];  // y_b - sum_{q >= b+2} L_{b,q} x_q, row `lane`
#pragma unroll
    for (int r = 0; r < R; ++r) rv[r] = yv[r] - part_sum(S, 0, r, lane);
    // z'_b = U r: z_i = sum_{j >= i} U_ij r_j, the j split over the warps
    double pz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) pz[r] = 0.0;
#pragma unroll
    for (int jj = 0; jj < kRowsPerWarp; ++jj) {
        const int j = warp * kRowsPerWarp + jj;
        const double uij = S.U[lane][j];
#pragma unroll
        for (int r = 0; r < R; ++r) pz[r] = fma(uij, __shfl_sync(kFull, rv[r], j), pz[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[1][warp][r][lane] = pz[r];
    __syncthreads();
    double z[R];
#pragma unroll
    for (int r = 0; r < R; ++r) z[r] = part_sum(S, 1, r, lane);
    __syncthreads();  // part[0] free again
    // x_b = z'_b - H_b x_{b+1}: the step that waits on the previous block
    double px[R];
#pragma unroll
    for (int r = 0; r < R; ++r) px[r] = 0.0;
    if (has_next) {
        double xv[R];
        wait_block<R>(sy, a.xtag, ep64, b + 1, who, xv, true);
#pragma unroll
        for (int jj = 0; jj < kRowsPerWarp; ++jj)
#pragma unroll
            for (int r = 0; r < R; ++r)
                px[r] = fma(h[jj], __shfl_sync(kFull, xv[r], warp * kRowsPerWarp + jj), px[r]);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) S.part[0][warp][r][lane] = px[r];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double x = z[r] - part_sum(S, 0, r, lane);
            put_tagged(a.xtag + tag_at<R>(b, lane, r), x, ep64);
            if (active && r < a.nr && CHK_RECT(sy, c0 + lane + r * a.ldb, a.n, a.nr, a.ldb)) a.B[c0 + lane + r * a.ldb] = (T)x;
        }
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(kSolveThreads) solve_kernel(SolveArgs<T> a)
{
    __shared__ SolveSmem<R> S;
    __shared__ int s_task, s_last;
    SyncArgs sy;
    sy.abort_flag = a.ctl + kCtlAbort;
    sy.status = a.status;
    sy.user_info = nullptr;
    sy.epoch = ld_relaxed_gpu(a.ctl + kCtlEpoch);
    sy.timeout_ns = a.timeout_ns;
    sy.chk_cut = a.chk_cut;
    const long long ep64 = (long long)sy.epoch << 32;
    // bounds-checked builds: the workspace regions inside their allocations
    const bool ws_in = CHK_REGION(sy, a.inv, (size_t)a.nb * kW * kW * sizeof(double), a.ws_data, a.ws_data_bytes) &&
                       CHK_REGION(sy, a.yflag, (size_t)a.nb * sizeof(int), a.ws_iflags, a.ws_iflags_n * sizeof(int)) &&
                       CHK_REGION(sy, a.ytag, (size_t)a.nb * kW * R * 2 * sizeof(long long), a.ws_progress,
                                  a.ws_progress_n * sizeof(long long)) &&
                       CHK_REGION(sy, a.xtag, (size_t)a.nb * kW * R * 2 * sizeof(long long), a.ws_progress,
                                  a.ws_progress_n * sizeof(long long));

    for (;;) {
        if (threadIdx.x == 0) s_task = (!ws_in || aborted(sy)) ? -1 : atomicAdd(a.ctl + kCtlPairNext, 1);
        __syncthreads();
        const int t = s_task;
        if (t < 0 || t >= 2 * a.nb) break;
        if (t < a.nb) forward_task<T, R>(a, sy, ep64, t, S);
        else backward_task<T, R>(a, sy, ep64, 2 * a.nb - 1 - t, S);
        __syncthreads();
    }

    // The last block to finish zeroes the control words for the next launch
    // and advances the epoch.
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(a.ctl + kCtlExited, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = threadIdx.x; i < kCtlInts; i += blockDim.x)
            if (i != kCtlEpoch) a.ctl[i] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            a.ctl[kCtlEpoch] = a.ctl[kCtlEpoch] + 1;
            __threadfence();
        }
    }
}

template <typename T, int R>
int launch_solve(const void *L, long long n, long long ld, void *B, long long ldb, int nr, const Scratch &sc,
                 cudaStream_t stream, const T *Y = nullptr, long long ys = 0, long long cs = 0)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CHM_ERR_CUDA;
    static int occ[64] = {0};
    if (!occ[dev]) {
        int b = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, solve_kernel<T, R>, kSolveThreads, 0) !=
                cudaSuccess ||
            b < 1)
            return CHM_ERR_CUDA;
        occ[dev] = b;
    }
    const int nb = (int)((n + kW - 1) / kW);
    SolveArgs<T> a;
    a.L = static_cast<const T *>(L);
    a.n = n;
    a.ld = ld;
    a.B = static_cast<T *>(B);
    a.ldb = ldb;
    a.nb = nb;
    a.nr = nr;
    a.Y = Y;
    a.ys = ys;
    a.cs = cs;
    a.back_only = Y != nullptr;
    a.inv = reinterpret_cast<double *>(sc.data);
    a.yflag = sc.iflags;
    a.ytag = sc.progress;
    a.xtag = sc.progress + (size_t)nb * kW * R * 2;
    a.ctl = sc.ctl;
    a.status = sc.status;
    a.timeout_ns = timeout_ns();
    a.ws_data = sc.data;
    a.ws_data_bytes = sc.data_bytes;
    a.ws_iflags = sc.iflags;
    a.ws_iflags_n = sc.iflags_cap;
    a.ws_progress = sc.progress;
    a.ws_progress_n = sc.progress_cap;
    a.chk_cut = check_cut();
    const int grid = (int)std::min<long long>(2ll * nb, (long long)sm_count(dev) * occ[dev]);
    solve_kernel<T, R><<<grid, kSolveThreads, 0, stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? CHM_OK : CHM_ERR_CUDA;
}

template <typename T>
int solve_all(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs, const Scratch &sc,
              cudaStream_t stream)
{
    T *b = static_cast<T *>(B);
    for (long long r0 = 0; r0 < nrhs; r0 += kSolveRhs) {
        const int nr = (int)std::min<long long>(kSolveRhs, nrhs - r0);
        const int rc = nr == 1 ? launch_solve<T, 1>(L, n, ld, b + r0 * ldb, ldb, 1, sc, stream)
                               : launch_solve<T, kSolveRhs>(L, n, ld, b + r0 * ldb, ldb, nr, sc, stream);
        if (rc != CHM_OK) return rc;
    }
    return CHM_OK;
}

}  // namespace

ScratchNeed solve_need(long long n)
{
    const size_t nb = (size_t)((n + kW - 1) / kW);
    ScratchNeed need;
    need.iflags = (nb + 63) & ~(size_t)63;
    need.progress = 2 * nb * kW * kSolveRhs * 2;
    need.data = nb * kW * kW * sizeof(double);
    return need;
}

namespace {
template <typename T>
int solve_back_t(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs, const T *Y,
                 long long ys, long long cs, const Scratch &sc, cudaStream_t stream)
{
    T *b = static_cast<T *>(B);
    for (long long r0 = 0; r0 < nrhs; r0 += kSolveRhs) {
        const int nr = (int)std::min<long long>(kSolveRhs, nrhs - r0);
        const T *y = Y + r0 * cs;
        const int rc = nr == 1 ? launch_solve<T, 1>(L, n, ld, b + r0 * ldb, ldb, 1, sc, stream, y, ys, cs)
                               : launch_solve<T, kSolveRhs>(L, n, ld, b + r0 * ldb, ldb, nr, sc, stream, y, ys, cs);
        if (rc != CHM_OK) return rc;
    }
    return CHM_OK;
}
}  // namespace

int solve_enqueue(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs, int dtype,
                  const Scratch &sc, cudaStream_t stream)
{
    if (n <= 0 || nrhs <= 0) return CHM_OK;
    return dtype == CHM_F64 ? solve_all<double>(L, n, ld, B, ldb, nrhs, sc, stream)
                            : solve_all<float>(L, n, ld, B, ldb, nrhs, sc, stream);
}

int solve_back_enqueue(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs,
                       const void *Y, long long ys, long long cs, int dtype, const Scratch &sc, cudaStream_t stream)
{
    if (n <= 0 || nrhs <= 0) return CHM_OK;
    return dtype == CHM_F64
               ? solve_back_t<double>(L, n, ld, B, ldb, nrhs, static_cast<const double *>(Y), ys, cs, sc, stream)
               : solve_back_t<float>(L, n, ld, B, ldb, nrhs, static_cast<const float *>(Y), ys, cs, sc, stream);
}

namespace {

int solve_dispatch(const void *L, long long n, long long ld, void *B, long long ldb, long long nrhs, int dtype,
                   cudaStream_t stream)
{
    if (n < 0 || nrhs < 0 || n > (1ll << 26)) return CHM_ERR_ARG;
    if (dtype != CHM_F64 && dtype != CHM_F32_MIXED) return CHM_ERR_ARG;
    if (ld < std::max(1ll, n) || ldb < std::max(1ll, n)) return CHM_ERR_ARG;
    const size_t elt = dtype == CHM_F64 ? 8 : 4;
    if (n > 0 && (!L || (uintptr_t)L % elt)) return CHM_ERR_ARG;
    if (n > 0 && nrhs > 0 && (!B || (uintptr_t)B % elt)) return CHM_ERR_ARG;
    if (n == 0 || nrhs == 0) return CHM_OK;
    int rc = check_reachable(L);
    if (rc == CHM_OK) rc = check_reachable(B);
    if (rc != CHM_OK) return rc;
    return with_stream_scratch(stream, solve_need(n), [&](const Scratch &sc) {
        return dtype == CHM_F64 ? solve_all<double>(L, n, ld, B, ldb, nrhs, sc, stream)
                                : solve_all<float>(L, n, ld, B, ldb, nrhs, sc, stream);
    });
}

}  // namespace
}  // namespace chm

extern "C" int chm_solve(const void *L, int64_t n, int64_t ld, void *B, int64_t ldb, int64_t nrhs, int dtype,
                         chm_stream_t stream)
{
    return chm::solve_dispatch(L, n, ld, B, ldb, nrhs, dtype, (cudaStream_t)stream);
}
