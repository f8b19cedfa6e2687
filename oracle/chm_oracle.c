/*
 * Serial CPU oracle for the rank-k Cholesky up/downdate by hyperbolic
 * rotations (Walder 2010, "Rank k Cholesky Up/Down-dating on the GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header or constant with the
 * CUDA library.
 *
 * What it computes (Sec. 1): given an upper-triangular L with A = L^T L and
 * V (n x k), the factor Lt with Lt^T Lt = A + sigma V V^T, by the paper's
 * serial hyperbolic algorithm (Algorithm 1), in plain IEEE double with no
 * contraction (build with -ffp-contract=off), one core, no blocking.
 *
 * Storage (the paper does not fix it; Matlab's chol convention): L is
 * column-major upper triangular with leading dimension ld, element (i,j) at
 * L[i + j*ld]; only i <= j is read or written.  V is column-major n x k with
 * leading dimension ldv and is never written (a private copy is rotated).
 * sigma[p] in {+1,-1} is the sign of column p (+1 update, -1 downdate).
 *
 * Rank k (Sec. 4.1): the k columns of V are processed in ascending order; for
 * a fixed row i every column's rotation is computed and applied before row
 * i+1.  Every ordering that respects the data dependencies performs the same
 * floating-point operations on the same operands, so this equals k successive
 * rank-1 modifications bit for bit (a property the tests check).
 *
 * Failure (the paper is silent): if L_ii <= 0 (or non-finite) on entry to a
 * Compute step, or L_ii^2 + sigma V_i^2 <= 0 (or non-finite), the routine
 * stops, stores the 0-based row i in *info and returns ORC_ERR_NOT_PD.
 * L is then partially modified.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NOT_PD (-2)
#define ORC_ERR_NOMEM (-5)

static int finite_pos(double x) { return x > 0.0 && x <= DBL_MAX; }

/*
 * Algorithm 1, helper "Compute": w = sqrt(L_ii^2 + sigma V_i^2),
 * c = w / L_ii, s = V_i / L_ii, L_ii <- w.  Returns 0 if the step is not
 * defined (the modified matrix is not positive definite).
 */
static int compute_step(double *c, double *s, double *Lii, double Vi, int sigma)
{
    double l = *Lii;
    if (!finite_pos(l)) return 0;
    double t = l * l + (double)sigma * Vi * Vi;
    if (!finite_pos(t)) return 0;
    double w = sqrt(t);
    *c = w / l;
    *s = Vi / l;
    *Lii = w;
    return 1;
}

/*
 * Algorithm 1, helper "Apply": L_ij <- (L_ij + sigma s V_j) / c, then
 * V_j <- c V_j - s L_ij with the NEW L_ij (the two statements run in order).
 */
static void apply_step(double c, double s, double *Lij, double *Vj, int sigma)
{
    double l = (*Lij + (double)sigma * s * *Vj) / c;
    *Lij = l;
    *Vj = c * *Vj - s * l;
}

static int check_args(int64_t n, int64_t ld, int64_t ldv, int64_t k, const void *L,
                      const void *V, const int8_t *sigma)
{
    if (n < 0 || k < 0) return 0;
    if (ld < (n > 1 ? n : 1) || ldv < (n > 1 ? n : 1)) return 0;
    if (n > 0 && !L) return 0;
    if (n > 0 && k > 0 && (!V || !sigma)) return 0;
    for (int64_t p = 0; p < k; ++p)
        if (sigma[p] != 1 && sigma[p] != -1) return 0;
    return 1;
}

/*
 * CholeskyModifyB (Algorithm 1, second alternative), rank k:
 *   for i = 1..n: for each column p of V: Compute(c, s, L_ii, V_i^p);
 *                 for j = i+1..n: Apply(c, s, L_ij, V_j^p).
 * Only rows 0..m_rows-1 are processed (m_rows = n for the full factor).  The
 * final values of rows < m depend only on rows < m of L and on V, so a
 * truncated run gives those rows exactly.
 */
int orc_modify_b(double *L, int64_t n, int64_t ld, const double *V, int64_t ldv, int64_t k,
                 const int8_t *sigma, int64_t m_rows, int64_t *info)
{
    if (info) *info = -1;
    if (!check_args(n, ld, ldv, k, L, V, sigma)) return ORC_ERR_ARG;
    if (m_rows < 0 || m_rows > n) m_rows = n;
    if (n == 0 || k == 0) return ORC_OK;
    double *W = (double *)malloc((size_t)n * (size_t)k * sizeof(double));
    if (!W) return ORC_ERR_NOMEM;
    for (int64_t p = 0; p < k; ++p)
        memcpy(W + p * n, V + p * ldv, (size_t)n * sizeof(double));
    for (int64_t i = 0; i < m_rows; ++i) {
        for (int64_t p = 0; p < k; ++p) {
            double *v = W + p * n;
            double c, s;
            if (!compute_step(&c, &s, &L[i + i * ld], v[i], sigma[p])) {
                if (info) *info = i;
                free(W);
                return ORC_ERR_NOT_PD;
            }
            for (int64_t j = i + 1; j < n; ++j)
                apply_step(c, s, &L[i + j * ld], &v[j], sigma[p]);
        }
    }
    free(W);
    return ORC_OK;
}

/*
 * CholeskyModifyA (Algorithm 1, first alternative), rank k, column order:
 *   for i = 1..n: for j = 1..i-1: for each p: Apply(c_j^p, s_j^p, L_ji, V_i^p);
 *                 then for each p: Compute(c_i^p, s_i^p, L_ii, V_i^p).
 * As printed, the paper places Compute before the inner loop; that would form
 * (c_i, s_i) from a V_i that rows 1..i-1 have not yet rotated, which does not
 * give a Cholesky factor of A + sigma V V^T.  This routine takes the reading
 * in which Compute follows the inner loop, matching CholeskyModifyB.
 */
int orc_modify_a(double *L, int64_t n, int64_t ld, const double *V, int64_t ldv, int64_t k,
                 const int8_t *sigma, int64_t *info)
{
    if (info) *info = -1;
    if (!check_args(n, ld, ldv, k, L, V, sigma)) return ORC_ERR_ARG;
    if (n == 0 || k == 0) return ORC_OK;
    double *cs = (double *)malloc((size_t)n * (size_t)k * 2 * sizeof(double));
    double *vi = (double *)malloc((size_t)k * sizeof(double));
    if (!cs || !vi) { free(cs); free(vi); return ORC_ERR_NOMEM; }
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = 0; p < k; ++p) vi[p] = V[i + p * ldv];
        for (int64_t j = 0; j < i; ++j)
            for (int64_t p = 0; p < k; ++p)
                apply_step(cs[2 * (j * k + p)], cs[2 * (j * k + p) + 1], &L[j + i * ld], &vi[p],
                           sigma[p]);
        for (int64_t p = 0; p < k; ++p) {
            if (!compute_step(&cs[2 * (i * k + p)], &cs[2 * (i * k + p) + 1], &L[i + i * ld],
                              vi[p], sigma[p])) {
                if (info) *info = i;
                free(cs); free(vi);
                return ORC_ERR_NOT_PD;
            }
        }
    }
    free(cs); free(vi);
    return ORC_OK;
}

/*
 * Mixed precision (FP32 storage and Apply, FP64 Compute): L and V are float.
 * The k columns of V are taken in groups of `kgroup` consecutive columns
 * (kgroup <= 0: one group), the vectors one launch or one pass of the GPU
 * path handles.  Each group is CholeskyModifyB restricted to its columns:
 * for each row i, for each column p of the group in order,
 *   Compute in double: L_ii is promoted from float when the group reaches
 *     row i and carried in double across the group's columns; V_i^p is the
 *     promoted float carry; w = sqrt(L_ii^2 + sigma V_i^2), c = w / L_ii,
 *     s = V_i / L_ii, L_ii <- w; then c and s are rounded to float;
 *   Apply in float arithmetic, one rounding per operation, in the order
 *     printed (L_ij <- (L_ij + sigma s V_j) / c, then V_j <- c V_j - s L_ij
 *     with the new L_ij);
 * and the new L_ii is rounded to float once the group has passed row i.
 * Failure: a group that fails at row i records i; later groups then process
 * only the rows above it (whose values are still defined), so the row
 * returned is the smallest failing row, that of CholeskyModifyB on all k
 * columns.  Rows at and below it are left partially modified.
 */
int orc_modify_mixed32(float *L, int64_t n, int64_t ld, const float *V, int64_t ldv, int64_t k,
                       const int8_t *sigma, int64_t m_rows, int64_t kgroup, int64_t *info)
{
    if (info) *info = -1;
    if (!check_args(n, ld, ldv, k, L, V, sigma)) return ORC_ERR_ARG;
    if (m_rows < 0 || m_rows > n) m_rows = n;
    if (n == 0 || k == 0) return ORC_OK;
    if (kgroup <= 0 || kgroup > k) kgroup = k;
    float *W = (float *)malloc((size_t)n * (size_t)k * sizeof(float));
    if (!W) return ORC_ERR_NOMEM;
    for (int64_t p = 0; p < k; ++p)
        memcpy(W + p * n, V + p * ldv, (size_t)n * sizeof(float));
    int64_t fail = -1;
    for (int64_t g0 = 0; g0 < k; g0 += kgroup) {
        const int64_t g1 = g0 + kgroup < k ? g0 + kgroup : k;
        for (int64_t i = 0; i < m_rows; ++i) {
            double lii = (double)L[i + i * ld];
            int ok = 1;
            for (int64_t p = g0; p < g1 && ok; ++p) {
                float *v = W + p * n;
                double c, s;
                if (!compute_step(&c, &s, &lii, (double)v[i], sigma[p])) {
                    ok = 0;
                    break;
                }
                float cf = (float)c, sf = (float)s, sg = (float)sigma[p];
                for (int64_t j = i + 1; j < n; ++j) {
                    float prod = sg * sf;
                    prod = prod * v[j];
                    float num = L[i + j * ld] + prod;
                    float l = num / cf;
                    L[i + j * ld] = l;
                    float a = cf * v[j];
                    float b = sf * l;
                    v[j] = a - b;
                }
            }
            if (!ok) {
                fail = (fail < 0 || i < fail) ? i : fail;
                m_rows = i;  /* later groups: the rows above the failure only */
                break;
            }
            L[i + i * ld] = (float)lii;
        }
    }
    free(W);
    if (fail >= 0) {
        if (info) *info = fail;
        return ORC_ERR_NOT_PD;
    }
    return ORC_OK;
}

/*
 * Solve with the factor.  The factor is maintained so that systems with
 * A = L^T L can be solved cheaply (Sec. 1); this overwrites the n x nrhs
 * column-major B (leading dimension ldb) with X = A^{-1} B by the two
 * textbook triangular solves, in plain double, one column of B at a time:
 *   forward substitution with L^T (lower):  y_i = (b_i - sum_{j<i} L_ji y_j) / L_ii,
 *   back substitution with L (upper):       x_i = (y_i - sum_{j>i} L_ij x_j) / L_ii,
 * each sum accumulated in ascending j.  If some L_ii <= 0 or is not finite
 * (L is then not a Cholesky factor) it returns ORC_ERR_NOT_PD with *info = i
 * and leaves B unchanged.
 */
int orc_solve(const double *L, int64_t n, int64_t ld, double *B, int64_t ldb, int64_t nrhs,
              int64_t *info)
{
    if (info) *info = -1;
    if (n < 0 || nrhs < 0 || ld < (n > 1 ? n : 1) || ldb < (n > 1 ? n : 1)) return ORC_ERR_ARG;
    if (n == 0 || nrhs == 0) return ORC_OK;
    if (!L || !B) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (!finite_pos(L[i + i * ld])) {
            if (info) *info = i;
            return ORC_ERR_NOT_PD;
        }
    }
    for (int64_t r = 0; r < nrhs; ++r) {
        double *x = B + r * ldb;
        for (int64_t i = 0; i < n; ++i) {
            double s = x[i];
            for (int64_t j = 0; j < i; ++j) s -= L[j + i * ld] * x[j];
            x[i] = s / L[i + i * ld];
        }
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = x[i];
            for (int64_t j = i + 1; j < n; ++j) s -= L[i + j * ld] * x[j];
            x[i] = s / L[i + i * ld];
        }
    }
    return ORC_OK;
}
