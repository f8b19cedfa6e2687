// Pass kernels of the rank-k up/downdate for large factors (Walder 2010,
// Algorithm 1; Sec. 4.1's blocking of the update vectors).  A pass takes a
// block of kb <= 16 update vectors and crosses the factor in HBM once for
// the Apply sweep, instead of once per vector.
//
// What a pass computes, for the factor F (upper, A = F^T F), the vectors
// V (n x kb) and the signs Sigma = diag(sigma):
//   1. P = F^{-T} V, a forward substitution with F^T.  Rotating [F; V^T]
//      is rotating [I; P^T] and multiplying by F on the right, so every
//      rotation of Algorithm 1 is fixed by P alone.
//   2. For row r, with the prefix Gram H_r = Sigma + sum_{i<r} p_i p_i^T
//      (p_i the i-th row of P) factored as H_r = U_r Sigma U_r^T (U_r lower
//      triangular), the rotated vectors at the diagonal are y_r = U_r^{-1} p_r
//      (the carries V_r of Algorithm 1 divided by L_rr), and the rotation of
//      vector q at row r is
//          D_0 = 1,  D_q = D_{q-1} + sigma_q y_q^2,
//          c_q = sqrt(D_q / D_{q-1}),  s_q = y_q / sqrt(D_{q-1})
//      (Compute), with the new diagonal L_rr sqrt(D_kb).
//   3. The Apply sweep in scaled variables: a column carries
//      u_hat_q = u_q / t_q with t_q = diag(U_r)_q, and row r is held as
//      S = L_r. / e (e its scale), so that each vector costs two FMAs,
//          S <- S + a_q u_hat_q,   u_hat_q <- u_hat_q - b_q S,
//          a_q = sigma_q y_q t_q,  b_q = y_q / (D_q t_q),
//      and the row ends as L = S / sqrt(D_kb).  (Exact identities of the
//      rotations; the V update uses the new L_ij, Algorithm 1's mixed form.)
// Steps 1 and 2 read the factor once and do O(n^2 kb) and O(n kb^2) work; the
// only serial chain is the forward substitution, run by one thread block
// with the near-diagonal tiles of the next d blocks in shared memory while
// every other warp accumulates the far part of a column block's sum.
//
// Precision: CHM_F64 does everything in double.  CHM_F32_MIXED runs the
// linear work (step 1 and the sweep: the Apply arithmetic) in float and
// step 2 (the prefix Grams, their factors, square roots and ratios: the
// Compute) in double on the promoted float values; the new diagonal is
// formed in double and rounded to float once per pass.
#pragma once

#include "chm_device.cuh"

namespace chm {
namespace pass {

constexpr int kB = 32;     // rows of a row block == columns of a column block
constexpr int kPad = 33;   // shared-memory row stride of a 32 x 32 matrix
constexpr int kMaxKb = 16; // vectors per pass

// Control words of a pass (zeroed before each pass).
constexpr int kCtlWorkTicket = 0;   // next worker task of the forward substitution
constexpr int kCtlRole = 1;         // thread blocks of the substitution started
constexpr int kCtlSweepTicket = 2;  // next sweep task
constexpr int kCtlAbort = 3;        // non-zero once a wait has timed out
constexpr int kCtlInts = 16;

template <typename T>
struct Args {
    T *L;
    const T *V;
    long long n, ld, ldv;
    int nb;                         // row blocks
    int kb;                         // vectors of this pass (<= KB of the kernels)
    int d;                          // lookahead of the substitution chain (near tiles)
    int epoch;                      // tags this pass's flags
    unsigned long long down_mask;   // bit q: vector q is a downdate
    // workspace
    T *P;            // [nb * 32][KB]: F^T P = V, rows past n zero
    T *Zf;           // [nb][32][KB]: V_b - (far tiles)^T P
    T *Dinv;         // [nb][32][32]: (D_b^T)^{-1}, D_b the diagonal block, row-major
    T *G;            // [nb][32][32]: Dinv_b F_{b-1,b}^T, row-major
    double *gram;    // [nb][KB][KB]: sum over the block's rows of p p^T
    double *H;       // [nb][KB][KB]: Sigma + sum over earlier blocks
    T *coef;         // [nb * 32][2 KB]: (a_q, b_q) of each row
    T *escale;       // [nb * 32]: 1 / sqrt(D_kb) of each row
    double *dfac;    // [nb * 32]: sqrt(D_kb) of each row
    int *pflag;      // [nb]: P of the block published (== epoch)
    int *zflag;      // [nb]: far sum of the column block published (== epoch)
    int *ctl;        // kCtlInts control words
    long long *status;     // sticky {status, row} of the stream
    long long *user_info;  // optional {status, row} of the call
    long long timeout_ns;
};

template <typename T>
__device__ __forceinline__ SyncArgs sync_of(const Args<T> &A)
{
    SyncArgs s;
    s.abort_flag = A.ctl + kCtlAbort;
    s.status = A.status;
    s.user_info = A.user_info;
    s.epoch = A.epoch;
    s.timeout_ns = A.timeout_ns;
    return s;
}

template <typename T>
__device__ __forceinline__ double sigma_of(const Args<T> &A, int q)
{
    return ((A.down_mask >> q) & 1ull) ? -1.0 : 1.0;
}

// Asynchronous global -> shared copies of one element (L2 only for 8 and 16
// bytes; 4-byte copies go through L1), completed by cp_wait.
template <typename T>
__device__ __forceinline__ void cp_elem(T *smem, const T *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(T) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- prep

// Per diagonal block b (one warp): Dinv_b = (D_b^T)^{-1} and
// G_b = Dinv_b F_{b-1,b}^T from the factor as it enters the pass, and the
// check that its diagonal is positive and finite (Algorithm 1's Compute
// needs L_ii > 0).  Rows and columns past n are the identity.
template <typename T>
__global__ void __launch_bounds__(32) prep_kernel(Args<T> A)
{
    __shared__ T D[kB][kPad];   // D[i][j] = L(c0 + i, c0 + j), i <= j
    __shared__ T Di[kB][kPad];  // Dinv
    __shared__ T Ft[kB][kPad];  // Ft[l][m] = L(c0 - 32 + m, c0 + l)
    __shared__ T invd[kB];
    const int lane = threadIdx.x;
    const SyncArgs sy = sync_of(A);
    const long long n = A.n, ld = A.ld;
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
        const long long c0 = (long long)b * kB;
        const int rows = (int)min((long long)kB, n - c0);
#pragma unroll 4
        for (int j = 0; j < kB; ++j) {
            T v = T(0);
            if (j < rows && lane <= j) v = A.L[c0 + lane + (c0 + j) * ld];
            else if (lane == j) v = T(1);
            D[lane][j] = v;
        }
        __syncwarp();
        const T dl = D[lane][lane];
        const bool bad = lane < rows && !(dl > T(0) && (double)dl <= DBL_MAX);
        const unsigned badm = __ballot_sync(0xffffffffu, bad);
        if (badm && lane == 0) record_error(sy, kStatusNotPD, c0 + (__ffs(badm) - 1));
        invd[lane] = T(1) / dl;
        __syncwarp();
        // column `lane` of (D^T)^{-1}: x_i = (delta_{i,lane} - sum_{m<i} D[m][i] x_m) / D[i][i]
        T x[kB];
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            T s = (i == lane) ? T(1) : T(0);
#pragma unroll
            for (int m = 0; m < i; ++m) s = fma(-D[m][i], x[m], s);
            x[i] = s * invd[i];
        }
        T *dg = A.Dinv + (size_t)b * kB * kB;
#pragma unroll
        for (int i = 0; i < kB; ++i) {
            Di[i][lane] = x[i];
            dg[i * kB + lane] = x[i];
        }
        __syncwarp();
        if (b > 0) {
            // the tile above the diagonal block: rows of block b - 1 (all < n), columns of block b
#pragma unroll 4
            for (int l = 0; l < kB; ++l) Ft[l][lane] = (l < rows) ? A.L[(c0 - kB + lane) + (c0 + l) * ld] : T(0);
            __syncwarp();
            T *gg = A.G + (size_t)b * kB * kB;
#pragma unroll 4
            for (int i = 0; i < kB; ++i) {
                T g = T(0);
                for (int l = 0; l <= i; ++l) g = fma(Di[i][l], Ft[l][lane], g);
                gg[i * kB + lane] = g;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- forward substitution

// out[i][q] = sum_l M[i][l] in[l][q] over the 256 threads of a block
// (threads per output TPO, consecutive lanes, summed by shuffles); `sub`
// subtracts the product from `out` instead.  Deterministic order.
template <typename T, int KB>
__device__ __forceinline__ void block_mv(const T (*M)[kPad], const T *in, T *out, bool sub)
{
    constexpr int NOUT = kB * KB;
    constexpr int TPO = NOUT >= 256 ? 1 : 256 / NOUT;
    constexpr int PER = NOUT >= 256 ? NOUT / 256 : 1;
    constexpr int LEN = kB / TPO;
    const int t = threadIdx.x;
    const int s = t % TPO;
#pragma unroll
    for (int o = 0; o < PER; ++o) {
        const int idx = t / TPO + o * (256 / TPO);
        const int i = idx % kB, q = idx / kB;
        T a0 = T(0), a1 = T(0);
#pragma unroll
        for (int u = 0; u < LEN; u += 2) {
            const int l = s * LEN + u;
            a0 = fma(M[i][l], in[l * KB + q], a0);
            a1 = fma(M[i][l + 1], in[(l + 1) * KB + q], a1);
        }
        T acc = a0 + a1;
#pragma unroll
        for (int off = TPO / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (s == 0) out[i * KB + q] = sub ? out[i * KB + q] - acc : acc;
    }
}

// Shared memory of the chain block.
template <typename T, int KB, int DMAX>
struct ChainSmem {
    T G[3][kB][kPad];              // G_m of step m (stage m % 3)
    T Di[3][kB][kPad];             // Dinv_{m+1}
    T near[3][DMAX - 1][kB][kPad]; // tiles (m, m + 2 .. m + d), [column][row]
    T acc[DMAX + 1][kB * KB];      // near sums of blocks m + 1 .. m + d
    T P[2][kB * KB];               // P_m, P_{m-1}
    T zhat[kB * KB];               // Dinv_m (Zf_m + acc_m), for the next step
    T w[kB * KB];
    T tmp[kB * KB];
    int stop;
};

template <typename T, int KB, int DMAX>
__device__ void chain_prefetch(const Args<T> &A, ChainSmem<T, KB, DMAX> &S, int m)
{
    // stage of step m: G_m, Dinv_{m+1}, near tiles (m, b), b = m + 2 .. m + d
    const int st = m % 3;
    const int t = threadIdx.x, l = t & 31, g8 = t >> 5;
    const long long n = A.n, ld = A.ld;
    if (m >= 1 && m < A.nb) {
        const T *src = A.G + (size_t)m * kB * kB;
        for (int i = g8; i < kB; i += 8) cp_elem(&S.G[st][i][l], src + i * kB + l);
    }
    if (m + 1 < A.nb) {
        const T *src = A.Dinv + (size_t)(m + 1) * kB * kB;
        for (int i = g8; i < kB; i += 8) cp_elem(&S.Di[st][i][l], src + i * kB + l);
    }
    if (m < A.nb) {
        const long long r0 = (long long)m * kB;
        for (int j = 2; j <= A.d; ++j) {
            const int b = m + j;
            if (b >= A.nb) break;
            const long long c0 = (long long)b * kB;
            for (int i = g8; i < kB; i += 8) {
                if (c0 + i < n) cp_elem(&S.near[st][j - 2][i][l], A.L + (r0 + l) + (c0 + i) * ld);
                else S.near[st][j - 2][i][l] = T(0);
            }
        }
    }
    cp_commit();
}

// The block that walks the forward substitution F^T P = V block by block:
//   P_m = Zhat_m - G_m P_{m-1},  Zhat_m = Dinv_m (Zf_m - sum_{r=m-d}^{m-2} F_{r,m}^T P_r),
// the near sums from its own copies of the tiles, the far sum Zf_m from
// the worker of column block m (m > d), or V_m.
template <typename T, int KB, int DMAX>
__device__ void trsm_chain(const Args<T> &A, unsigned char *smem)
{
    ChainSmem<T, KB, DMAX> &S = *reinterpret_cast<ChainSmem<T, KB, DMAX> *>(smem);
    const int t = threadIdx.x;
    const int nb = A.nb, d = A.d;
    const long long n = A.n;
    const SyncArgs sy = sync_of(A);
    for (int x = t; x < (DMAX + 1) * kB * KB; x += 256) (&S.acc[0][0])[x] = T(0);
    if (t == 0) S.stop = 0;
    // Zhat_0 = Dinv_0 V_0
    {
        const T *src = A.Dinv;
        for (int i = t >> 5; i < kB; i += 8) S.Di[2][i][t & 31] = src[i * kB + (t & 31)];
        for (int x = t; x < kB * KB; x += 256) {
            const int i = x / KB, q = x % KB;
            S.w[x] = (i < n && q < A.kb) ? A.V[i + q * A.ldv] : T(0);
        }
        __syncthreads();
        block_mv<T, KB>(S.Di[2], S.w, S.zhat, false);
        __syncthreads();
    }
    chain_prefetch<T, KB, DMAX>(A, S, 0);
    chain_prefetch<T, KB, DMAX>(A, S, 1);
    for (int m = 0; m < nb; ++m) {
        const int st = m % 3;
        chain_prefetch<T, KB, DMAX>(A, S, m + 2);
        cp_wait<2>();
        __syncthreads();
        T *Pm = S.P[m & 1];
        // critical step: P_m = Zhat_m - G_m P_{m-1}
        if (m == 0) {
            for (int x = t; x < kB * KB; x += 256) Pm[x] = S.zhat[x];
        } else {
            block_mv<T, KB>(S.G[st], S.P[(m - 1) & 1], S.tmp, false);
            __syncthreads();
            for (int x = t; x < kB * KB; x += 256) Pm[x] = S.zhat[x] - S.tmp[x];
        }
        __syncthreads();
        for (int x = t; x < kB * KB; x += 256) __stcg(A.P + (size_t)m * kB * KB + x, Pm[x]);
        __syncthreads();
        if (t == 0) {
            __threadfence();
            st_release_gpu(A.pflag + m, A.epoch);
        }
        // near sums of later blocks with P_m: tiles (m, m + 2 .. m + d)
        for (int j = 2; j <= d; ++j) {
            const int b = m + j;
            if (b >= nb) break;
            block_mv<T, KB>(S.near[st][j - 2], Pm, S.acc[b % (DMAX + 1)], true);
        }
        // Zhat_{m+1} = Dinv_{m+1} (Zf_{m+1} + acc_{m+1})
        if (m + 1 < nb) {
            const int b = m + 1;
            if (b > d) {
                if (t == 0) {
                    const bool ok = bounded_wait(
                        sy, [&] { return ld_relaxed_gpu(A.zflag + b) == A.epoch; },
                        [] { fence_acq_rel_gpu(); }, b);
                    S.stop = ok ? 0 : 1;
                }
                __syncthreads();
                if (S.stop) {
                    cp_wait<0>();
                    return;
                }
                const T *zf = A.Zf + (size_t)b * kB * KB;
                for (int x = t; x < kB * KB; x += 256) S.w[x] = __ldcg(zf + x) + S.acc[b % (DMAX + 1)][x];
            } else {
                const long long r0 = (long long)b * kB;
                for (int x = t; x < kB * KB; x += 256) {
                    const int i = x / KB, q = x % KB;
                    const T v = (r0 + i < n && q < A.kb) ? A.V[r0 + i + q * A.ldv] : T(0);
                    S.w[x] = v + S.acc[b % (DMAX + 1)][x];
                }
            }
            __syncthreads();
            block_mv<T, KB>(S.Di[st], S.w, S.zhat, false);
            for (int x = t; x < kB * KB; x += 256) S.acc[b % (DMAX + 1)][x] = T(0);
        }
        __syncthreads();
    }
    cp_wait<0>();
}

// Worker warps: the far part of column block b's sum,
//   Zf_b = V_b - sum_{r < b - d} F_{r,b}^T P_r,
// one tile per published P_r, the next tile fetched while this one is used.
template <typename T, int KB>
__device__ void trsm_workers(const Args<T> &A, unsigned char *smem)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kTile = kB * kPad;
    T *base = reinterpret_cast<T *>(smem) + (size_t)warp * 2 * (kTile + kB * KB);
    T *tile[2] = {base, base + kTile};
    T *Pr = base + 2 * kTile;  // [32][KB]
    const long long n = A.n, ld = A.ld;
    const int nb = A.nb, d = A.d;
    const SyncArgs sy = sync_of(A);
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = ld_relaxed_gpu(A.ctl + kCtlAbort) ? -1 : atomicAdd(A.ctl + kCtlWorkTicket, 1);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk < 0) return;
        const int b = d + 1 + tk;
        if (b >= nb) return;
        const long long c0 = (long long)b * kB;
        const bool col_ok = c0 + lane < n;
        T z[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) z[q] = (col_ok && q < A.kb) ? A.V[c0 + lane + q * A.ldv] : T(0);
        const int nfar = b - d;
        auto fetch = [&](int r, T *dst) {
            const long long r0 = (long long)r * kB;
#pragma unroll 8
            for (int i = 0; i < kB; ++i) {
                if (c0 + i < n) cp_elem(dst + i * kPad + lane, A.L + (r0 + lane) + (c0 + i) * ld);
                else dst[i * kPad + lane] = T(0);
            }
            cp_commit();
        };
        fetch(0, tile[0]);
        for (int r = 0; r < nfar; ++r) {
            if (r + 1 < nfar) fetch(r + 1, tile[(r + 1) & 1]);
            int ok = 1;
            if (lane == 0)
                ok = bounded_wait(sy, [&] { return ld_relaxed_gpu(A.pflag + r) == A.epoch; },
                                  [] { fence_acq_rel_gpu(); }, b) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) return;
            const T *src = A.P + (size_t)r * kB * KB;
#pragma unroll
            for (int x = lane; x < kB * KB; x += 32) Pr[x] = __ldcg(src + x);
            if (r + 1 < nfar) cp_wait<1>();
            else cp_wait<0>();
            __syncwarp();
            const T *tl = tile[r & 1] + lane * kPad;
            if (KB == 1) {
                T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
#pragma unroll
                for (int l = 0; l < kB; l += 4) {
                    s0 = fma(tl[l], Pr[l], s0);
                    s1 = fma(tl[l + 1], Pr[l + 1], s1);
                    s2 = fma(tl[l + 2], Pr[l + 2], s2);
                    s3 = fma(tl[l + 3], Pr[l + 3], s3);
                }
                z[0] -= (s0 + s1) + (s2 + s3);
            } else {
#pragma unroll 4
                for (int l = 0; l < kB; ++l) {
                    const T f = tl[l];
#pragma unroll
                    for (int q = 0; q < KB; ++q) z[q] = fma(-f, Pr[l * KB + q], z[q]);
                }
            }
            __syncwarp();
        }
        T *zf = A.Zf + (size_t)b * kB * KB + (size_t)lane * KB;
#pragma unroll
        for (int q = 0; q < KB; ++q) __stcg(zf + q, z[q]);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            st_release_gpu(A.zflag + b, A.epoch);
        }
    }
}

template <typename T, int KB, int DMAX>
__global__ void __launch_bounds__(256, 1) trsm_kernel(Args<T> A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_role;
    if (threadIdx.x == 0) s_role = atomicAdd(A.ctl + kCtlRole, 1);
    __syncthreads();
    if (s_role == 0) trsm_chain<T, KB, DMAX>(A, smem);
    else trsm_workers<T, KB>(A, smem);
}

// ---------------------------------------------------------------- Compute

// gram[b] = sum over the rows of block b of p p^T (double), one warp per block.
template <typename T, int KB>
__global__ void __launch_bounds__(32) gram_kernel(Args<T> A)
{
    __shared__ double p[kB][KB];
    const int lane = threadIdx.x;
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
        const T *src = A.P + (size_t)b * kB * KB;
        for (int x = lane; x < kB * KB; x += 32) (&p[0][0])[x] = (double)src[x];
        __syncwarp();
        double *g = A.gram + (size_t)b * KB * KB;
        for (int e = lane; e < KB * KB; e += 32) {
            const int q = e / KB, r = e % KB;
            double s0 = 0.0, s1 = 0.0;
#pragma unroll
            for (int i = 0; i < kB; i += 2) {
                s0 = fma(p[i][q], p[i][r], s0);
                s1 = fma(p[i + 1][q], p[i + 1][r], s1);
            }
            g[e] = s0 + s1;
        }
        __syncwarp();
    }
}

// H[b] = Sigma + sum_{b' < b} gram[b'] for every entry: thread (entry,
// segment) of one block of 1024 threads; blockIdx.x picks 32 entries.
template <typename T, int KB>
__global__ void __launch_bounds__(1024) scan_kernel(Args<T> A)
{
    __shared__ double seg[32][33];
    const int e = blockIdx.x * 32 + (threadIdx.x & 31);  // entry
    const int s = threadIdx.x >> 5;                      // segment
    const int nb = A.nb;
    const int len = (nb + 31) / 32;
    const int b0 = s * len, b1 = min(nb, b0 + len);
    const bool valid = e < KB * KB;
    double sum = 0.0;
    if (valid)
        for (int b = b0; b < b1; ++b) sum += A.gram[(size_t)b * KB * KB + e];
    seg[s][threadIdx.x & 31] = sum;
    __syncthreads();
    double pre = 0.0;
    if (valid) {
        const int q = e / KB, r = e % KB;
        pre = (q == r) ? sigma_of(A, q) : 0.0;
        if (q >= A.kb || r >= A.kb) pre = (q == r) ? 1.0 : 0.0;  // padding vectors: identity
        for (int s2 = 0; s2 < s; ++s2) pre += seg[s2][threadIdx.x & 31];
        for (int b = b0; b < b1; ++b) {
            A.H[(size_t)b * KB * KB + e] = pre;
            pre += A.gram[(size_t)b * KB * KB + e];
        }
    }
}

// Per row block b (one warp): U with H_b = U Sigma U^T, then the rows in
// order: lane r's rotated vector y_r = x_r, its rotations (D, a, b) and the
// transform of the later rows' vectors,
//   x_q <- (D_{q-1} x_q - y_q sum_{q'<q} sigma_q' y_q' x_q') / sqrt(D_{q-1} D_q),
// the carry scales t_q <- t_q sqrt(D_q / D_{q-1}).  Lanes are rows; vectors
// q < kb (padding vectors have p = 0 and change nothing).
template <typename T, int KB>
__global__ void __launch_bounds__(32) coef_kernel(Args<T> A)
{
    __shared__ double U[KB][KB + 1];
    __shared__ double iu[KB];
    __shared__ double sh_y[KB], sh_al[KB], sh_be[KB];
    __shared__ double sh_t[KB];
    const int lane = threadIdx.x;
    const SyncArgs sy = sync_of(A);
    const long long n = A.n;
    const int kb = A.kb;
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
        const long long r0 = (long long)b * kB;
        const int rows = (int)min((long long)kB, n - r0);
        // LDL^T of H_b (lane = row of H), U = L sqrt|D|
        if (lane < KB)
            for (int j = 0; j < KB; ++j) U[lane][j] = A.H[(size_t)b * KB * KB + lane * KB + j];
        __syncwarp();
        bool badH = false;
        for (int j = 0; j < kb; ++j) {
            // column j: D_j on lane j, then L_ij for i > j (U holds L below the
            // diagonal and D on it while being built)
            if (lane == j) {
                double dj = U[j][j];
                for (int m = 0; m < j; ++m) dj -= U[j][m] * U[j][m] * U[m][m];
                U[j][j] = dj;
            }
            __syncwarp();
            const double dj = U[j][j];
            if (lane > j && lane < kb) {
                double v = U[lane][j];
                for (int m = 0; m < j; ++m) v -= U[lane][m] * U[j][m] * U[m][m];
                U[lane][j] = v / dj;
            }
            __syncwarp();
        }
        if (lane < kb) {
            const double dd = U[lane][lane];
            badH = !(dd * sigma_of(A, lane) > 0.0 && fabs(dd) <= DBL_MAX);
        }
        __syncwarp();
        // U = L sqrt|D| (column scaling), iu = 1 / diag(U)
        if (lane < kb) {
            const double sd = sqrt(fabs(U[lane][lane]));
            sh_t[lane] = sd;
            iu[lane] = 1.0 / sd;
        }
        __syncwarp();
        if (lane < kb)
            for (int j = 0; j < lane; ++j) U[lane][j] *= sh_t[j];
        __syncwarp();
        if (lane < kb) U[lane][lane] = sh_t[lane];
        __syncwarp();
        {
            const unsigned m = __ballot_sync(0xffffffffu, badH);
            if (m && lane == 0) record_error(sy, kStatusNotPD, r0);
        }
        // x = U^{-1} p for this lane's row
        double x[KB];
        const T *prow = A.P + (size_t)(r0 + lane) * KB;
#pragma unroll
        for (int q = 0; q < KB; ++q) x[q] = (q < kb) ? (double)__ldcg(prow + q) : 0.0;
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            if (q < kb) {
                double s = x[q];
#pragma unroll
                for (int m = 0; m < q; ++m) s -= U[q][m] * x[m];
                x[q] = s * iu[q];
            }
        }
        double tq[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) tq[q] = (q < kb) ? sh_t[q] : 1.0;
        for (int r = 0; r < rows; ++r) {
            if (lane == r) {
                double Dp = 1.0;
                bool bad = false;
                T *cf = A.coef + (size_t)(r0 + r) * 2 * KB;
#pragma unroll
                for (int q = 0; q < KB; ++q) {
                    if (q < kb) {
                        const double sg = sigma_of(A, q), y = x[q];
                        const double Dq = fma(sg * y, y, Dp);
                        bad = bad || !(Dq > 0.0 && Dq <= DBL_MAX);
                        const double rs = rsqrt_refined(Dp * Dq);   // 1 / sqrt(D_{q-1} D_q)
                        sh_y[q] = sg * y;
                        sh_al[q] = Dp * rs;                       // sqrt(D_{q-1} / D_q)
                        sh_be[q] = y * rs;
                        cf[2 * q] = (T)(sg * y * tq[q]);
                        cf[2 * q + 1] = (T)(y * rcp_refined(Dq * tq[q]));
                        Dp = Dq;
                    } else {
                        sh_y[q] = 0.0;
                        sh_al[q] = 1.0;
                        sh_be[q] = 0.0;
                        cf[2 * q] = T(0);
                        cf[2 * q + 1] = T(0);
                    }
                }
                const double rD = rsqrt_refined(Dp);
                A.escale[r0 + r] = (T)rD;
                A.dfac[r0 + r] = Dp * rD;
                if (bad) record_error(sy, kStatusNotPD, r0 + r);
            }
            __syncwarp();
            // every lane: the carry scales; later rows: their vectors
#pragma unroll
            for (int q = 0; q < KB; ++q) tq[q] /= sh_al[q] > 0.0 ? sh_al[q] : 1.0;
            if (lane > r) {
                double acc = 0.0;
#pragma unroll
                for (int q = 0; q < KB; ++q) {
                    if (q < kb) {
                        const double xq = x[q];
                        x[q] = sh_al[q] * xq - sh_be[q] * acc;
                        acc = fma(sh_y[q], xq, acc);
                    }
                }
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- sweep

// Column block b, rows 0 .. b of the pass's Apply: lane = column, kb carries
// in registers, tiles and their rows' coefficients staged in a ring of
// three slots (cp.async) so that two tiles are in flight while one is used.
template <typename T, int KB>
struct SweepSlot {
    T tile[kB][kPad];     // [column][row]
    T cf[kB][2 * KB];     // (a, b) per row
    T e[kB];
    double df[kB];
};

template <typename T, int KB>
__global__ void __launch_bounds__(128) sweep_kernel(Args<T> A, int warps_per_block)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SweepSlot<T, KB> *slot = reinterpret_cast<SweepSlot<T, KB> *>(smem) + (size_t)warp * 3;
    const long long n = A.n, ld = A.ld;
    const int nb = A.nb;
    (void)warps_per_block;
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = atomicAdd(A.ctl + kCtlSweepTicket, 1);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk >= nb) return;
        const int b = nb - 1 - tk;  // largest first
        const long long c0 = (long long)b * kB;
        const bool active = c0 + lane < n;
        T uh[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) uh[q] = (active && q < A.kb) ? A.V[c0 + lane + q * A.ldv] : T(0);
        auto fetch = [&](int r) {
            SweepSlot<T, KB> &s = slot[r % 3];
            const long long r0 = (long long)r * kB;
            const bool diag = r == b;
#pragma unroll 8
            for (int i = 0; i < kB; ++i) {
                // the diagonal tile needs rows <= column only
                if (c0 + i < n && (!diag || lane <= i)) cp_elem(&s.tile[i][lane], A.L + (r0 + lane) + (c0 + i) * ld);
            }
            const T *cf = A.coef + (size_t)r0 * 2 * KB;
            for (int x = lane; x < kB * 2 * KB; x += 32) cp_elem(&s.cf[0][0] + x, cf + x);
            cp_elem(&s.e[lane], A.escale + r0 + lane);
            if (diag) cp_elem(&s.df[lane], A.dfac + r0 + lane);
            cp_commit();
        };
        fetch(0);
        if (b >= 1) fetch(1);
        for (int r = 0; r <= b; ++r) {
            if (r + 2 <= b) fetch(r + 2);
            if (r + 2 <= b) cp_wait<2>();
            else if (r + 1 <= b) cp_wait<1>();
            else cp_wait<0>();
            __syncwarp();
            SweepSlot<T, KB> &s = slot[r % 3];
            const bool diag = r == b;
            const long long r0 = (long long)r * kB;
            const int rows = diag ? lane : (int)min((long long)kB, n - r0);
            T *col = s.tile[lane];
            if (active) {
#pragma unroll 4
                for (int i = 0; i < kB; ++i) {
                    if (i < rows) {
                        T v = col[i];
#pragma unroll
                        for (int q = 0; q < KB; ++q) {
                            v = fma(s.cf[i][2 * q], uh[q], v);
                            uh[q] = fma(-s.cf[i][2 * q + 1], v, uh[q]);
                        }
                        col[i] = v * s.e[i];
                    }
                }
                if (diag) col[lane] = (T)((double)col[lane] * s.df[lane]);
            }
            __syncwarp();
#pragma unroll 8
            for (int i = 0; i < kB; ++i)
                if (c0 + i < n && (!diag || lane <= i)) A.L[(r0 + lane) + (c0 + i) * ld] = s.tile[i][lane];
            __syncwarp();
        }
    }
}

}  // namespace pass
}  // namespace chm
