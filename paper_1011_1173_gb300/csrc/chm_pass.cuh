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
// Offsets the substitution's critical warp takes itself, at most (through G^(j) = Dinv F_{b-j,b}^T).
constexpr int kMaxCrit = 4;
// Offsets whose G^(j) the pass forms, at most: the lookahead's bound (the
// near warps' terms are G^(j) P as well, so that W_m needs no product
// with Dinv_m on the chain block).
constexpr int kMaxG = 10;

// Control words of a pass (zeroed before each pass).
constexpr int kCtlWorkTicket = 0;   // next worker task of the forward substitution
constexpr int kCtlRole = 1;         // thread blocks of the substitution started
constexpr int kCtlSweepTicket = 2;  // next sweep task
constexpr int kCtlAbort = 3;        // non-zero once a wait has timed out
constexpr int kCtlPostTicket = 4;   // next coefficient or sweep task of a fused pass
constexpr int kCtlAugTicket = 5;    // the right-hand sides' recurrence (one task)
constexpr int kCtlInts = 16;

template <typename T>
struct Args {
    T *L;
    const T *V;
    long long n, ld, ldv;
    int nb;                         // row blocks
    int kb;                         // vectors of this pass (<= KB of the kernels)
    int kr;                         // the first kr of them rotate the factor (update vectors);
                                    // vectors kr .. kb - 1 are right-hand sides the substitution
                                    // carries along (chm_modify_solve): columns of B
    const T *B;                     // right-hand sides: vector q >= kr is column q - kr of B
    long long ldb;
    int d;                          // lookahead of the substitution chain (near tiles)
    int c;                          // offsets the chain's critical warp takes (G^(1..c))
    int epoch;                      // tags this pass's flags
    unsigned long long down_mask;   // bit q: vector q is a downdate
    // workspace
    T *P;            // [nb * 32][KB]: F^T P = V, rows past n zero
    T *Dinv;         // [nb][32][32]: (D_b^T)^{-1}, D_b the diagonal block, row-major
    T *G;            // [d][nb][32][32]: G^(j)_b = Dinv_b F_{b-j,b}^T, row-major
    double *gram;    // [nb][KB][KB]: sum over the block's rows of p p^T
    double *H;       // [nb][KB][KB]: Sigma + sum over earlier blocks
    T *coef;         // [nb * 32][2 KB]: (a_q, b_q) of each row
    T *escale;       // [nb * 32]: 1 / sqrt(D_kb) of each row
    double *dfac;    // [nb * 32]: sqrt(D_kb) of each row
    T *snap;         // [nbound][nb * 32][KB]: each column's partial residual of the substitution,
                     // V_j - sum over rows below s seg 32 of F_ij p_i, at boundary s = 1 .. nbound
    double *rst;     // [nbound][KB (KB + 1) / 2]: packed LDL^T of the prefix Gram at each boundary
    const int2 *tasks;  // [ntasks]: the sweep's (column block, segment) tasks, longest first
    int ntasks;
    int seg;         // row blocks per sweep segment
    // fused pass (the substitution kernel's workers also compute the
    // coefficients and sweep, each part as soon as its inputs are out)
    int fused;
    const int2 *post;   // [npost]: after the far sums, (-1, r) coefficients of row block r or
                        // (b, s) sweep segment s of column block b, in an order their inputs allow
    int npost;
    int *cflag;         // [nb]: row block b's coefficients published (== epoch)
    long long *wprog;   // [nb]: (epoch << 32) + row blocks the worker of column block b has consumed
    long long *Ptag; // [nb * 32][KB][words of T]: P as epoch-tagged words, for readers within the launch
    long long *Htag; // [nb][KB * KB][2]: a fused pass's prefix Grams H_b as tagged doubles
    long long *Ztag; // [nb][32][KB][words of T]: Zf as epoch-tagged words
    int *ctl;        // kCtlInts control words
    long long *status;     // sticky {status, row} of the stream
    long long *user_info;  // optional {status, row} of the call
    long long timeout_ns;
    long long *trace;      // optional [nb][16] %globaltimer stamps of the substitution:
                           // 0 P posted, 1 W posted, 2 far sum staged, 4 P published,
                           // 5 first near warp done, 6 W warp's inputs in, 7 critical
                           // warp's inputs in, 8 a worker's last P seen, 9 its far sum out
    const char *ws;        // the workspace allocation the regions above are carved from
    size_t ws_bytes;
    long long chk_cut;     // bounds-checked build: columns taken off the factor's declared extent
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
    s.chk_cut = A.chk_cut;
    return s;
}

// Entry (row, q) of the pass's input vectors: column q of V for the update
// vectors (q < kr), column q - kr of B for the right-hand sides (q < kb),
// zero past them and past the order.
template <typename T>
__device__ __forceinline__ T vin(const Args<T> &A, const SyncArgs &sy, long long row, int q)
{
    (void)sy;
    if (row >= A.n || q >= A.kb) return T(0);
    if (q < A.kr) return CHK_RECT(sy, row + q * A.ldv, A.n, A.kr, A.ldv) ? A.V[row + q * A.ldv] : T(0);
    const int c = q - A.kr;
    return CHK_RECT(sy, row + c * A.ldb, A.n, A.kb - A.kr, A.ldb) ? A.B[row + c * A.ldb] : T(0);
}

// Bounds-checked builds: every workspace region a kernel with KB vectors
// per pass indexes lies inside the workspace allocation, and the pass's
// shape fits the regions (the kernel returns at once otherwise).
template <typename T, int KB>
__device__ __forceinline__ bool ws_ok(const Args<T> &A, const SyncArgs &sy)
{
#ifdef CHM_CHECK
    const size_t nb = (size_t)A.nb, rows = nb * kB, e = sizeof(T);
    const size_t tagw = e / 4;  // 64-bit words of one tagged value
    return CHK_RECT(sy, (long long)A.kb, KB + 1, 1, 1 << 30) && CHK_RECT(sy, (long long)A.kr, (long long)A.kb + 1, 1, 1 << 30) &&
           CHK_RECT(sy, (long long)A.c, kMaxCrit + 1, 1, 1 << 30) &&
           CHK_RECT(sy, A.n, (long long)rows + 1, 1, 1ll << 62) &&
           CHK_REGION(sy, A.P, rows * KB * e, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.Ptag, rows * KB * tagw * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.Htag, nb * KB * KB * 16, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.Ztag, rows * KB * tagw * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.Dinv, nb * kB * kB * e, A.ws, A.ws_bytes) &&
           CHK_RECT(sy, (long long)A.d, kMaxG + 1, 1, 1 << 30) &&
           CHK_REGION(sy, A.G, (size_t)A.d * nb * kB * kB * e, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.gram, nb * KB * KB * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.H, nb * KB * KB * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.coef, rows * 2 * KB * e, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.escale, rows * e, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.dfac, rows * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.snap, (nb > 1 ? (nb - 1) / (size_t)A.seg : 0) * rows * KB * e, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.rst, (nb > 1 ? (nb - 1) / (size_t)A.seg : 0) * KB * (KB + 1) / 2 * 8, A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.tasks, (size_t)A.ntasks * sizeof(int2), A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.ctl, kCtlInts * sizeof(int), A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.cflag, nb * sizeof(int), A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.wprog, nb * sizeof(long long), A.ws, A.ws_bytes) &&
           CHK_REGION(sy, A.post, (size_t)A.npost * sizeof(int2), A.ws, A.ws_bytes);
#else
    (void)A;
    (void)sy;
    return true;
#endif
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
// G^(j)_b = Dinv_b F_{b-j,b}^T, j = 1 .. d, from the factor as it enters the pass, and the
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
    if (!ws_ok<T, kMaxKb>(A, sy)) return;  // touches no region that depends on the pass's vectors
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
        const long long c0 = (long long)b * kB;
        const int rows = (int)min((long long)kB, n - c0);
#pragma unroll 4
        for (int j = 0; j < kB; ++j) {
            T v = T(0);
            if (j < rows && lane <= j && CHK_TRI(sy, c0 + lane + (c0 + j) * ld, n, ld)) v = A.L[c0 + lane + (c0 + j) * ld];
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
        for (int j = 1; j <= A.d && j <= b; ++j) {
            // the tile j blocks above the diagonal block: rows of block b - j (all < n), columns of block b
            const long long rj = c0 - (long long)j * kB;
#pragma unroll 4
            for (int l = 0; l < kB; ++l)
                Ft[l][lane] = (l < rows && CHK_TRI(sy, (rj + lane) + (c0 + l) * ld, n, ld)) ? A.L[(rj + lane) + (c0 + l) * ld] : T(0);
            __syncwarp();
            T *gg = A.G + ((size_t)(j - 1) * A.nb + b) * kB * kB;
#pragma unroll 4
            for (int i = 0; i < kB; ++i) {
                T g = T(0);
                for (int l = 0; l <= i; ++l) g = fma(Di[i][l], Ft[l][lane], g);
                gg[i * kB + lane] = g;
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- forward substitution

// Shared-memory row stride of a staged 32 x 32 tile: 16-byte rows (36 floats,
// 34 doubles), so that tiles arrive in 16-byte chunks and a lane reading its
// own row with 16-byte loads hits distinct banks.
template <typename T>
struct Stride {
    static constexpr int value = kB + 16 / (int)sizeof(T);
};
// 16-byte vector of T.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
};
template <>
struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
};
template <typename T>
__device__ __forceinline__ T vget(const typename Vec16<T>::type &v, int u);
template <>
__device__ __forceinline__ float vget<float>(const float4 &v, int u)
{
    return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w;
}
template <>
__device__ __forceinline__ double vget<double>(const double2 &v, int u)
{
    return u == 0 ? v.x : v.y;
}

__device__ __forceinline__ void cp16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
// The chain block's prefetches ask L2 to keep the lines (they are read a
// few steps later, while the workers and the sweep stream the factor).
__device__ __forceinline__ void prefetch_l2(const void *gmem)
{
    asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(gmem));
}
// A plain prefetch into L2 (normal eviction priority).
__device__ __forceinline__ void prefetch_l2n(const void *gmem)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gmem));
}
// An L2 policy that evicts first: the sweep's tiles are read and written
// once, so they should not push out what the chain block prefetched.
__device__ __forceinline__ unsigned long long evict_first_policy()
{
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void cp16_hint(void *smem, const void *gmem, unsigned long long pol)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "l"(pol)
                 : "memory");
}
template <typename V>
__device__ __forceinline__ void st16_hint(V *gmem, const V &v, unsigned long long pol)
{
    const unsigned *w = reinterpret_cast<const unsigned *>(&v);
    asm volatile("st.global.L2::cache_hint.v4.b32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(gmem), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "l"(pol)
                 : "memory");
}

// Warp-cooperative stage of the tile rows r0.. r0 + 31, columns c0 .. c0 + 31
// of L into dst[column][Stride] (columns >= n are zero).  `vec`: 16-byte
// copies (every column's segment 16-byte aligned and all 32 rows inside the
// column, r0 + 32 <= n); otherwise one element per copy, rows >= nrows zero.
template <typename T>
__device__ __forceinline__ void stage_tile(const SyncArgs &sy, T *dst, const T *L, long long ld, long long r0,
                                           long long c0, long long n, int nrows, bool vec, int lane)
{
    constexpr int S = Stride<T>::value;
    if (vec) {
        constexpr int E = 16 / (int)sizeof(T);  // elements per chunk
        constexpr int CPC = kB / E;             // chunks per column
        for (int c = lane; c < kB * CPC; c += 32) {
            const int col = c / CPC, ch = c % CPC;
            T *d = dst + col * S + ch * E;
            const long long o = (r0 + ch * E) + (c0 + col) * ld;
            if (c0 + col < n && CHK_TRI(sy, o, n, ld) && CHK_TRI(sy, o + E - 1, n, ld)) {
                cp16(d, L + o);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) d[e] = T(0);
            }
        }
    } else {
        for (int col = 0; col < kB; ++col) {
            T *d = dst + col * S + lane;
            const long long o = (r0 + lane) + (c0 + col) * ld;
            if (c0 + col < n && lane < nrows && CHK_TRI(sy, o, n, ld)) cp_elem(d, L + o);
            else *d = T(0);
        }
    }
}
// The same for a dense row-major 32 x 32 matrix of the workspace (always
// 16-byte aligned): dst[row][Stride].
template <typename T>
__device__ __forceinline__ void stage_dense(T *dst, const T *src, int lane)
{
    constexpr int S = Stride<T>::value;
    constexpr int E = 16 / (int)sizeof(T);
    constexpr int CPR = kB / E;
    for (int c = lane; c < kB * CPR; c += 32) {
        const int row = c / CPR, ch = c % CPR;
        cp16(dst + row * S + ch * E, src + row * kB + ch * E);
    }
}

// A [32][KB] array of per-row vectors in shared memory: row stride KS so
// that 32 lanes each reading or writing their own row in 16-byte pieces hit
// distinct banks (an odd number of 16-byte units per row), and rows of
// fewer than 16 bytes stay contiguous.
template <typename T, int KB>
struct Rows {
    static constexpr int bytes = KB * (int)sizeof(T);
    static constexpr int E = 16 / (int)sizeof(T);
    static constexpr int KS = bytes < 16 ? KB : (((bytes / 16) & 1) ? KB : KB + E);
    static constexpr int size = kB * KS;
};
template <typename T, int KB>
__device__ __forceinline__ void row_store(T *base, int lane, const T (&v)[KB])
{
    using R = Rows<T, KB>;
    T *p = base + lane * R::KS;
    if (R::bytes % 16 == 0) {
        using V = typename Vec16<T>::type;
#pragma unroll
        for (int g = 0; g < KB / R::E; ++g) {
            V x;
            T *xp = reinterpret_cast<T *>(&x);
#pragma unroll
            for (int u = 0; u < R::E; ++u) xp[u] = v[g * R::E + u];
            reinterpret_cast<V *>(p)[g] = x;
        }
    } else {
#pragma unroll
        for (int q = 0; q < KB; ++q) p[q] = v[q];
    }
}
template <typename T, int KB>
__device__ __forceinline__ void row_load(const T *base, int lane, T (&v)[KB])
{
    using R = Rows<T, KB>;
    const T *p = base + lane * R::KS;
    if (R::bytes % 16 == 0) {
        using V = typename Vec16<T>::type;
#pragma unroll
        for (int g = 0; g < KB / R::E; ++g) {
            const V x = reinterpret_cast<const V *>(p)[g];
            const T *xp = reinterpret_cast<const T *>(&x);
#pragma unroll
            for (int u = 0; u < R::E; ++u) v[g * R::E + u] = xp[u];
        }
    } else {
#pragma unroll
        for (int q = 0; q < KB; ++q) v[q] = p[q];
    }
}

// Lane i: out[q] (+)= sum_l M[i][l] x[l][q] (M staged with Stride, x a Rows array).
template <typename T, int KB>
__device__ __forceinline__ void lane_mv(const T *M, const T *x, T (&out)[KB], int i, bool acc = false)
{
    constexpr int S = Stride<T>::value;
    constexpr int E = Vec16<T>::n;
    constexpr int XS = Rows<T, KB>::KS;
    using V = typename Vec16<T>::type;
    T a0[KB], a1[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
        a0[q] = acc ? out[q] : T(0);
        a1[q] = T(0);
    }
    const V *row = reinterpret_cast<const V *>(M + i * S);
#pragma unroll
    for (int c = 0; c < kB / E; ++c) {
        const V m = row[c];
#pragma unroll
        for (int u = 0; u < E; ++u) {
            const int l = c * E + u;
            const T mv = vget<T>(m, u);
            if (KB % E == 0) {
                // x[l][*] as 16-byte broadcast loads
                const V *xr = reinterpret_cast<const V *>(x + l * XS);
#pragma unroll
                for (int g = 0; g < KB / E; ++g) {
                    const V xv = xr[g];
#pragma unroll
                    for (int w = 0; w < E; ++w) {
                        const int q = g * E + w;
                        if (l & 1) a1[q] = fma(mv, vget<T>(xv, w), a1[q]);
                        else a0[q] = fma(mv, vget<T>(xv, w), a0[q]);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < KB; ++q) {
                    if (l & 1) a1[q] = fma(mv, x[l * XS + q], a1[q]);
                    else a0[q] = fma(mv, x[l * XS + q], a0[q]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) out[q] = a0[q] + a1[q];
}
// The same with this lane's row of M in registers (the same order of
// operations, so the same result bit for bit).
template <typename T, int KB>
__device__ __forceinline__ void lane_mv_reg(const T (&mrow)[kB], const T *x, T (&out)[KB])
{
    constexpr int E = Vec16<T>::n;
    constexpr int XS = Rows<T, KB>::KS;
    using V = typename Vec16<T>::type;
    T a0[KB], a1[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
        a0[q] = T(0);
        a1[q] = T(0);
    }
#pragma unroll
    for (int l = 0; l < kB; ++l) {
        const T mv = mrow[l];
        if (KB % E == 0) {
            const V *xr = reinterpret_cast<const V *>(x + l * XS);
#pragma unroll
            for (int g = 0; g < KB / E; ++g) {
                const V xv = xr[g];
#pragma unroll
                for (int w = 0; w < E; ++w) {
                    const int q = g * E + w;
                    if (l & 1) a1[q] = fma(mv, vget<T>(xv, w), a1[q]);
                    else a0[q] = fma(mv, vget<T>(xv, w), a0[q]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < KB; ++q) {
                if (l & 1) a1[q] = fma(mv, x[l * XS + q], a1[q]);
                else a0[q] = fma(mv, x[l * XS + q], a0[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) out[q] = a0[q] + a1[q];
}

// A value published as epoch-tagged 64-bit words (one per 32 bits of T):
// each 8-byte store is single-copy atomic, so a reader that sees every word
// tagged with the current epoch has the value, and no fence or flag is needed.
template <typename T>
struct Tag {
    static constexpr int words = (int)sizeof(T) / 4;
};
__device__ __forceinline__ void put_tag(long long *w, float v, long long ep64)
{
    __stcg(w, ep64 | (long long)(unsigned)__float_as_uint(v));
}
__device__ __forceinline__ void put_tag(long long *w, double v, long long ep64)
{
    put_tagged(w, v, ep64);
}
__device__ __forceinline__ bool get_tag(const long long *w, long long ep64, float *v)
{
    const long long x = ld_relaxed_gpu(w);
    if ((x & ~0xffffffffll) != ep64) return false;
    *v = __uint_as_float((unsigned)(x & 0xffffffffll));
    return true;
}
__device__ __forceinline__ bool get_tag(const long long *w, long long ep64, double *v)
{
    return get_tagged(w, ep64, v);
}

// Every lane reads its KB tagged values (a row of P) until all of the
// warp's words carry the epoch; sleeps between polls up to max_ns.  False if
// the launch is being aborted or the wait ran out (recorded).
//
// While the row is not out, the warp polls one word of it (the last word
// lane 31's row gets, the publisher's last store): one L2 request per poll
// instead of 32 KB words.  A thousand worker warps may be waiting on the
// same row at the front of the chain, and their full-row polls, KB times
// heavier, slow the L2 slices that the chain's own stores go to.
template <typename T, int KB>
__device__ __forceinline__ bool warp_tagged_row(const SyncArgs &sy, const long long *src, long long ep64, T (&v)[KB],
                                                unsigned max_ns, long long who)
{
    constexpr int TW = Tag<T>::words;
    bool ok = true;
#pragma unroll
    for (int q = 0; q < KB; ++q) ok = get_tag(src + q * TW, ep64, &v[q]) && ok;
    if (__all_sync(0xffffffffu, ok)) return true;
    const long long t0 = global_ns();
    const long long *probe = reinterpret_cast<const long long *>(
                                 __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(src), 31)) +
                             (KB - 1) * TW;
    bool probing = true;  // warp-uniform: the probe phase, then the full-row phase
    unsigned ns = 16;
    for (unsigned it = 1;; ++it) {
        __nanosleep(ns);
        if (ns < max_ns) ns <<= 1;
        if (probing) {
            // every lane loads the same word: one request for the warp
            const bool out = (ld_relaxed_gpu(probe) & ~0xffffffffll) == ep64;
            if (__any_sync(0xffffffffu, out)) {
                probing = false;
                ns = 16;
            }
        }
        if (!probing) {
            if (!ok) {
                ok = true;
#pragma unroll
                for (int q = 0; q < KB; ++q) ok = get_tag(src + q * TW, ep64, &v[q]) && ok;
            }
            if (__all_sync(0xffffffffu, ok)) return true;
        }
        if ((it & 15u) == 0u) {
            int bad = 0;
            if ((threadIdx.x & 31) == 0) {
                if (aborted(sy)) {
                    bad = 1;
                } else if (global_ns() - t0 > sy.timeout_ns || it > (1u << 26)) {
                    record_error(sy, kStatusTimeout, who);
                    bad = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, bad, 0)) return false;
        }
    }
}

// Warp-wide bounded wait on a shared-memory counter (every lane polls; the
// verdict is lane 0's).  False if the block is stopping or the wait ran out.
__device__ __forceinline__ bool warp_seq_wait(const SyncArgs &sy, const volatile int *seq, int want,
                                              volatile int *stop, long long who)
{
    int ok = 1;
    if (*seq < want) {
        // spin on the counter (the producers are warps of this block, so the
        // wait is short and a sleep would only add its own granularity)
        const long long t0 = global_ns();
        for (unsigned it = 1;; ++it) {
            if (*seq >= want) break;
            if ((it & 1023u) == 0u) {
                if (*stop || aborted(sy)) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > sy.timeout_ns || it > (1u << 28)) {
                    if ((threadIdx.x & 31) == 0) record_error(sy, kStatusTimeout, who);
                    *stop = 1;
                    ok = 0;
                    break;
                }
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    __threadfence_block();
    return ok != 0;
}
__device__ __forceinline__ void warp_seq_post(volatile int *seq, int v)
{
    __syncwarp();
    __threadfence_block();
    if ((threadIdx.x & 31) == 0) *seq = v;
}

// mbarriers in shared memory (one arrival per lane of each producer warp):
// a waiting warp is suspended by the hardware instead of polling, so it
// takes no issue slots or shared-memory bandwidth from the working warps.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(unsigned long long *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
// Arrive once this thread's earlier cp.async copies have landed.
__device__ __forceinline__ void mb_arrive_cp(unsigned long long *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Warp-wide bounded wait for the phase of `bar` with this parity to complete.
__device__ __forceinline__ bool mb_wait(const SyncArgs &sy, unsigned long long *bar, unsigned parity,
                                        volatile int *stop, long long who)
{
    bool ok = mb_try_wait(bar, parity);
    if (!__all_sync(0xffffffffu, ok)) {
        const long long t0 = global_ns();
        for (unsigned it = 1;; ++it) {
            ok = ok || mb_try_wait(bar, parity);
            if (__all_sync(0xffffffffu, ok)) break;
            if ((it & 15u) == 0u) {
                int bad = 0;
                if ((threadIdx.x & 31) == 0) {
                    if (*stop || aborted(sy)) {
                        bad = 1;
                    } else if (global_ns() - t0 > sy.timeout_ns || it > (1u << 26)) {
                        record_error(sy, kStatusTimeout, who);
                        *stop = 1;
                        bad = 1;
                    }
                }
                if (__shfl_sync(0xffffffffu, bad, 0)) return false;
            }
        }
    }
    return true;
}

// One entry of a block's Gram, sum over its 32 rows of P_iq P_ir, for the
// prefix Grams (in double).  From double P: fused multiply-adds in double.
// From float P (the mixed path) the FP64 rate, not the data, would bound a
// single warp at one FP64 instruction per 64 cycles, so the sum is formed
// on the FP32 pipes with no rounding lost: each product splits exactly into
// hi + lo (hi = fl(a b), lo = fma(a, b, -hi)), the hi parts are summed with
// Neumaier's compensation (the running sum s and its error c), the lo parts
// in float (each below 2^-24 of its product), and s, c and the lo sum are
// added in double: an error of about 32 u^2 of the sum of |a b| (u = 2^-24),
// against about 32 u_d = 2^-48 of it for a sum in double.
__device__ __forceinline__ double gram_entry(const double *pm, int KS, int q, int r)
{
    double s0 = 0.0, s1 = 0.0;
#pragma unroll 8
    for (int i = 0; i < kB; i += 2) {
        s0 = fma(pm[i * KS + q], pm[i * KS + r], s0);
        s1 = fma(pm[(i + 1) * KS + q], pm[(i + 1) * KS + r], s1);
    }
    return s0 + s1;
}
__device__ __forceinline__ double gram_entry(const float *pm, int KS, int q, int r)
{
    float s = 0.f, c = 0.f, l = 0.f;
#pragma unroll 8
    for (int i = 0; i < kB; ++i) {
        // the _rn intrinsics keep the compiler from fusing these operations
        const float a = pm[i * KS + q], b = pm[i * KS + r];
        const float hi = __fmul_rn(a, b);
        const float lo = fmaf(a, b, -hi);
        const float t = __fadd_rn(s, hi);
        c = __fadd_rn(c, fabsf(s) >= fabsf(hi) ? __fadd_rn(__fsub_rn(s, t), hi) : __fadd_rn(__fsub_rn(hi, t), s));
        s = t;
        l = __fadd_rn(l, lo);
    }
    return (double)s + ((double)c + (double)l);
}

// Warps of the forward-substitution kernel and the chain block's roles: the
// critical warp, the W warp, seven near warps, the far-sum stager, the
// loader, two publishers (even and odd blocks: the fence that orders a
// block's values before its flag costs about a chain step) and, in a fused
// pass, the warp that forms the prefix Grams.
constexpr int kTrsmWarps = 14;
constexpr int kWCrit = 0, kWZhat = 1, kWNear0 = 2;
constexpr int kNearWarps = 7;  // warps 2 .. 8
constexpr int kWZf = 9, kWLoad = 10, kWPub = 11, kWPub2 = 12, kWH = 13;

// Lookahead bound (d), offsets on the critical warp (c) and ring depths per
// instantiation, sized to the 227 KB of shared memory.
template <typename T, int KB>
struct ChainCfg {
    static constexpr int DMAX = sizeof(T) == 4 ? (KB <= 2 ? 10 : KB <= 4 ? 9 : KB <= 8 ? 8 : 6)
                                               : (KB <= 2 ? 6 : KB <= 8 ? 4 : 3);
    static constexpr int CMAX = sizeof(T) == 4 ? (KB <= 2 ? 4 : KB <= 8 ? 2 : 1) : 1;
    static constexpr int RP = DMAX + 2;   // P ring
    static constexpr int RT = DMAX;       // per near offset
    static constexpr int RZ = 4;          // W ring
    static constexpr int RF = 4;          // far-sum ring
    static constexpr int RH = 4;          // prefix-Gram ring (fused passes)
    static constexpr size_t tile = sizeof(T) * kB * Stride<T>::value;
    static constexpr int NEAR = DMAX - CMAX > 1 ? DMAX - CMAX : 1;  // near offset slots (d - c of them used)
    static constexpr size_t rest = sizeof(T) * Rows<T, KB>::size *
                                       ((size_t)RP + (size_t)NEAR * RT + RZ + RF + 1) +
                                   256 + (size_t)RH * KB * KB * sizeof(double);
    // staged per step: G^(1..c) on the loader, one tile per near offset on the near warps
    static constexpr size_t stage = (size_t)(CMAX + NEAR) * tile;
    static constexpr int fit = (int)((224u * 1024u - rest) / stage);
    static constexpr int RS = fit > 4 ? 4 : fit;
};

template <typename T, int KB>
struct ChainSmem {
    using C = ChainCfg<T, KB>;
    static constexpr int S = Stride<T>::value;
    static constexpr int RW = Rows<T, KB>::size;
    T G[C::RS][C::CMAX][kB * S];          // G^(j)_m, j = 1 .. c, of step m
    T near[C::NEAR][C::RS][kB * S];       // per near offset: tiles (m, m + j), [column][row]
    T P[C::RP][RW];
    T Tn[C::NEAR][C::RT][RW];             // F_{b-j,b}^T P_{b-j} per near offset j
    T Z[C::RZ][RW];                       // W_b
    T F[C::RF][RW];                       // far sums Zf_b
    T w[RW];                              // the W warp's work vector
    double Hr[C::RH][KB * KB];            // prefix Grams H_m on their way to the publisher
    // full / empty rings: stage (G, Dinv), W, P, far sums; near warps' steps
    unsigned long long st_full[C::RS], st_empty[C::RS];
    unsigned long long w_full[C::RZ], w_empty[C::RZ];
    unsigned long long p_full[C::RP], p_empty[C::RP];
    unsigned long long f_full[C::RF], f_empty[C::RF];
    unsigned long long t_full[kNearWarps][C::RT];
    unsigned long long h_full[C::RH], h_empty[C::RH];
    int stop;
};

// The chain block: every role is one warp, linked by mbarrier rings (full /
// empty per resource slot; an item m uses slot m % R with phase parity
// (m / R) & 1, and no producer can lap a consumer by construction).  With
// G^(j)_m = Dinv_m F_{m-j,m}^T for the d nearest offsets,
//   P_m = W_m - sum_{j=1}^{c} G^(j)_m P_{m-j},
//   W_m = Dinv_m Zf_m - sum_{j=c+1}^{d} G^(j)_m P_{m-j},
// so the critical warp's step waits on no other warp's work of the last c
// steps: the near warps (offsets c + 1 .. d) and the W warp have c steps of
// slack, and the W warp, whose far part Dinv_m Zf_m the workers post, only
// subtracts.  The loader stages G^(1..c) (its copies arrive on the stage's
// barrier when they land) and prefetches Dinv to L2, from where the W warp
// loads its row of it for the first d + 1 blocks, each near warp stages its
// own G^(j), the far-sum warp polls the workers' tagged sums ahead of use,
// the publisher writes each P as tagged words.
template <typename T, int KB>
__device__ void trsm_chain(const Args<T> &A, unsigned char *smem)
{
    using C = ChainCfg<T, KB>;
    ChainSmem<T, KB> &S = *reinterpret_cast<ChainSmem<T, KB> *>(smem);
    constexpr int TW = Tag<T>::words;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = A.nb, d = A.d, cc = A.c;
    const long long n = A.n, ld = A.ld;
    const long long ep64 = (long long)A.epoch << 32;
    const SyncArgs sy = sync_of(A);
    volatile int *stop = &S.stop;
    const bool vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
    const int nnear = d - cc;  // near offsets j = c + 1 .. d, offset j on near warp (j - c - 1) % kNearWarps
    const int nnw = nnear < kNearWarps ? nnear : kNearWarps;  // near warps in use
    if (threadIdx.x == 0) {
        for (int i = 0; i < C::RS; ++i) {
            mb_init(&S.st_full[i], 32);
            mb_init(&S.st_empty[i], 32);  // the critical warp
        }
        for (int i = 0; i < C::RZ; ++i) {
            mb_init(&S.w_full[i], 32);
            mb_init(&S.w_empty[i], 32);
        }
        for (int i = 0; i < C::RP; ++i) {
            mb_init(&S.p_full[i], 32);
            // the publisher, the near warps and, in a fused pass, the H warp
            mb_init(&S.p_empty[i], 32 * (1 + nnw + (A.fused ? 1 : 0)));
        }
        for (int i = 0; i < C::RF; ++i) {
            mb_init(&S.f_full[i], 32);
            mb_init(&S.f_empty[i], 32);
        }
        for (int t = 0; t < kNearWarps; ++t)
            for (int i = 0; i < C::RT; ++i) mb_init(&S.t_full[t][i], 32);
        for (int i = 0; i < C::RH; ++i) {
            mb_init(&S.h_full[i], 32);
            mb_init(&S.h_empty[i], 32);
        }
        S.stop = 0;
    }
    __syncthreads();
#define MW(bar, item, ring, who)                                                               \
    do {                                                                                       \
        if (!mb_wait(sy, &(bar)[(item) % (ring)], (unsigned)(((item) / (ring)) & 1), stop, (who))) { \
            cp_wait<0>();                                                                      \
            return;                                                                            \
        }                                                                                      \
    } while (0)

    // Publication of P: the blocks m = first, first + step, ... are stored
    // plainly (for the kernels after this one) and as epoch-tagged words for
    // the readers within this launch, which take a word once it carries this
    // pass's epoch; no fence is needed (a fence waits for the stores to be
    // acknowledged, which under the sweep's and the workers' traffic costs
    // several chain steps).
    auto publish = [&](int first, int step) {
        for (int m = first; m < nb; m += step) {
            MW(S.p_full, m, C::RP, m);
            T v[KB];
            row_load<T, KB>(S.P[m % C::RP], lane, v);
            __syncwarp();
            mb_arrive(&S.p_empty[m % C::RP]);
            T *plain = A.P + ((size_t)m * kB + lane) * KB;
            long long *tag = A.Ptag + ((size_t)m * kB + lane) * KB * TW;
#pragma unroll
            for (int q = 0; q < KB; ++q) {
                __stcg(plain + q, v[q]);
                put_tag(tag + q * TW, v[q], ep64);
            }
            if (A.fused) {
                // H_m from the H warp, as tagged doubles
                MW(S.h_full, m, C::RH, m);
                long long *hg = A.Htag + (size_t)m * KB * KB * 2;
                for (int e = lane; e < KB * KB; e += 32) put_tagged(hg + 2 * e, S.Hr[m % C::RH][e], ep64);
                __syncwarp();
                mb_arrive(&S.h_empty[m % C::RH]);
            }
            if (A.trace && lane == 0) A.trace[(size_t)m * 16 + 4] = global_ns();
        }
    };

    // Fused pass: the prefix Grams H_m = Sigma + sum_{i < m} P_i^T P_i (in
    // double; the padding vectors' entries an identity) for the workers'
    // coefficient tasks, handed to the publisher through a shared-memory
    // ring and released with P_m under the publisher's one fence per block.
    auto hwarp = [&]() {
        constexpr int NE = KB * KB, NL = (NE + 31) / 32;
        constexpr int KS = Rows<T, KB>::KS;
        double h[NL];
#pragma unroll
        for (int u = 0; u < NL; ++u) {
            const int e = lane + 32 * u, q = e / KB, r = e % KB;
            h[u] = (e < NE && q == r) ? (q < A.kr ? sigma_of(A, q) : 1.0) : 0.0;
        }
        for (int m = 0; m < nb; ++m) {
            // H_m (it needs only the blocks before m) to the publisher first
            if (m >= C::RH) MW(S.h_empty, m - C::RH, C::RH, m);
            double *hs = S.Hr[m % C::RH];
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int e = lane + 32 * u;
                if (e < NE) hs[e] = h[u];
            }
            __syncwarp();
            mb_arrive(&S.h_full[m % C::RH]);
            // then block m's Gram into the running sum
            MW(S.p_full, m, C::RP, m);
            const T *pm = S.P[m % C::RP];
            double g[NL];
#pragma unroll
            for (int u = 0; u < NL; ++u) {
                const int e = lane + 32 * u, q = e / KB, r = e % KB;
                g[u] = 0.0;
                if (e < NE && q < A.kr && r < A.kr) g[u] = gram_entry(pm, KS, q, r);  // update vectors only
            }
            __syncwarp();
            mb_arrive(&S.p_empty[m % C::RP]);
#pragma unroll
            for (int u = 0; u < NL; ++u) h[u] += g[u];
        }
    };

    if (warp == kWLoad) {
        // G^(1..c) and Dinv of a step, prefetched to L2 16 steps ahead (the
        // copies into the stage ring, and the W warp's loads of Dinv, then
        // come from L2 while the workers stream the factor from HBM)
        constexpr int PF = 16;
        auto prefetch = [&](int m) {
            if (m >= nb) return;
            constexpr int LINE = 128 / (int)sizeof(T);  // elements per 128-byte line
            for (int j = 1; j <= cc && j <= m; ++j) {
                const T *g = A.G + ((size_t)(j - 1) * nb + m) * kB * kB;
                for (int e = lane * LINE; e < kB * kB; e += 32 * LINE) prefetch_l2(g + e);
            }
            if (m + 1 < nb) {
                const T *di = A.Dinv + (size_t)(m + 1) * kB * kB;
                for (int e = lane * LINE; e < kB * kB; e += 32 * LINE) prefetch_l2(di + e);
            }
        };
        for (int m = 0; m < PF; ++m) prefetch(m);
        for (int m = 0; m < nb; ++m) {
            prefetch(m + PF);
            const int st = m % C::RS;
            if (m >= C::RS) MW(S.st_empty, m - C::RS, C::RS, -10);
            if (A.trace && lane == 0) A.trace[(size_t)m * 16 + 3] = global_ns();
            for (int j = 1; j <= cc && j <= m; ++j)
                stage_dense(S.G[st][j - 1], A.G + ((size_t)(j - 1) * nb + m) * kB * kB, lane);
            mb_arrive_cp(&S.st_full[st]);
        }
        cp_wait<0>();
    } else if (warp == kWCrit) {
        for (int m = 0; m < nb; ++m) {
            MW(S.w_full, m, C::RZ, m);
            MW(S.st_full, m, C::RS, m);
            if (m >= C::RP) MW(S.p_empty, m - C::RP, C::RP, m);
            if (A.trace && lane == 0) A.trace[(size_t)m * 16 + 7] = global_ns();
            T out[KB], acc[KB];
#pragma unroll
            for (int q = 0; q < KB; ++q) acc[q] = T(0);
            for (int j = 1; j <= cc && j <= m; ++j)
                lane_mv<T, KB>(S.G[m % C::RS][j - 1], S.P[(m - j) % C::RP], acc, lane, true);
            row_load<T, KB>(S.Z[m % C::RZ], lane, out);
#pragma unroll
            for (int q = 0; q < KB; ++q) out[q] -= acc[q];
            row_store<T, KB>(S.P[m % C::RP], lane, out);
            __syncwarp();
            mb_arrive(&S.p_full[m % C::RP]);
            mb_arrive(&S.w_empty[m % C::RZ]);
            mb_arrive(&S.st_empty[m % C::RS]);
            if (A.trace && lane == 0) A.trace[(size_t)m * 16 + 0] = global_ns();
        }
    } else if (warp >= kWNear0 && warp < kWNear0 + kNearWarps) {
        const int t = warp - kWNear0;
        if (t >= nnw) return;
        // this warp's offsets' matrices G^(j)_b = Dinv_b F_{m,b}^T (b = m + j,
        // formed by prep_kernel from the factor as it entered the pass), staged
        // RS - 1 steps ahead: the running sums are then Dinv_b times the near
        // part, and W_b needs no product with Dinv_b on this block
        auto stage = [&](int m) {
            if (m < nb) {
                for (int j = cc + 1 + t; j <= d; j += kNearWarps) {
                    const int b = m + j;
                    if (b >= nb) break;
                    stage_dense(S.near[j - cc - 1][m % C::RS], A.G + ((size_t)(j - 1) * nb + b) * kB * kB, lane);
                }
            }
            cp_commit();
        };
        // and, further ahead, the same matrices into L2
        auto prefetch = [&](int m) {
            if (m >= nb) return;
            constexpr int LINE = 128 / (int)sizeof(T);  // elements per 128-byte line
            for (int j = cc + 1 + t; j <= d; j += kNearWarps) {
                const int b = m + j;
                if (b >= nb) break;
                const T *g = A.G + ((size_t)(j - 1) * nb + b) * kB * kB;
                for (int e = lane * LINE; e < kB * kB; e += 32 * LINE) prefetch_l2(g + e);
            }
        };
        constexpr int PF = 16;
        for (int m = 0; m < PF; ++m) prefetch(m);
        for (int m = 0; m < C::RS - 1; ++m) stage(m);
        for (int m = 0; m < nb; ++m) {
            prefetch(m + PF);
            stage(m + C::RS - 1);
            MW(S.p_full, m, C::RP, m);
            cp_wait<C::RS - 1>();
            __syncwarp();
            const T *pm = S.P[m % C::RP];
            for (int j = cc + 1 + t; j <= d; j += kNearWarps) {
                const int b = m + j;
                if (b >= nb) break;
                T out[KB];
                lane_mv<T, KB>(S.near[j - cc - 1][m % C::RS], pm, out, lane);
                // the running sum of block b's near terms, offsets d, d - 1, ..., j:
                // offset j + 1's warp left the terms above in its slot at step m - 1
                if (j < d && j + 1 <= b) {
                    MW(S.t_full[(j - cc) % kNearWarps], m - 1, C::RT, b);
                    T up[KB];
                    row_load<T, KB>(S.Tn[j - cc][b % C::RT], lane, up);
#pragma unroll
                    for (int q = 0; q < KB; ++q) out[q] += up[q];
                }
                row_store<T, KB>(S.Tn[j - cc - 1][b % C::RT], lane, out);
            }
            __syncwarp();
            mb_arrive(&S.p_empty[m % C::RP]);
            mb_arrive(&S.t_full[t][m % C::RT]);
            if (A.trace && t == 0 && lane == 0) A.trace[(size_t)m * 16 + 5] = global_ns();
            if (A.trace && t == nnw - 1 && lane == 0) A.trace[(size_t)m * 16 + 12] = global_ns();
        }
    } else if (warp == kWZhat) {
        T *wv = S.w;
        // W_b = Dinv_b Zf_b - sum_{j=c+1}^{d} G^(j)_b P_{b-j}: the workers post
        // Dinv_b Zf_b and the near warps' running sum holds the G terms, so
        // the warp only subtracts.  The first d + 1 blocks have no far part:
        // W_b = Dinv_b V_b - (near terms), with row `lane` of Dinv_b loaded
        // from L2 (the loader prefetched it) before the warp waits
        T drow[kB];
        auto load_drow = [&](int b) {
            using V = typename Vec16<T>::type;
            constexpr int E = Vec16<T>::n;
            const V *src = reinterpret_cast<const V *>(A.Dinv + (size_t)b * kB * kB + (size_t)lane * kB);
#pragma unroll
            for (int c = 0; c < kB / E; ++c) {
                const V x = __ldcg(src + c);
#pragma unroll
                for (int u = 0; u < E; ++u) drow[c * E + u] = vget<T>(x, u);
            }
        };
        load_drow(0);
        for (int b = 0; b < nb; ++b) {
            const long long r0 = (long long)b * kB;
            T w[KB];
            if (b > d) {
                MW(S.f_full, b - d - 1, C::RF, b);
                if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 10] = global_ns();
                row_load<T, KB>(S.F[(b - d - 1) % C::RF], lane, w);
                __syncwarp();
                mb_arrive(&S.f_empty[(b - d - 1) % C::RF]);
            } else {
#pragma unroll
                for (int q = 0; q < KB; ++q) w[q] = vin(A, sy, r0 + lane, q);
                row_store<T, KB>(wv, lane, w);
                __syncwarp();
                lane_mv_reg<T, KB>(drow, wv, w);
                __syncwarp();
                if (b + 1 <= d && b + 1 < nb) load_drow(b + 1);
            }
            if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 6] = global_ns();
            if (cc + 1 <= d && cc + 1 <= b) {
                // the near terms, summed by the near warps (offset c + 1 holds all of them)
                MW(S.t_full[0], b - cc - 1, C::RT, b);
                T tn[KB];
                row_load<T, KB>(S.Tn[0][b % C::RT], lane, tn);
#pragma unroll
                for (int q = 0; q < KB; ++q) w[q] -= tn[q];
            }
            if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 11] = global_ns();
            // W_{b - RZ}'s slot is free once the critical warp has used it
            if (b >= C::RZ) MW(S.w_empty, b - C::RZ, C::RZ, b);
            row_store<T, KB>(S.Z[b % C::RZ], lane, w);
            __syncwarp();
            mb_arrive(&S.w_full[b % C::RZ]);
            if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 1] = global_ns();
        }
    } else if (warp == kWZf) {
        for (int b = d + 1; b < nb; ++b) {
            const int k = b - d - 1;
            if (k >= C::RF) MW(S.f_empty, k - C::RF, C::RF, b);
            const long long *src = A.Ztag + ((size_t)b * kB + lane) * KB * TW;
            T v[KB];
            const long long t0 = global_ns();
            unsigned ns = 32;
            for (unsigned it = 0;; ++it) {
                bool ok = true;
#pragma unroll
                for (int q = 0; q < KB; ++q) ok = get_tag(src + q * TW, ep64, &v[q]) && ok;
                if (__all_sync(0xffffffffu, ok)) break;
                if ((it & 15u) == 15u) {
                    int bad = 0;
                    if (lane == 0) {
                        if (*stop || aborted(sy)) bad = 1;
                        else if (global_ns() - t0 > sy.timeout_ns || it > (1u << 26)) {
                            record_error(sy, kStatusTimeout, b);
                            *stop = 1;
                            bad = 1;
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) return;
                }
                __nanosleep(ns);
                if (ns < 128) ns <<= 1;
            }
            row_store<T, KB>(S.F[k % C::RF], lane, v);
            __syncwarp();
            mb_arrive(&S.f_full[k % C::RF]);
            if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 2] = global_ns();
        }
    } else if (warp == kWPub || warp == kWPub2) {
        publish(warp == kWPub ? 0 : 1, 2);
    } else if (warp == kWH) {
        if (A.fused) hwarp();
    }
#undef MW
}

// Worker warps: the far part of column block b's sum,
//   Zf_b = V_b - sum_{r < b - d} F_{r,b}^T P_r,
// tiles staged a few ahead (they are the factor as it entered the pass), each
// P_r polled as tagged words, Dinv_b Zf_b published as tagged words.
template <typename T, int KB>
struct WorkerCfg {
    // staged tiles per warp: five in float, where a worker that falls a few
    // tiles behind the chain must catch up before its column is due
    // (n = 32768: rank 1 1.48 ms with 3, 1.40 with 4, 1.31 with 5, 1.40 with
    // 6, which leaves fewer workers than columns; 4 vectors per pass 2.06 /
    // 1.89 / 1.87 ms with 3 / 4 / 5; rank 16 7.8 / 6.8 / 6.6; rank 64
    // 31.1 / 26.1 / 25.0); in float64 three, which keeps a worker per column
    // (four: rank 1 5.46 against 4.51 ms)
    static constexpr int NS = sizeof(T) == 4 ? 5 : 3;
    // tiles prefetched to L2 ahead of the one in use: about 32 KB per warp,
    // 32 MB over a thousand workers at the front of the chain
    static constexpr int PF = (int)(32768 / (sizeof(T) * kB * kB));
    static constexpr size_t warp_bytes = sizeof(T) * ((size_t)NS * kB * Stride<T>::value + Rows<T, KB>::size);
    static constexpr int warps = (int)((200u * 1024u) / warp_bytes) < kTrsmWarps
                                     ? (int)((200u * 1024u) / warp_bytes) : kTrsmWarps;
};

// Returns true once the far-sum tasks are all taken (a fused pass's worker
// then takes coefficient and sweep tasks), false if the launch is aborting.
template <typename T, int KB>
__device__ bool trsm_workers(const Args<T> &A, unsigned char *smem)
{
    using W = WorkerCfg<T, KB>;
    constexpr int SD = Stride<T>::value;
    constexpr int TW = Tag<T>::words;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= W::warps) return false;
    T *base = reinterpret_cast<T *>(smem + (size_t)warp * W::warp_bytes);
    T *Pr = base + (size_t)W::NS * kB * SD;  // Rows<T, KB>
    const long long n = A.n, ld = A.ld;
    const int nb = A.nb, d = A.d;
    const long long ep64 = (long long)A.epoch << 32;
    const SyncArgs sy = sync_of(A);
    const bool vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = ld_relaxed_gpu(A.ctl + kCtlAbort) ? -1 : atomicAdd(A.ctl + kCtlWorkTicket, 1);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk < 0) return false;
        const int b = d + 1 + tk;
        if (b >= nb) return true;
        const long long c0 = (long long)b * kB;
        const bool col_ok = c0 + lane < n;
        T z[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q)
            z[q] = col_ok ? vin(A, sy, c0 + lane, q) : T(0);
        const int nfar = b - d;
        for (int r = 0; r < W::NS - 1 && r < nfar; ++r) {
            stage_tile(sy, base + (size_t)(r % W::NS) * kB * SD, A.L, ld, (long long)r * kB, c0, n, kB, vec, lane);
            cp_commit();
        }
        for (int r = 0; r < nfar; ++r) {
            if (r > 0 && r % A.seg == 0) {
                // a sweep segment boundary: the residual before row block r
                T *sn = A.snap + (((size_t)(r / A.seg - 1) * nb + b) * kB + lane) * KB;
#pragma unroll
                for (int q = 0; q < KB; ++q) sn[q] = z[q];
                if (A.fused) {
                    // tiles 0 .. r - 1 are read and the residual is out: the
                    // sweep may now rewrite the tiles of the segment that ends here
                    __syncwarp();
                    if (lane == 0) {
                        __threadfence();
                        st_release_gpu(A.wprog + b, ep64 + r);
                    }
                }
            }
            const int rn = r + W::NS - 1;
            if (rn < nfar)
                stage_tile(sy, base + (size_t)(rn % W::NS) * kB * SD, A.L, ld, (long long)rn * kB, c0, n, kB, vec, lane);
            cp_commit();
            // the tile W::PF ahead into L2, so that its staging a few steps
            // later waits on L2 rather than on HBM (a worker keeps up with
            // the chain only if a tile arrives within a chain step or two)
            if (r + W::PF < nfar) {
                const long long off = (long long)(r + W::PF) * kB + (c0 + lane) * ld;
                if (col_ok && CHK_TRI(sy, off, n, ld) && CHK_TRI(sy, off + kB - 1, n, ld)) {
                    prefetch_l2n(A.L + off);
                    if (sizeof(T) * kB > 128) prefetch_l2n(A.L + off + 128 / sizeof(T));
                }
            }
            // P_r: every lane takes its row as tagged words, polling until
            // all carry this pass's epoch (often only near the block's last
            // tiles: the far sum is due when the chain reaches b - d, and a
            // worker further back catches up in one burst)
            T pv[KB];
            if (!warp_tagged_row<T, KB>(sy, A.Ptag + ((size_t)r * kB + lane) * KB * TW, ep64, pv,
                                        r + 4 >= nfar ? 64u : 1024u, b)) {
                cp_wait<0>();
                return false;
            }
            row_store<T, KB>(Pr, lane, pv);
            if (A.trace && lane == 0 && r == nfar - 1) A.trace[(size_t)b * 16 + 8] = global_ns();
            cp_wait<W::NS - 1>();
            __syncwarp();
            T t[KB];
            lane_mv<T, KB>(base + (size_t)(r % W::NS) * kB * SD, Pr, t, lane);
#pragma unroll
            for (int q = 0; q < KB; ++q) z[q] -= t[q];
            __syncwarp();
        }
        // post Dinv_b Zf_b (the chain block's W warp then only subtracts):
        // Dinv_b staged into a free tile slot, Zf_b into the P row buffer
        stage_dense(base, A.Dinv + (size_t)b * kB * kB, lane);
        cp_commit();
        row_store<T, KB>(Pr, lane, z);
        cp_wait<0>();
        __syncwarp();
        lane_mv<T, KB>(base, Pr, z, lane);
        __syncwarp();
        long long *zt = A.Ztag + ((size_t)b * kB + lane) * KB * TW;
#pragma unroll
        for (int q = 0; q < KB; ++q) put_tag(zt + q * TW, z[q], ep64);
        if (A.trace && lane == 0) A.trace[(size_t)b * 16 + 9] = global_ns();
        if (A.fused) {
            // every tile of the far part read: the sweep's segments of this column may go
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                st_release_gpu(A.wprog + b, ep64 + nfar);
            }
        }
    }
}



// ---------------------------------------------------------------- Compute

// gram[b] = sum over the rows of block b of p p^T (double), one warp per block.
template <typename T, int KB>
__global__ void __launch_bounds__(32) gram_kernel(Args<T> A)
{
    __shared__ double p[kB][KB];
    const int lane = threadIdx.x;
    if (!ws_ok<T, KB>(A, sync_of(A))) return;
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
    if (!ws_ok<T, KB>(A, sync_of(A))) return;
    const int len = (nb + 31) / 32;
    const int b0 = s * len, b1 = min(nb, b0 + len);
    const bool valid = e < KB * KB;
    double sum = 0.0;
    if (valid) {
#pragma unroll 8
        for (int b = b0; b < b1; ++b) sum += __ldcg(A.gram + (size_t)b * KB * KB + e);
    }
    seg[s][threadIdx.x & 31] = sum;
    __syncthreads();
    double pre = 0.0;
    if (valid) {
        const int q = e / KB, r = e % KB;
        pre = (q == r) ? sigma_of(A, q) : 0.0;
        if (q >= A.kr || r >= A.kr) pre = (q == r) ? 1.0 : 0.0;  // padding and right-hand sides: identity
        for (int s2 = 0; s2 < s; ++s2) pre += seg[s2][threadIdx.x & 31];
        for (int b = b0; b < b1; ++b) {
            A.H[(size_t)b * KB * KB + e] = pre;
            pre += A.gram[(size_t)b * KB * KB + e];
        }
    }
}

// Per row block b (one warp, lane = row r0 + lane), every row on its own:
// its prefix Gram H_r = H_b + sum_{i < r in the block} p_i p_i^T (an
// in-place prefix over the block's rows in shared memory, packed lower
// triangles), then H_r = L D L^T (L unit lower), z = L^{-1} p_r, and with
// |D_q| = sigma_q D_q (the factor of H_r = U Sigma U^T is U = L |D|^{1/2},
// so y_q = z_q / |D_q|^{1/2} and t_q = |D_q|^{1/2}):
//   Dc_q = 1 + sum_{q' <= q} sigma_q' z_q'^2 / |D_q'|,
//   a_q = sigma_q z_q,   b_q = z_q / (|D_q| Dc_q),
//   e = Dc_kb^{-1/2},    the diagonal factor Dc_kb^{1/2}.
// All in double.  A pivot of the wrong sign or a non-positive Dc is the
// Compute step's failure (the modified matrix is not positive definite).
template <int KB>
struct Packed {
    static constexpr int entries = KB * (KB + 1) / 2;
    static constexpr int stride = entries | 1;  // odd: the lanes' rows fall in distinct banks
    static constexpr size_t smem = sizeof(double) * (kB + 1) * stride;
};
__device__ __forceinline__ int pidx(int i, int j) { return i * (i + 1) / 2 + j; }  // j <= i

// One row block's coefficients (one warp); Hs: Packed<KB>::smem bytes of
// shared memory.  P and H are read through L2 (a fused pass's workers read
// what other SMs wrote during the launch).
template <typename T, int KB>
__device__ bool coef_block(const Args<T> &A, const SyncArgs &sy, int b, double *Hs, bool tagged)
{
    using PK = Packed<KB>;
    constexpr int NE = PK::entries, HS = PK::stride;
    const int lane = threadIdx.x & 31;
    const long long n = A.n;
    const int kb = A.kr;  // the update vectors (right-hand sides take no part in the Compute)
    const long long r0 = (long long)b * kB;
    const int rows = (int)min((long long)kB, n - r0);
    double p[KB];
    if (tagged) {
        // P_b and H_b as the chain block publishes them within the launch
        constexpr int TW = Tag<T>::words;
        const long long ep64 = (long long)A.epoch << 32;
        T pv[KB];
        if (!warp_tagged_row<T, KB>(sy, A.Ptag + (size_t)(r0 + lane) * KB * TW, ep64, pv, 256u, b)) return false;
#pragma unroll
        for (int q = 0; q < KB; ++q) p[q] = (q < kb) ? (double)pv[q] : 0.0;
        for (int e0 = 0; e0 < NE; e0 += 32) {
            const int e = e0 + lane;
            double v = 0.0;
            bool ok = true;
            if (e < NE) {
                int i = 0;
                while ((i + 1) * (i + 2) / 2 <= e) ++i;
                const long long *w = A.Htag + ((size_t)b * KB * KB + i * KB + (e - i * (i + 1) / 2)) * 2;
                ok = get_tagged(w, ep64, &v);
                const long long t0 = ok ? 0 : global_ns();
                for (unsigned it = 0; !ok; ++it) {
                    __nanosleep(128);
                    ok = get_tagged(w, ep64, &v);
                    if (!ok && (it & 255u) == 255u) {
                        if (aborted(sy)) break;
                        if (global_ns() - t0 > sy.timeout_ns || it > (1u << 26)) {
                            record_error(sy, kStatusTimeout, b);
                            break;
                        }
                    }
                }
            }
            if (!__all_sync(0xffffffffu, ok)) return false;
            if (e < NE) Hs[e] = v;
        }
    } else {
        const T *prow = A.P + (size_t)(r0 + lane) * KB;
#pragma unroll
        for (int q = 0; q < KB; ++q) p[q] = (q < kb) ? (double)__ldcg(prow + q) : 0.0;
        // row 0: H_b; row lane + 1: this lane's outer product
        const double *hb = A.H + (size_t)b * KB * KB;
        for (int e = lane; e < NE; e += 32) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            Hs[e] = __ldcg(hb + i * KB + (e - i * (i + 1) / 2));
        }
    }
    double *mine = Hs + (size_t)(lane + 1) * HS;
#pragma unroll
    for (int i = 0; i < KB; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) mine[pidx(i, j)] = p[i] * p[j];
    __syncwarp();
    for (int e = lane; e < NE; e += 32) {
        double acc = Hs[e];
        for (int r = 1; r <= kB; ++r) {
            acc += Hs[(size_t)r * HS + e];
            Hs[(size_t)r * HS + e] = acc;
        }
    }
    __syncwarp();
    // this row's H (the prefix before it): row `lane`
    double *h = Hs + (size_t)lane * HS;
    for (int j = 0; j < kb; ++j) {
        double dj = h[pidx(j, j)];
        for (int m = 0; m < j; ++m) dj -= h[pidx(j, m)] * h[pidx(j, m)] * h[pidx(m, m)];
        h[pidx(j, j)] = dj;
        const double idj = rcp_refined(dj);
        for (int i = j + 1; i < kb; ++i) {
            double t = h[pidx(i, j)];
            for (int m = 0; m < j; ++m) t -= h[pidx(i, m)] * h[pidx(j, m)] * h[pidx(m, m)];
            h[pidx(i, j)] = t * idj;
        }
    }
    // at a sweep segment boundary, the prefix Gram's LDL^T before the block
    if (lane == 0 && b > 0 && b % A.seg == 0) {
        double *dst = A.rst + (size_t)(b / A.seg - 1) * (KB * (KB + 1) / 2);
        for (int e = 0; e < NE; ++e) dst[e] = h[e];
    }
    // z = L^{-1} p and the coefficients
    double z[KB];
    double Dc = 1.0;
    bool bad = false;
    T *cf = A.coef + (size_t)(r0 + lane) * 2 * KB;
#pragma unroll
    for (int q = 0; q < KB; ++q) {
        if (q < kb) {
            double zq = p[q];
#pragma unroll
            for (int m = 0; m < q; ++m) zq -= h[pidx(q, m)] * z[m];
            z[q] = zq;
            const double sg = sigma_of(A, q);
            const double ad = sg * h[pidx(q, q)];  // |D_q|
            bad = bad || !(ad > 0.0 && ad <= DBL_MAX);
            Dc = fma(sg * zq, zq * rcp_refined(ad), Dc);
            bad = bad || !(Dc > 0.0 && Dc <= DBL_MAX);
            if (lane < rows) {
                cf[2 * q] = (T)(sg * zq);
                cf[2 * q + 1] = (T)(zq * rcp_refined(ad * Dc));
            }
        } else {
            z[q] = 0.0;
            if (lane < rows) {
                cf[2 * q] = T(0);
                cf[2 * q + 1] = T(0);
            }
        }
    }
    const double rD = rsqrt_refined(Dc);
    if (lane < rows) {
        A.escale[r0 + lane] = (T)rD;
        A.dfac[r0 + lane] = Dc * rD;
        if (bad) record_error(sy, kStatusNotPD, r0 + lane);
    }
    __syncwarp();
    return true;
}

template <typename T, int KB>
__global__ void __launch_bounds__(32) coef_kernel(Args<T> A)
{
    extern __shared__ double Hs[];  // [kB + 1][HS]
    const SyncArgs sy = sync_of(A);
    if (!ws_ok<T, KB>(A, sy)) return;
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) coef_block<T, KB>(A, sy, b, Hs, false);
}

// ---------------------------------------------------------------- sweep

// Column block b, rows 0 .. b of the pass's Apply: lane = column, kb carries
// in registers, the column's 32 entries of a tile in registers during the
// recurrence; tiles and their rows' coefficients staged in a ring of NSLOT
// slots (cp.async), so that NSLOT - 1 tiles are in flight while one is used.
template <typename T, int KB>
struct SweepSlot {
    T tile[kB * Stride<T>::value];  // [column][row]
    T cf[kB * 2 * KB];              // (a, b) per row
    T e[kB];
    double df[kB];
};
template <typename T, int KB>
struct SweepCfg {
    static constexpr int WARPS = sizeof(T) == 4 ? 8 : 4;
    static constexpr int fit = (int)((224u * 1024u / WARPS) / sizeof(SweepSlot<T, KB>));
    static constexpr int NSLOT = fit > 6 ? 6 : (fit < 2 ? 2 : fit);
    static constexpr size_t smem = (size_t)WARPS * NSLOT * sizeof(SweepSlot<T, KB>);
};

// One tile's rotations for column `lane`: rows 0 .. 31 (all present), kb
// carries in registers, the row scales applied at the end.  The rows'
// coefficients come in 16-byte broadcast loads ahead of the dependent FMA
// chain (the only serial part: two FMAs per row and vector).
template <typename T, int KB>
__device__ __forceinline__ void rotate_full(T (&v)[kB], T (&uh)[KB], const T *cf, const T *e)
{
    using V = typename Vec16<T>::type;
    constexpr int E = Vec16<T>::n;
    constexpr int RW = 2 * KB;  // coefficients per row
#pragma unroll
    for (int i = 0; i < kB; ++i) {
        T c[RW];
        if ((RW * (int)sizeof(T)) % 16 == 0) {
#pragma unroll
            for (int g = 0; g < RW / E; ++g) {
                const V x = reinterpret_cast<const V *>(cf + i * RW)[g];
#pragma unroll
                for (int u = 0; u < E; ++u) c[g * E + u] = vget<T>(x, u);
            }
        } else {
#pragma unroll
            for (int u = 0; u < RW; ++u) c[u] = cf[i * RW + u];
        }
        T x = v[i];
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            x = fma(c[2 * q], uh[q], x);
            uh[q] = fma(-c[2 * q + 1], x, uh[q]);
        }
        v[i] = x;
    }
#pragma unroll
    for (int g = 0; g < kB / E; ++g) {
        const V x = reinterpret_cast<const V *>(e)[g];
#pragma unroll
        for (int u = 0; u < E; ++u) v[g * E + u] *= vget<T>(x, u);
    }
}

// Warp-wide bounded wait for a flag (== epoch) that another SM releases;
// lane 0 polls and acquires, the warp barrier orders the other lanes' later
// reads after it.  False if the launch is being aborted or the wait ran out.
__device__ __forceinline__ bool warp_flag(const SyncArgs &sy, const int *f, int epoch, long long who)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = wait_eq(sy, f, epoch, who) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}
__device__ __forceinline__ bool warp_count(const SyncArgs &sy, const long long *w, long long want, long long who)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = wait_ge(sy, w, want, who) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    return ok != 0;
}

// Per-lane addressing of column block b's tiles for the sweep: staging of
// a tile (rows r0 .. r0 + 31, the diagonal tile's rows <= column only) and
// of its rows' coefficients into a slot with cp.async, and the rotation of a
// staged tile (lane = column, the carries uh in registers) with its store.
template <typename T, int KB>
struct TileIO {
    static constexpr int SD = Stride<T>::value;
    static constexpr int E = 16 / (int)sizeof(T);
    static constexpr int CPC = kB / E;         // 16-byte chunks per column segment
    static constexpr int CPL = kB * CPC / 32;  // chunks per lane per tile
    using V = typename Vec16<T>::type;
    const Args<T> &A;
    const SyncArgs &sy;
    int b, lane, ch, col0, cstep;
    long long n, ld, c0, gofs;
    bool vec, active;
    const T *gbase;
    unsigned colmask;
    unsigned long long pol;
    __device__ TileIO(const Args<T> &a, const SyncArgs &s, int b_) : A(a), sy(s), b(b_)
    {
        lane = threadIdx.x & 31;
        n = A.n;
        ld = A.ld;
        vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
        // this lane's chunk of every staged column segment: chunk ch of columns
        // col0 + t * (32 / CPC), t = 0 .. CPL - 1
        ch = lane % CPC;
        col0 = lane / CPC;
        cstep = 32 / CPC;
        c0 = (long long)b * kB;
        active = c0 + lane < n;
        gofs = (long long)ch * E + (c0 + col0) * ld;
        gbase = A.L + gofs;
        colmask = 0;
#pragma unroll
        for (int t = 0; t < CPL; ++t)
            if (c0 + col0 + t * cstep < n) colmask |= 1u << t;
        pol = evict_first_policy();
    }
    __device__ void stage_tile(SweepSlot<T, KB> &sl, int r) const
    {
        const long long r0 = (long long)r * kB;
        if (r < b && vec) {
            const T *g = gbase + r0;
            T *d = sl.tile + col0 * SD + ch * E;
#pragma unroll
            for (int t = 0; t < CPL; ++t) {
                if ((colmask >> t & 1u) && CHK_TRI(sy, gofs + r0 + (long long)t * cstep * ld, n, ld) &&
                    CHK_TRI(sy, gofs + r0 + (long long)t * cstep * ld + E - 1, n, ld))
                    cp16_hint(d + t * cstep * SD, g + (long long)t * cstep * ld, pol);
                else {
#pragma unroll
                    for (int u = 0; u < E; ++u) d[t * cstep * SD + u] = T(0);
                }
            }
        } else if (r < b) {
            ::chm::pass::stage_tile(sy, sl.tile, A.L, ld, r0, c0, n, kB, false, lane);
        } else {
            // the diagonal tile: rows <= column only
            for (int col = 0; col < kB; ++col)
                if (c0 + col < n && lane <= col && CHK_TRI(sy, (r0 + lane) + (c0 + col) * ld, n, ld))
                    cp_elem(&sl.tile[col * SD + lane], A.L + (r0 + lane) + (c0 + col) * ld);
        }
    }
    __device__ void stage_coef(SweepSlot<T, KB> &sl, int r) const
    {
        const long long r0 = (long long)r * kB;
        const T *cf = A.coef + (size_t)r0 * 2 * KB;
        for (int c = lane; c < kB * 2 * KB / E; c += 32) cp16(sl.cf + c * E, cf + c * E);
        if (lane < kB / E) cp16(sl.e + lane * E, A.escale + r0 + lane * E);
        if (r == b && lane < kB / 2) cp16(sl.df + 2 * lane, A.dfac + r0 + 2 * lane);
    }
    __device__ void rotate_store(SweepSlot<T, KB> &sl, int r, T (&uh)[KB]) const
    {
        const bool diag = r == b;
        const long long r0 = (long long)r * kB;
        T v[kB];
        V *colv = reinterpret_cast<V *>(sl.tile + lane * SD);
#pragma unroll
        for (int c = 0; c < kB / E; ++c) {
            const V x = colv[c];
#pragma unroll
            for (int u = 0; u < E; ++u) v[c * E + u] = vget<T>(x, u);
        }
        if (!diag) {
            if (active) rotate_full<T, KB>(v, uh, sl.cf, sl.e);
        } else if (active) {
            // rows above the diagonal of column `lane`, then the diagonal
#pragma unroll
            for (int i = 0; i < kB; ++i) {
                if (i < lane) {
                    T x = v[i];
#pragma unroll
                    for (int q = 0; q < KB; ++q) {
                        x = fma(sl.cf[i * 2 * KB + 2 * q], uh[q], x);
                        uh[q] = fma(-sl.cf[i * 2 * KB + 2 * q + 1], x, uh[q]);
                    }
                    v[i] = x * sl.e[i];
                } else if (i == lane) {
                    v[i] = (T)((double)v[i] * sl.df[i]);
                }
            }
        }
        T *col = sl.tile + lane * SD;
#pragma unroll
        for (int c = 0; c < kB / E; ++c) {
            V x;
            T *xp = reinterpret_cast<T *>(&x);
#pragma unroll
            for (int u = 0; u < E; ++u) xp[u] = v[c * E + u];
            reinterpret_cast<V *>(col)[c] = x;
        }
        __syncwarp();
        if (!diag && vec) {
            T *g = const_cast<T *>(gbase) + r0;
            const T *d = sl.tile + col0 * SD + ch * E;
#pragma unroll
            for (int t = 0; t < CPL; ++t)
                if ((colmask >> t & 1u) && CHK_TRI(sy, gofs + r0 + (long long)t * cstep * ld, n, ld) &&
                    CHK_TRI(sy, gofs + r0 + (long long)t * cstep * ld + E - 1, n, ld))
                    st16_hint(reinterpret_cast<V *>(g + (long long)t * cstep * ld), *reinterpret_cast<const V *>(d + t * cstep * SD),
                              pol);
        } else {
#pragma unroll 8
            for (int cc = 0; cc < kB; ++cc)
                if (c0 + cc < n && (!diag || lane <= cc) && CHK_TRI(sy, (r0 + lane) + (c0 + cc) * ld, n, ld))
                    A.L[(r0 + lane) + (c0 + cc) * ld] = sl.tile[cc * SD + lane];
        }
        __syncwarp();
    }
};

// Segment sg of column block b: row blocks rb .. re (the last segment ends
// at the diagonal tile), tiles and their rows' coefficients staged through
// NSLOT slots.  In a fused pass the segment first waits until nothing else
// will read its tiles (the column's worker is past re, or for the last
// segment the chain has published P_b, which needs every near term of b),
// and each tile waits for its row block's coefficients.  Returns false if
// the launch is being aborted.
template <typename T, int KB, int NSLOT>
__device__ bool sweep_segment(const Args<T> &A, const SyncArgs &sy, int b, int sg, SweepSlot<T, KB> *slot)
{
    const int lane = threadIdx.x & 31;
    const long long n = A.n;
    const int nb = A.nb;
    const int nseg = 1 + max(0, (b - A.d - 1) / A.seg);
    if (b < 0 || b >= nb || sg < 0 || sg >= nseg) {
        // not a task of this pass (an internal invariant, checked in every build)
        if (lane == 0) record_error(sy, kStatusBounds, (long long)b);
        return false;
    }
    const int rb = sg * A.seg, re = sg == nseg - 1 ? b : rb + A.seg - 1;
    const long long ep64 = (long long)A.epoch << 32;
    if (A.fused) {
        // last segment: P_b out (its first tagged word) means the chain has
        // consumed every near term of column block b
        bool ok;
        if (sg == nseg - 1) {
            T pv[1];
            ok = warp_tagged_row<T, 1>(sy, A.Ptag + (size_t)b * kB * KB * Tag<T>::words, ep64, pv, 256u, b);
        } else {
            ok = warp_count(sy, A.wprog + b, ep64 + re + 1, b);
        }
        if (!ok) return false;
        if (sg > 0 && !warp_flag(sy, A.cflag + rb, A.epoch, b)) return false;  // its LDL^T at rb
    }
    const long long c0 = (long long)b * kB;
    const bool active = c0 + lane < n;
    T uh[KB];
    if (sg == 0) {
#pragma unroll
        for (int q = 0; q < KB; ++q)
            uh[q] = (active && q < A.kr) ? vin(A, sy, c0 + lane, q) : T(0);
    } else {
        // the carry entering row block rb, rebuilt from the substitution's
        // residual w there: u_hat = |D|^{-1} L^{-1} w with H = L D L^T the
        // prefix Gram before the block (the scaled rotations' carry is
        // this linear image of the residual at every row)
        const T *w = A.snap + (((size_t)(sg - 1) * nb + b) * kB + lane) * KB;
        const double *h = A.rst + (size_t)(sg - 1) * (KB * (KB + 1) / 2);
        double z[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            if (q < A.kr) {
                double zq = active ? (double)__ldcg(w + q) : 0.0;
#pragma unroll
                for (int m = 0; m < q; ++m) zq -= __ldcg(h + pidx(q, m)) * z[m];
                z[q] = zq;
                uh[q] = (T)(zq / (sigma_of(A, q) * __ldcg(h + pidx(q, q))));
            } else {
                z[q] = 0.0;
                uh[q] = T(0);
            }
        }
    }
    const TileIO<T, KB> io(A, sy, b);
    bool alive = true;
    auto fetch = [&](int r) {
        if (A.fused && alive) alive = warp_flag(sy, A.cflag + r, A.epoch, b);  // the row block's coefficients
        if (!alive) return;
        SweepSlot<T, KB> &sl = slot[r % NSLOT];
        io.stage_tile(sl, r);
        io.stage_coef(sl, r);
    };
    for (int r = rb; r < rb + NSLOT - 1; ++r) {
        if (r <= re) fetch(r);
        cp_commit();
    }
    for (int r = rb; r <= re; ++r) {
        if (r + NSLOT - 1 <= re) fetch(r + NSLOT - 1);
        cp_commit();
        cp_wait<NSLOT - 1>();
        __syncwarp();
        if (!alive) break;
        io.rotate_store(slot[r % NSLOT], r, uh);
    }
    cp_wait<0>();
    __syncwarp();
    return alive;
}

// The right-hand sides' column (chm_modify_solve).  Bordering A with B,
//   [[A, B], [B^T, c]] = [[F, Y], [0, g]]^T [[F, Y], [0, g]],  Y = F^{-T} B,
// and modifying the bordered matrix by V with zero rows below n leaves the
// border's column of the new factor at L~^{-T} B: the pass's rotations
// applied to Y as to one more column of the factor, with carries that start
// at zero (V has no entries there).  So after the substitution has carried
// B along (P's columns kr .. kb - 1 hold Y), this task runs the sweep's
// two-FMA recurrence down Y, row block by row block behind the chain, and
// writes L~^{-T} B over Y in P (read by the solve that follows the pass).
// One warp of a fused pass (the host carries right-hand sides only in
// fused passes); lane = right-hand side.  `sm`: Aug<T, KB>::bytes of shared
// memory.  Each row block waits for its coefficients and takes P_r as
// tagged words.  Returns false if the launch is being aborted.
template <typename T, int KB>
struct Aug {
    static constexpr int YS = KB + 1;  // row stride of the staged Y rows
    static constexpr size_t bytes = sizeof(T) * (size_t)kB * (YS + 2 * KB + 1);
};
template <typename T, int KB>
__device__ bool aug_task(const Args<T> &A, const SyncArgs &sy, T *sm)
{
    constexpr int YS = Aug<T, KB>::YS;
    constexpr int TW = Tag<T>::words;
    const int lane = threadIdx.x & 31;
    const int kr = A.kr, nr = A.kb - A.kr;
    const long long n = A.n;
    const long long ep64 = (long long)A.epoch << 32;
    T *Ys = sm;                      // [32][YS]: row i's P entries
    T *cf = Ys + kB * YS;            // [32][2 KB]: row i's (a_q, b_q)
    T *es = cf + kB * 2 * KB;        // [32]: row i's scale
    T uh[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) uh[q] = T(0);
    for (int r = 0; r < A.nb; ++r) {
        const long long r0 = (long long)r * kB;
        const int rows = (int)min((long long)kB, n - r0);
        T pv[KB];
        if (!warp_flag(sy, A.cflag + r, A.epoch, r)) return false;  // row block r's coefficients
        if (!warp_tagged_row<T, KB>(sy, A.Ptag + (size_t)(r0 + lane) * KB * TW, ep64, pv, 256u, r)) return false;
#pragma unroll
        for (int q = 0; q < KB; ++q) Ys[lane * YS + q] = pv[q];
        if (lane < rows) {
#pragma unroll
            for (int q = 0; q < 2 * KB; ++q) cf[lane * 2 * KB + q] = __ldcg(A.coef + (size_t)(r0 + lane) * 2 * KB + q);
            es[lane] = __ldcg(A.escale + r0 + lane);
        }
        __syncwarp();
        if (lane < nr) {
            for (int i = 0; i < rows; ++i) {
                T x = Ys[i * YS + kr + lane];
#pragma unroll
                for (int q = 0; q < KB; ++q) {
                    if (q < kr) {
                        x = fma(cf[i * 2 * KB + 2 * q], uh[q], x);
                        uh[q] = fma(-cf[i * 2 * KB + 2 * q + 1], x, uh[q]);
                    }
                }
                Ys[i * YS + kr + lane] = x * es[i];
            }
        }
        __syncwarp();
        if (lane < rows) {
            for (int q = kr; q < A.kb; ++q) A.P[(size_t)(r0 + lane) * KB + q] = Ys[lane * YS + q];
        }
        __syncwarp();
    }
    return true;
}

// The one task of the right-hand sides' column, if this pass carries any
// (and rotates anything): taken by the first warp that asks.
template <typename T, int KB>
__device__ __forceinline__ bool take_aug(const Args<T> &A)
{
    if (A.kb <= A.kr || A.kr == 0) return false;
    int t = 1;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(A.ctl + kCtlAugTicket, 1);
    return __shfl_sync(0xffffffffu, t, 0) == 0;
}

template <typename T, int KB>
__global__ void __launch_bounds__(SweepCfg<T, KB>::WARPS * 32) sweep_kernel(Args<T> A)
{
    using C = SweepCfg<T, KB>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SweepSlot<T, KB> *slot = reinterpret_cast<SweepSlot<T, KB> *>(smem) + (size_t)warp * C::NSLOT;
    const SyncArgs sy = sync_of(A);
    if (!ws_ok<T, KB>(A, sy)) return;
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = atomicAdd(A.ctl + kCtlSweepTicket, 1);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk >= A.ntasks) return;
        const int2 task = __ldg(A.tasks + tk);
        if (!sweep_segment<T, KB, C::NSLOT>(A, sy, task.x, task.y, slot)) return;
    }
}

// ---------------------------------------------------------------- fused pass

// After the far sums are all taken, a worker warp of a fused pass takes the
// coefficient and sweep tasks in the host's order: every task's inputs come
// from the chain, the far-sum workers or tasks earlier in the order, so the
// warps that wait always wait on work that is running.
template <typename T, int KB>
struct FusedCfg {
    static constexpr size_t warp_bytes = WorkerCfg<T, KB>::warp_bytes;
    static constexpr int fit = (int)(warp_bytes / sizeof(SweepSlot<T, KB>));
    static constexpr int NSLOT = fit > 3 ? 3 : (fit < 2 ? 2 : fit);
    // a worker warp's shared memory holds two sweep slots and a coefficient
    // task's Gram rows (up to 8 vectors per pass)
    static constexpr bool ok = fit >= 2 && Packed<KB>::smem <= warp_bytes;
};

template <typename T, int KB>
__device__ void post_tasks(const Args<T> &A, const SyncArgs &sy, unsigned char *wsmem)
{
    const int lane = threadIdx.x & 31;
    static_assert(Aug<T, KB>::bytes <= WorkerCfg<T, KB>::warp_bytes, "a worker warp's shared memory holds the task");
    if (take_aug<T, KB>(A) && !aug_task<T, KB>(A, sy, reinterpret_cast<T *>(wsmem))) return;
    for (;;) {
        int tk = 0;
        if (lane == 0) tk = aborted(sy) ? (1 << 30) : atomicAdd(A.ctl + kCtlPostTicket, 1);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if (tk >= A.npost) return;
        const int2 t = __ldg(A.post + tk);
        if (t.x < 0) {
            const int r = t.y;
            if (r < 0 || r >= A.nb) {
                if (lane == 0) record_error(sy, kStatusBounds, (long long)r);
                return;
            }
            if (!coef_block<T, KB>(A, sy, r, reinterpret_cast<double *>(wsmem), true)) return;
            __syncwarp();
            if (lane == 0) {
                __threadfence();
                st_release_gpu(A.cflag + r, A.epoch);
            }
        } else if (!sweep_segment<T, KB, FusedCfg<T, KB>::NSLOT>(A, sy, t.x, t.y,
                                                                 reinterpret_cast<SweepSlot<T, KB> *>(wsmem))) {
            return;
        }
    }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kTrsmWarps * 32, 1) trsm_kernel(Args<T> A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_role;
    if (!ws_ok<T, KB>(A, sync_of(A))) return;
    if (threadIdx.x == 0) s_role = atomicAdd(A.ctl + kCtlRole, 1);
    __syncthreads();
    if (s_role == 0) {
        trsm_chain<T, KB>(A, smem);
        return;
    }
    const bool more = trsm_workers<T, KB>(A, smem);
    if constexpr (FusedCfg<T, KB>::ok) {
        const int warp = threadIdx.x >> 5;
        if (A.fused && more && warp < WorkerCfg<T, KB>::warps)
            post_tasks<T, KB>(A, sync_of(A), smem + (size_t)warp * WorkerCfg<T, KB>::warp_bytes);
    }
}

}  // namespace pass
}  // namespace chm
