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
    T *Dinv;         // [nb][32][32]: (D_b^T)^{-1}, D_b the diagonal block, row-major
    T *G;            // [nb][32][32]: Dinv_b F_{b-1,b}^T, row-major
    double *gram;    // [nb][KB][KB]: sum over the block's rows of p p^T
    double *H;       // [nb][KB][KB]: Sigma + sum over earlier blocks
    T *coef;         // [nb * 32][2 KB]: (a_q, b_q) of each row
    T *escale;       // [nb * 32]: 1 / sqrt(D_kb) of each row
    double *dfac;    // [nb * 32]: sqrt(D_kb) of each row
    long long *Ptag; // [nb * 32][KB][words of T]: P as epoch-tagged words
    long long *Ztag; // [nb][32][KB][words of T]: Zf as epoch-tagged words
    int *ctl;        // kCtlInts control words
    long long *status;     // sticky {status, row} of the stream
    long long *user_info;  // optional {status, row} of the call
    long long timeout_ns;
    long long *trace;      // optional [nb][8] %globaltimer stamps of the substitution:
                           // P posted, Zhat posted, far sum staged, stage loaded,
                           // P published; a worker's last P seen, its far sum published
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
__device__ __forceinline__ void prefetch_l2(const void *gmem)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(gmem));
}

// Warp-cooperative stage of the tile rows r0.. r0 + 31, columns c0 .. c0 + 31
// of L into dst[column][Stride] (columns >= n are zero).  `vec`: 16-byte
// copies (every column's segment 16-byte aligned and all 32 rows inside the
// column, r0 + 32 <= n); otherwise one element per copy, rows >= nrows zero.
template <typename T>
__device__ __forceinline__ void stage_tile(T *dst, const T *L, long long ld, long long r0, long long c0,
                                           long long n, int nrows, bool vec, int lane)
{
    constexpr int S = Stride<T>::value;
    if (vec) {
        constexpr int E = 16 / (int)sizeof(T);  // elements per chunk
        constexpr int CPC = kB / E;             // chunks per column
        for (int c = lane; c < kB * CPC; c += 32) {
            const int col = c / CPC, ch = c % CPC;
            T *d = dst + col * S + ch * E;
            if (c0 + col < n) {
                cp16(d, L + (r0 + ch * E) + (c0 + col) * ld);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) d[e] = T(0);
            }
        }
    } else {
        for (int col = 0; col < kB; ++col) {
            T *d = dst + col * S + lane;
            if (c0 + col < n && lane < nrows) cp_elem(d, L + (r0 + lane) + (c0 + col) * ld);
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

// Lane i: out[q] = sum_l M[i][l] x[l][q] (M staged with Stride, x [32][KB]).
template <typename T, int KB>
__device__ __forceinline__ void lane_mv(const T *M, const T *x, T (&out)[KB], int i)
{
    constexpr int S = Stride<T>::value;
    constexpr int E = Vec16<T>::n;
    using V = typename Vec16<T>::type;
    T a0[KB], a1[KB];
#pragma unroll
    for (int q = 0; q < KB; ++q) a0[q] = a1[q] = T(0);
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
                const V *xr = reinterpret_cast<const V *>(x + l * KB);
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
                    if (l & 1) a1[q] = fma(mv, x[l * KB + q], a1[q]);
                    else a0[q] = fma(mv, x[l * KB + q], a0[q]);
                }
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

// Warps of the forward-substitution kernel and the chain block's roles.
constexpr int kTrsmWarps = 12;
constexpr int kWCrit = 0, kWZhat = 1, kWNear0 = 2;
constexpr int kNearWarps = kTrsmWarps - 5;  // warps 2 .. 8
constexpr int kWZf = kTrsmWarps - 3, kWLoad = kTrsmWarps - 2, kWPub = kTrsmWarps - 1;

// Lookahead bound (near tiles d - 1 per step) and ring depths per
// instantiation, sized to the 227 KB of shared memory.
template <typename T, int KB>
struct ChainCfg {
    static constexpr int DMAX = sizeof(T) == 4 ? (KB <= 2 ? 10 : KB <= 4 ? 9 : KB <= 8 ? 8 : 6)
                                               : (KB <= 2 ? 5 : KB <= 8 ? 4 : 3);
    static constexpr int RP = DMAX + 2;   // P ring
    static constexpr int RT = DMAX;       // per near offset
    static constexpr int RZ = 4;          // Zhat ring
    static constexpr int RF = 4;          // far-sum ring
    static constexpr int PF = 8;          // steps of L2 prefetch ahead of the stage
    static constexpr size_t tile = sizeof(T) * kB * Stride<T>::value;
    static constexpr size_t stage = (size_t)(DMAX + 1) * tile;  // G, Dinv, d - 1 near tiles
    static constexpr size_t rest = sizeof(T) * kB * KB * ((size_t)RP + (size_t)(DMAX - 1) * RT + RZ + RF + 1) +
                                   tile + 256;
    static constexpr int fit = (int)((224u * 1024u - rest) / stage);
    static constexpr int RS = fit > 4 ? 4 : fit;  // staged steps
};

template <typename T, int KB>
struct ChainSmem {
    using C = ChainCfg<T, KB>;
    static constexpr int S = Stride<T>::value;
    T G[C::RS][kB * S];                   // G_m of step m
    T Di[C::RS][kB * S];                  // Dinv_{m+1}
    T near[C::DMAX - 1][C::RS][kB * S];   // per offset j = 2 .. d: tiles (m, m + j), [column][row]
    T Di0[kB * S];                        // Dinv_0
    T P[C::RP][kB * KB];
    T Tn[C::DMAX - 1][C::RT][kB * KB];    // F_{b-j,b}^T P_{b-j} per offset j
    T Z[C::RZ][kB * KB];                  // Zhat_b
    T F[C::RF][kB * KB];                  // far sums Zf_b
    T w[kB * KB];                         // Zhat warp's work vector
    int pseq, zseq, lseq, fseq, pubseq;
    int nseq[kNearWarps];
    int stop;
};

// The chain block: every role is one warp, linked by shared-memory
// sequence counters; nothing on the critical cycle
//   P_m -> F_{m,m+2}^T P_m -> Zhat_{m+2} -> P_{m+2}
// waits on global memory: the loader stages G, Dinv and the near tiles a
// few steps ahead (and prefetches further ones into L2), the far-sum warp
// polls the workers' tagged sums ahead of use, the publisher writes each P
// as tagged words.
template <typename T, int KB>
__device__ void trsm_chain(const Args<T> &A, unsigned char *smem)
{
    using C = ChainCfg<T, KB>;
    ChainSmem<T, KB> &S = *reinterpret_cast<ChainSmem<T, KB> *>(smem);
    constexpr int SD = Stride<T>::value;
    constexpr int TW = Tag<T>::words;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = A.nb, d = A.d;
    const long long n = A.n, ld = A.ld;
    const long long ep64 = (long long)A.epoch << 32;
    const SyncArgs sy = sync_of(A);
    volatile int *stop = &S.stop;
    const bool vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
    if (threadIdx.x == 0) {
        S.pseq = S.zseq = S.lseq = S.fseq = S.pubseq = 0;
        for (int t = 0; t < kNearWarps; ++t) S.nseq[t] = 0;
        S.stop = 0;
    }
    __syncthreads();
    const int nnear = d - 1;  // offsets j = 2 .. d, offset j on near warp (j - 2) % kNearWarps
#define CW(seqp, want, who)                                                     \
    do {                                                                        \
        if (!warp_seq_wait(sy, (seqp), (want), stop, (who))) {                  \
            cp_wait<0>();                                                       \
            return;                                                             \
        }                                                                       \
    } while (0)

    if (warp == kWLoad) {
        for (int m = 0; m < nb; ++m) {
            const int st = m % C::RS;
            if (m >= C::RS) {
                const int old = m - C::RS;
                CW(&S.pseq, old + 1, -10);
                CW(&S.zseq, old + 2, -12);
            }
            if (m >= 1) stage_dense(S.G[st], A.G + (size_t)m * kB * kB, lane);
            if (m + 1 < nb) stage_dense(S.Di[st], A.Dinv + (size_t)(m + 1) * kB * kB, lane);
            cp_commit();
            // later steps' near band into L2 (one line per column segment)
            const int mf = m + C::PF;
            if (mf < nb) {
                const long long rf = (long long)mf * kB;
                for (int c = lane; c < (d - 1) * kB; c += 32) {
                    const long long col = (long long)(mf + 2) * kB + c;
                    if (col < n) prefetch_l2(A.L + rf + col * ld);
                }
            }
            // stage m - 1 is complete once at most one group is pending
            cp_wait<1>();
            warp_seq_post(&S.lseq, m);
            if (A.trace && lane == 0 && m >= 1) A.trace[(size_t)(m - 1) * 8 + 3] = global_ns();
        }
        cp_wait<0>();
        warp_seq_post(&S.lseq, nb);
    } else if (warp == kWCrit) {
        for (int m = 0; m < nb; ++m) {
            CW(&S.zseq, m + 1, m);
            if (m >= 1) CW(&S.lseq, m + 1, m);
            if (m >= C::RP) CW(&S.pubseq, m - C::RP + 1, m);
            T out[KB];
            const T *z = S.Z[m % C::RZ];
            if (m == 0) {
#pragma unroll
                for (int q = 0; q < KB; ++q) out[q] = z[lane * KB + q];
            } else {
                lane_mv<T, KB>(S.G[m % C::RS], S.P[(m - 1) % C::RP], out, lane);
#pragma unroll
                for (int q = 0; q < KB; ++q) out[q] = z[lane * KB + q] - out[q];
            }
            T *pm = S.P[m % C::RP];
#pragma unroll
            for (int q = 0; q < KB; ++q) pm[lane * KB + q] = out[q];
            warp_seq_post(&S.pseq, m + 1);
            if (A.trace && lane == 0) A.trace[(size_t)m * 8 + 0] = global_ns();
        }
    } else if (warp >= kWNear0 && warp < kWNear0 + kNearWarps) {
        const int t = warp - kWNear0;
        if (t >= nnear) return;
        // this warp's offsets' tiles, staged RS - 1 steps ahead (the factor as
        // it entered the pass: nothing to wait for)
        auto stage = [&](int m) {
            if (m < nb) {
                for (int j = 2 + t; j <= d; j += kNearWarps) {
                    const int b = m + j;
                    if (b >= nb) break;
                    stage_tile(S.near[j - 2][m % C::RS], A.L, ld, (long long)m * kB, (long long)b * kB, n, kB,
                               vec, lane);
                }
            }
            cp_commit();
        };
        for (int m = 0; m < C::RS - 1; ++m) stage(m);
        for (int m = 0; m < nb; ++m) {
            stage(m + C::RS - 1);
            CW(&S.pseq, m + 1, m);
            cp_wait<C::RS - 1>();
            __syncwarp();
            const T *pm = S.P[m % C::RP];
            for (int j = 2 + t; j <= d; j += kNearWarps) {
                const int b = m + j;
                if (b >= nb) break;
                T out[KB];
                lane_mv<T, KB>(S.near[j - 2][m % C::RS], pm, out, lane);
                T *dst = S.Tn[j - 2][b % C::RT];
#pragma unroll
                for (int q = 0; q < KB; ++q) dst[lane * KB + q] = out[q];
            }
            warp_seq_post(&S.nseq[t], m + 1);
        }
    } else if (warp == kWZhat) {
        // Dinv_0 for Zhat_0
        stage_dense(S.Di0, A.Dinv, lane);
        cp_commit();
        cp_wait<0>();
        __syncwarp();
        for (int b = 0; b < nb; ++b) {
            const long long r0 = (long long)b * kB;
            // w = Zf_b - sum_{j=2}^{d} F_{b-j,b}^T P_{b-j}
            T w[KB];
            if (b > d) {
                CW(&S.fseq, b + 1, b);
                const T *f = S.F[b % C::RF];
#pragma unroll
                for (int q = 0; q < KB; ++q) w[q] = f[lane * KB + q];
            } else {
#pragma unroll
                for (int q = 0; q < KB; ++q)
                    w[q] = (r0 + lane < n && q < A.kb) ? A.V[r0 + lane + q * A.ldv] : T(0);
            }
            for (int j = 2; j <= d && j <= b; ++j) {
                const int t = (j - 2) % kNearWarps;
                CW(&S.nseq[t], b - j + 1, b);
                const T *tn = S.Tn[j - 2][b % C::RT];
#pragma unroll
                for (int q = 0; q < KB; ++q) w[q] -= tn[lane * KB + q];
            }
#pragma unroll
            for (int q = 0; q < KB; ++q) S.w[lane * KB + q] = w[q];
            __syncwarp();
            const T *Di = S.Di0;
            if (b >= 1) {
                CW(&S.lseq, b, b);  // stage b - 1 holds Dinv_b
                Di = S.Di[(b - 1) % C::RS];
            }
            T out[KB];
            lane_mv<T, KB>(Di, S.w, out, lane);
            T *z = S.Z[b % C::RZ];
#pragma unroll
            for (int q = 0; q < KB; ++q) z[lane * KB + q] = out[q];
            warp_seq_post(&S.zseq, b + 1);
            if (A.trace && lane == 0) A.trace[(size_t)b * 8 + 1] = global_ns();
        }
    } else if (warp == kWZf) {
        for (int b = d + 1; b < nb; ++b) {
            if (b >= C::RF) CW(&S.zseq, b - C::RF + 1, b);
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
            T *f = S.F[b % C::RF];
#pragma unroll
            for (int q = 0; q < KB; ++q) f[lane * KB + q] = v[q];
            warp_seq_post(&S.fseq, b + 1);
            if (A.trace && lane == 0) A.trace[(size_t)b * 8 + 2] = global_ns();
        }
    } else if (warp == kWPub) {
        for (int m = 0; m < nb; ++m) {
            CW(&S.pseq, m + 1, m);
            const T *pm = S.P[m % C::RP];
            long long *tg = A.Ptag + ((size_t)m * kB + lane) * KB * TW;
            T *plain = A.P + ((size_t)m * kB + lane) * KB;
#pragma unroll
            for (int q = 0; q < KB; ++q) {
                const T v = pm[lane * KB + q];
                put_tag(tg + q * TW, v, ep64);
                plain[q] = v;
            }
            warp_seq_post(&S.pubseq, m + 1);
            if (A.trace && lane == 0) A.trace[(size_t)m * 8 + 4] = global_ns();
        }
    }
#undef CW
}

// Worker warps: the far part of column block b's sum,
//   Zf_b = V_b - sum_{r < b - d} F_{r,b}^T P_r,
// tiles staged a few ahead (they are the factor as it entered the pass), each
// P_r polled as tagged words, Zf_b published as tagged words.
template <typename T, int KB>
struct WorkerCfg {
    static constexpr int NS = 3;  // staged tiles per warp
    static constexpr size_t warp_bytes = sizeof(T) * ((size_t)NS * kB * Stride<T>::value + kB * KB);
    static constexpr int warps = (int)((200u * 1024u) / warp_bytes) < kTrsmWarps
                                     ? (int)((200u * 1024u) / warp_bytes) : kTrsmWarps;
};

template <typename T, int KB>
__device__ void trsm_workers(const Args<T> &A, unsigned char *smem)
{
    using W = WorkerCfg<T, KB>;
    constexpr int SD = Stride<T>::value;
    constexpr int TW = Tag<T>::words;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp >= W::warps) return;
    T *base = reinterpret_cast<T *>(smem + (size_t)warp * W::warp_bytes);
    T *Pr = base + (size_t)W::NS * kB * SD;  // [32][KB]
    const long long n = A.n, ld = A.ld;
    const int nb = A.nb, d = A.d;
    const long long ep64 = (long long)A.epoch << 32;
    const SyncArgs sy = sync_of(A);
    const bool vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
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
        for (int r = 0; r < W::NS - 1 && r < nfar; ++r) {
            stage_tile(base + (size_t)(r % W::NS) * kB * SD, A.L, ld, (long long)r * kB, c0, n, kB, vec, lane);
            cp_commit();
        }
        for (int r = 0; r < nfar; ++r) {
            const int rn = r + W::NS - 1;
            if (rn < nfar)
                stage_tile(base + (size_t)(rn % W::NS) * kB * SD, A.L, ld, (long long)rn * kB, c0, n, kB, vec, lane);
            cp_commit();
            // P_r: lane l polls row l's tagged words
            const long long *src = A.Ptag + ((size_t)r * kB + lane) * KB * TW;
            T pv[KB];
            const long long t0 = global_ns();
            unsigned ns = 32;
            for (unsigned it = 0;; ++it) {
                bool ok = true;
#pragma unroll
                for (int q = 0; q < KB; ++q) ok = get_tag(src + q * TW, ep64, &pv[q]) && ok;
                if (__all_sync(0xffffffffu, ok)) break;
                if ((it & 15u) == 15u) {
                    int bad = 0;
                    if (lane == 0) {
                        if (aborted(sy)) bad = 1;
                        else if (global_ns() - t0 > sy.timeout_ns || it > (1u << 26)) {
                            record_error(sy, kStatusTimeout, b);
                            bad = 1;
                        }
                    }
                    if (__shfl_sync(0xffffffffu, bad, 0)) {
                        cp_wait<0>();
                        return;
                    }
                }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
#pragma unroll
            for (int q = 0; q < KB; ++q) Pr[lane * KB + q] = pv[q];
            if (A.trace && lane == 0 && r == nfar - 1) A.trace[(size_t)b * 8 + 6] = global_ns();
            cp_wait<W::NS - 1>();
            __syncwarp();
            T t[KB];
            lane_mv<T, KB>(base + (size_t)(r % W::NS) * kB * SD, Pr, t, lane);
#pragma unroll
            for (int q = 0; q < KB; ++q) z[q] -= t[q];
            __syncwarp();
        }
        cp_wait<0>();
        long long *zt = A.Ztag + ((size_t)b * kB + lane) * KB * TW;
#pragma unroll
        for (int q = 0; q < KB; ++q) put_tag(zt + q * TW, z[q], ep64);
        if (A.trace && lane == 0) A.trace[(size_t)b * 8 + 7] = global_ns();
    }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kTrsmWarps * 32, 1) trsm_kernel(Args<T> A)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_role;
    if (threadIdx.x == 0) s_role = atomicAdd(A.ctl + kCtlRole, 1);
    __syncthreads();
    if (s_role == 0) trsm_chain<T, KB>(A, smem);
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
        if (q >= A.kb || r >= A.kb) pre = (q == r) ? 1.0 : 0.0;  // padding vectors: identity
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

template <typename T, int KB>
__global__ void __launch_bounds__(32) coef_kernel(Args<T> A)
{
    using PK = Packed<KB>;
    constexpr int NE = PK::entries, HS = PK::stride;
    extern __shared__ double Hs[];  // [kB + 1][HS]
    const int lane = threadIdx.x;
    const SyncArgs sy = sync_of(A);
    const long long n = A.n;
    const int kb = A.kb;
    for (int b = blockIdx.x; b < A.nb; b += gridDim.x) {
        const long long r0 = (long long)b * kB;
        const int rows = (int)min((long long)kB, n - r0);
        double p[KB];
        const T *prow = A.P + (size_t)(r0 + lane) * KB;
#pragma unroll
        for (int q = 0; q < KB; ++q) p[q] = (q < kb) ? (double)__ldcg(prow + q) : 0.0;
        // row 0: H_b; row lane + 1: this lane's outer product
        const double *hb = A.H + (size_t)b * KB * KB;
        for (int e = lane; e < NE; e += 32) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            Hs[e] = hb[i * KB + (e - i * (i + 1) / 2)];
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
    }
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

template <typename T, int KB>
__global__ void __launch_bounds__(SweepCfg<T, KB>::WARPS * 32) sweep_kernel(Args<T> A)
{
    using C = SweepCfg<T, KB>;
    constexpr int SD = Stride<T>::value;
    constexpr int E = 16 / (int)sizeof(T);
    using V = typename Vec16<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    SweepSlot<T, KB> *slot = reinterpret_cast<SweepSlot<T, KB> *>(smem) + (size_t)warp * C::NSLOT;
    const long long n = A.n, ld = A.ld;
    const int nb = A.nb;
    const bool vec = ((ld * (long long)sizeof(T)) & 15) == 0 && (reinterpret_cast<uintptr_t>(A.L) & 15) == 0;
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
            SweepSlot<T, KB> &sl = slot[r % C::NSLOT];
            const long long r0 = (long long)r * kB;
            if (r < b) {
                stage_tile(sl.tile, A.L, ld, r0, c0, n, kB, vec, lane);
            } else {
                // the diagonal tile: rows <= column only
                for (int col = 0; col < kB; ++col)
                    if (c0 + col < n && lane <= col) cp_elem(&sl.tile[col * SD + lane], A.L + (r0 + lane) + (c0 + col) * ld);
            }
            const T *cf = A.coef + (size_t)r0 * 2 * KB;
            for (int c = lane; c < kB * 2 * KB / E; c += 32) cp16(sl.cf + c * E, cf + c * E);
            for (int c = lane; c < kB / E; c += 32) cp16(sl.e + c * E, A.escale + r0 + c * E);
            if (r == b && lane < kB / 2) cp16(sl.df + 2 * lane, A.dfac + r0 + 2 * lane);
        };
        for (int r = 0; r < C::NSLOT - 1; ++r) {
            if (r <= b) fetch(r);
            cp_commit();
        }
        for (int r = 0; r <= b; ++r) {
            if (r + C::NSLOT - 1 <= b) fetch(r + C::NSLOT - 1);
            cp_commit();
            cp_wait<C::NSLOT - 1>();
            __syncwarp();
            SweepSlot<T, KB> &sl = slot[r % C::NSLOT];
            const bool diag = r == b;
            const long long r0 = (long long)r * kB;
            const int rows = diag ? lane : (int)min((long long)kB, n - r0);
            T v[kB];
            V *colv = reinterpret_cast<V *>(sl.tile + lane * SD);
#pragma unroll
            for (int c = 0; c < kB / E; ++c) {
                const V x = colv[c];
#pragma unroll
                for (int u = 0; u < E; ++u) v[c * E + u] = vget<T>(x, u);
            }
            if (active) {
#pragma unroll
                for (int i = 0; i < kB; ++i) {
                    if (i < rows) {
                        T x = v[i];
#pragma unroll
                        for (int q = 0; q < KB; ++q) {
                            x = fma(sl.cf[i * 2 * KB + 2 * q], uh[q], x);
                            uh[q] = fma(-sl.cf[i * 2 * KB + 2 * q + 1], x, uh[q]);
                        }
                        v[i] = x * sl.e[i];
                    } else if (diag && i == lane) {
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
                constexpr int CPC = kB / E;
                for (int c = lane; c < kB * CPC; c += 32) {
                    const int cc = c / CPC, ch = c % CPC;
                    if (c0 + cc < n)
                        *reinterpret_cast<V *>(A.L + (r0 + ch * E) + (c0 + cc) * ld) =
                            *reinterpret_cast<const V *>(sl.tile + cc * SD + ch * E);
                }
            } else {
#pragma unroll 8
                for (int cc = 0; cc < kB; ++cc)
                    if (c0 + cc < n && (!diag || lane <= cc) && (diag || lane < rows))
                        A.L[(r0 + lane) + (c0 + cc) * ld] = sl.tile[cc * SD + lane];
            }
            __syncwarp();
        }
        cp_wait<0>();
    }
}

}  // namespace pass
}  // namespace chm
