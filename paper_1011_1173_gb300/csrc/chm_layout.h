// Scratch layout of the wave kernel, shared by the device code and the host
// side that carves scratch memory for one or many problems: the per-pair
// data records, the flag words, the problem record and the launch control
// words.  Plain C++ usable from host and device translation units.
#pragma once

#include <stddef.h>

#ifdef __CUDACC__
#define CHM_HD __host__ __device__
#else
#define CHM_HD
#endif

namespace chm {

// Columns per column block == rows per published rotation panel == one warp.
constexpr int kW = 32;
// Update vectors (waves) of one problem in one launch; more are split over launches.
constexpr int kMaxWaves = 64;
constexpr int kMaxSm = 1024;
constexpr int kMaxGroups = 128;
constexpr int kTracePoints = 16;

// Sweep coefficients of one row of one wave, in the Apply type T: the
// rotation's a and b, the new row scale e1, and g = e p (the row's old scale
// times the chain's p), with which a column's carry z drops the row's term.
template <typename T>
struct CoefRow {
    T a, b, e1, g;
};

// Row data of one wave (double): new row scale and its inverse, new
// diagonal and its inverse.  The "wave -1" entries (chain0) hold the
// original factor's data: {1, 1, L_ii, 1 / L_ii}.
struct ChainRow {
    double e1, ie1, d1, id1;
};

// ---------------------------------------------------------------- scratch layout

CHM_HD constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets inside the data record of one pair (nb column blocks).  Every
// array is written before it is read within a launch.
struct PairRec {
    size_t coef;   // [nb][kW] CoefRow (32-byte rows for either type)
    size_t chain;  // [nb][kW] ChainRow, this wave's row data after the wave
    size_t tend;   // [nb]     T after the block's last row
    size_t rdiag;  // [nb][kW][kW] -S_rc e_r / D_r, r < c (diagonal block), for this wave
    size_t rtile;  // [nb][kW][kW] -S_rc e_r (rows of block b, cols of b+1), for this wave
    size_t bytes;
};
CHM_HD inline PairRec pair_rec(int nb)
{
    PairRec r;
    size_t x = 0;
    const size_t rows = (size_t)nb * kW;
    r.coef = x;  x += rows * 32;
    r.chain = x; x += rows * sizeof(ChainRow);
    r.tend = x;  x = align256(x + (size_t)nb * sizeof(double));
    r.rdiag = x; x += rows * kW * sizeof(double);
    r.rtile = x; x += rows * kW * sizeof(double);
    r.bytes = align256(x);
    return r;
}
// A problem with k waves: k pair records, then chain0 ([nb][kW] ChainRow).
CHM_HD inline size_t prob_data_bytes(int nb, int k)
{
    return (size_t)k * pair_rec(nb).bytes + align256((size_t)nb * kW * sizeof(ChainRow));
}
// Its int flags: per pair pflag, dflag ([nb] each), then rflag0 [nb].
CHM_HD inline size_t prob_iflags(int nb, int k) { return ((size_t)(2 * k + 1) * nb + 63) & ~(size_t)63; }
// Its tagged 64-bit words, each (epoch << 32) | 32-bit payload: per pair
// [nb] progress words (payload: off-diagonal tiles done), then per pair
// [nb][kW][2] the carry z = T u_hat before the block's last tile and
// [nb][kW][2] the carry u_hat at the diagonal block (payload: the high and
// the low half of a double).  A reader takes a carry once both halves carry
// the current epoch, so the writer needs no fence.
// Then one word counts the final pass's finished column tasks (payload),
// and one word per pair (its k waves, then the final pass) counts the
// pair's column tasks handed out (payload); the wave block that takes the
// pair sets it to (epoch << 32) before announcing the pair.
constexpr int kTagsPerBlock = 1 + 4 * kW;
CHM_HD inline size_t prob_final_done(int nb, int k) { return (size_t)k * nb * kTagsPerBlock; }
CHM_HD inline size_t prob_ticket(int nb, int k, int q) { return prob_final_done(nb, k) + 1 + (size_t)q; }
CHM_HD inline size_t prob_progress(int nb, int k) { return (prob_ticket(nb, k, k + 1) + 31) & ~(size_t)31; }

// One problem of a launch (L and V of the launch's element type).
struct Prob {
    void *L;
    const void *V;
    long long n, ld, ldv;
    int k;                         // waves of this problem in the launch (<= kMaxWaves)
    int nb;                        // column blocks of kW columns
    int pair0;                     // index of its first pair (k waves, then the final pass)
    unsigned long long down_mask;  // bit q set: wave q is a downdate
    char *data;                    // prob_data_bytes(nb, k), 256-byte aligned
    int *iflags;                   // prob_iflags(nb, k) ints
    long long *progress;           // prob_progress(nb, k) tagged words
    long long *info;               // optional {status, row} of this problem
};

// Launch-wide control words (ints); everything but the epoch is zero at the
// start of a launch and is zeroed again by the launch's last block.
constexpr int kCtlPairNext = 0;   // next pair to take
constexpr int kCtlPairsDone = 1;  // pairs whose wave block finished
constexpr int kCtlSmRank = 2;     // SMs registered so far
constexpr int kCtlStarted = 3;    // blocks started
constexpr int kCtlExited = 4;     // blocks finished
constexpr int kCtlEpoch = 8;      // launch counter; flags of this launch equal it
constexpr int kCtlAbort = 32;     // non-zero once a wait has timed out
constexpr int kCtlGroupTicket = 64;                                  // u64 [kMaxGroups]: (current pair + 1) << 32
constexpr int kCtlGroupSweepers = kCtlGroupTicket + 2 * kMaxGroups;  // [kMaxGroups] sweep SMs per group
constexpr int kCtlSmSlot = kCtlGroupSweepers + kMaxGroups;           // [kMaxSm] arrivals per SM
constexpr int kCtlSmRole = kCtlSmSlot + kMaxSm;                      // [kMaxSm] 1 + role of the SM
constexpr int kCtlInts = kCtlSmRole + kMaxSm;
constexpr unsigned kGroupDone = 0xffffffffu;  // ticket high word: the group takes no more pairs

}  // namespace chm
