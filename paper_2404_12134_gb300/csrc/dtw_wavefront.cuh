// Hard-min band wavefront (DTW, Eq. 1 via Eq. 5 with gamma = 0).
#pragma once

#include "plan.cuh"
#include "wts_common.cuh"

namespace wts {

enum DPMode : int {
    kModeCost = 0,    // r(M,N) only
    kModePlen = 1,    // r(M,N) and |pi| (cells on the tie-rule path), score = r / |pi|
    kModeDirs = 2,    // r(M,N) and a 2-bit predecessor code per cell
    kModeSubDirs = 3, // Sub-DTW (Sec. 3.2): free start (the row above the matrix is 0), codes,
                      // and min_j r(M-1, j) with its first column j (R = 8 or 16)
};

struct DPParams {
    const PairDesc* pairs;
    const int32_t* order;
    const int32_t* prefix;
    int P;
    int n_items;
    int d;
    WsHeader* hdr;
    void* hbuf;          // hand-off rows: float r per column, or {float r, int cells} (kModePlen);
                         // pre-filled with 0xFF bytes (NaN) before the launch
    uint32_t* dirs;      // direction words (kModeDirs)
    float* cost_out;     // [*] indexed by PairDesc::out (may be null)
    int32_t* plen_out;   // [*] (kModePlen, may be null)
    float* score_out;    // [*] (kModePlen, may be null)
    int32_t* bstar_out;  // [*] (kModeSubDirs): the first column of minimum r in the last row
    float* cost_matrix;  // pairwise mode: [T][T] symmetric, written at (a,b) and (b,a) (may be null)
    int T;               // cycles (pairwise index decode)
    const int32_t* subset;  // pairwise subset (may be null)
    // checkpoint recomputation: run only bands [band_lo, band_lo + band_cnt) of
    // every pair, from their stored top rows, writing codes relative to band_lo
    int recompute;
    int band_lo, band_cnt;
    long long spin_limit;    // polls before a wait gives up
    int skip_handoff;        // fault injection (tests): producers do not write hand-off rows
    int banded;              // pairs carry a Sakoe-Chiba band (PairDesc::band_bound); R = 16 only;
                             // items then run band-major (every pair's band 0, then band 1, ...)
    int cost_kind;           // LocalCost; kCostL2 runs with R = 16 only
    int group_pairs;         // > 0 (every pair with the same bands): the work list takes pairs in
                             // groups of this many, band-major within a group; 0: pair after pair
};

// Launch the persistent wavefront for D (padded channels) and R (rows/lane);
// p.banded and p.cost_kind select the instance set.
cudaError_t launch_dtw_wavefront(int mode, int D, int R, const DPParams& p, int grid, int block, cudaStream_t st);
int dtw_wavefront_max_blocks_per_sm(int mode, int D, int R, int block, int banded = 0, int cost_kind = 0);

// The instance sets, one per translation unit (dtw_wavefront_<set>.cu):
// rows per lane, band, local cost.
#define WTS_WF_SETS(X) \
    X(r4)     /* R = 4,  Sub-DTW only, squared l2 */ \
    X(r8)     /* R = 8,  no band, squared l2 */ \
    X(r16)    /* R = 16, no band, squared l2 */ \
    X(r16b)   /* R = 16, band,    squared l2 */ \
    X(r32)    /* R = 32, no band, squared l2 (d <= 3) */ \
    X(l2)     /* R = 16, no band, l2 norm */ \
    X(l2b)    /* R = 16, band,    l2 norm */
#define WTS_WF_DECL(TAG)                                                                                  \
    cudaError_t wf_launch_##TAG(int mode, int D, const DPParams& p, int grid, int block, cudaStream_t st); \
    int wf_occ_##TAG(int mode, int D, int block);
WTS_WF_SETS(WTS_WF_DECL)
#undef WTS_WF_DECL

}  // namespace wts
