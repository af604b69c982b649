// Backtrack, DBA averaging and barycenter initialisation kernels.
#pragma once

#include "plan.cuh"
#include "wts_common.cuh"

namespace wts {

struct BTParams {
    const PairDesc* pairs;
    int P;
    int R;
    const uint32_t* dirs;
    int32_t* jlo;        // [P][M] indexed by PairDesc::out
    int32_t* jhi;
    int32_t* plen;       // [P] (may be null)
    int64_t M;           // row stride of jlo/jhi
    // codes available for bands [band_lo, band_hi) only (band b at dirs offset
    // b - band_lo); the walk stops on leaving them and keeps its position in
    // state[3*q .. 3*q+2] = (i, j, cells so far), resumed by the next call.
    // state == null: all bands, one walk.
    int band_lo, band_hi;
    int32_t* state;
    int first;           // 1: start every walk at (M-1, N-1)
    // Sub-DTW (Sec. 3.2): start at (M-1, bstar[out]) and stop when the walk
    // leaves row 0 (the free start), writing that column to astar[out]
    int subseq;
    const int32_t* bstar;
    int32_t* astar;
    // segmented walk (every code stored, not Sub-DTW): the rows are cut into
    // nseg segments of seg_rows rows, walked at once, each from a start column
    // in its top row; round r re-walks a segment whose start differs from the
    // exit of the segment above in round r - 1, so after nseg rounds every
    // segment starts where the path enters it.  seg[(q * nseg + k) * 4 + ..] =
    // {start column, exit column in even rounds, in odd rounds, status (1 = the
    // codes were invalid or a wait gave up)}; the exit is the path's column in
    // the row below the segment.
    int nseg, seg_rows, round;
    int32_t* seg;
    // the call's workspace header: a raised abort word (set with the status
    // when the DP left early) makes the walk do nothing (may be null)
    const WsHeader* hdr;
};

// Rows per segment of the segmented walk.
constexpr int kBtSegRows = 2048;

cudaError_t launch_backtrack(const BTParams& p, cudaStream_t st);
// After the nseg rounds of a segmented walk: |pi| = sum_i (jhi(i) - jlo(i) + 1)
// per pair, or -1 if a segment failed or the segments do not join up.
cudaError_t launch_backtrack_seg_final(const BTParams& p, cudaStream_t st);

// B_out[i] = mean of the cycle samples aligned to row i over all cycles;
// counts[i] = number of aligned samples; cost_before = sum_k costs[k].
cudaError_t launch_dba_average(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               const int32_t* jlo, const int32_t* jhi, const float* costs,
                               float* B_out, int32_t* counts, double* cost_before, cudaStream_t st);

// score[k] = cost[k] / plen[k] (one FP32 division, Eq. 8); NaN where the walk failed.
cudaError_t launch_score_divide(const float* cost, const int32_t* plen, float* score, int T, cudaStream_t st);

cudaError_t launch_resample(const float* x, int64_t N, int d, float* out, int64_t M, cudaStream_t st);
cudaError_t launch_euclid_mean(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               float* out, cudaStream_t st);
cudaError_t launch_medoid(const float* C, int T, int32_t* index_out, double* sums_out, cudaStream_t st);

}  // namespace wts
