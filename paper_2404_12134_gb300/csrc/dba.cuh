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
};

cudaError_t launch_backtrack(const BTParams& p, cudaStream_t st);

// B_out[i] = mean of the cycle samples aligned to row i over all cycles;
// counts[i] = number of aligned samples; cost_before = sum_k costs[k].
cudaError_t launch_dba_average(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               const int32_t* jlo, const int32_t* jhi, const float* costs,
                               float* B_out, int32_t* counts, double* cost_before, cudaStream_t st);

cudaError_t launch_resample(const float* x, int64_t N, int d, float* out, int64_t M, cudaStream_t st);
cudaError_t launch_euclid_mean(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               float* out, cudaStream_t st);
cudaError_t launch_medoid(const float* C, int T, int32_t* index_out, double* sums_out, cudaStream_t st);

}  // namespace wts
