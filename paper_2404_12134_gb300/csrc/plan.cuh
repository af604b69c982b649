// Workspace layout and work list of one library call.
//
// The caller owns all device memory (inputs, outputs and one workspace
// buffer).  The host computes the layout below from the host copy of the
// cycle offsets; a one-CTA setup kernel rebuilds the same per-pair offsets on
// the device, so no host-to-device copy is issued inside a call (calls can be
// captured in a CUDA graph).
#pragma once

#include <cmath>
#include <cstddef>
#include <cstdint>

#include "wts_common.cuh"

namespace wts {

enum Op : int {
    kOpScore = 1,      // cost + |pi| fused (anomaly_score)
    kOpAlign = 2,      // cost + 2-bit directions + backtrack (dtw_align)
    kOpDba = 3,        // kOpAlign + averaging (dba_iterate)
    kOpSoft = 4,       // soft-DTW forward (R stored) + backward
    kOpPairwise = 5,   // cost-only DTW between all cycle pairs (medoid init)
    kOpCost = 6,       // cost only
    kOpSubdtw = 7,     // Sub-DTW: free-start codes, first cheapest end column, backtrack to the start
};

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-pair storage, shared by host sizing and the device setup kernel.
__host__ __device__ inline int64_t pair_hbuf_slots(int64_t nb, int64_t N) { return (nb - 1) * N; }
// Predecessor codes of one band: 2R bits per lane and step, R/16 words per
// (step, lane) for R >= 16; for R = 8 one word holds two consecutive steps
// (steps 2u and 2u+1 in its low and high halves).
__host__ __device__ inline int64_t band_dir_words(int64_t N, int R)
{
    // N + 31 steps; R < 16: 32 / (2R) steps per word
    return R >= 16 ? (N + 31) * 32 * (R / 16) : ((N + 30 + 32 / (2 * R)) / (32 / (2 * R))) * 32;
}
__host__ __device__ inline int64_t pair_dir_words(int64_t nb, int64_t N, int R) { return nb * band_dir_words(N, R); }
__host__ __device__ inline int64_t pair_rstore_floats(int64_t nb, int64_t N, int R) { return nb * (N + 31) * 32 * R; }
// Soft-DTW column checkpoints (checkpoint mode without a band): every kCk
// forward steps, each lane's R values of its last column and the value above
// its first row; per band [ceil((N + 31) / kCk)][R + 1][32] floats
constexpr int kCk = 16;
__host__ __device__ inline int64_t band_ckcol_floats(int64_t N, int R) { return ((N + 31 + kCk - 1) / kCk) * (R + 1) * 32; }

struct Layout {
    int op = 0;
    int T = 0;            // cycles in the batch
    int P = 0;            // alignment problems (T, or T(T-1)/2 for pairwise)
    int d = 0, D = 0, R = 0, BR = 0;
    int64_t M = 0;        // prototype length (shared-prototype ops)
    int64_t n_items = 0;  // total (pair, band) items
    int64_t hbuf_slots = 0, dir_words = 0, rstore_floats = 0;
    size_t hbuf_bytes = 0, ebuf_bytes = 0;
    size_t off_hdr = 0, off_pairs = 0, off_order = 0, off_prefix = 0;
    size_t off_hbuf = 0, off_dirs = 0, off_jlo = 0, off_jhi = 0, off_costs = 0, off_btstate = 0;
    int group_bands = 0;  // checkpoint mode: bands whose codes are recomputed at a time (0 = codes stored)
    int banded = 0;       // a Sakoe-Chiba band applies (the banded kernels run with R = 16)
    int cost_kind = 0;    // local cost: 0 squared l2, 1 the l2 norm (DTW kernels with R = 16)
    int nseg = 0;         // segments of the segmented backtrack (codes stored, not Sub-DTW)
    int soft_fused = 0;   // soft-DTW checkpoint mode without a band: column checkpoints, fused backward
    int store_pairs = 0;  // soft_fused: the first store_pairs pairs of the longest-first order keep R
    size_t off_seg = 0;

    size_t off_plen = 0, off_rstore = 0, off_gpart = 0, off_ebuf = 0, off_pcost = 0;
    size_t total = 0;
};

// Device-side parameters of the setup kernel.
struct SetupParams {
    int op;
    int T, P, d, R, BR;
    int64_t M;
    const float* B;            // shared prototype (or null for pairwise)
    const float* data;         // packed cycles
    const int64_t* offsets;    // [T+1]
    PairDesc* pairs;           // [P]
    int32_t* order;            // [P] longest first
    int32_t* prefix;           // [P+1] first item of the q-th pair in order
    int sort;                  // 1: order longest-first, 0: identity
    int group_bands;           // > 0: directions for only this many bands per pair (checkpoint mode)
    double band;               // Sakoe-Chiba width (0 = none): band_bound = floor(band * M * N)
    int store_pairs;           // soft-DTW column checkpoints: pairs of rank < store_pairs keep R instead
};

// Rank of pair p in the longest-first order (cells descending, ties by index),
// the order of the work list.
__host__ __device__ inline bool longer_first(int64_t cells_q, int q, int64_t cells_p, int p)
{
    return cells_q > cells_p || (cells_q == cells_p && q < p);
}

// floor(band * M * N) in double, as the host validation and the oracle take it
__host__ __device__ inline int64_t band_bound_of(double band, int64_t M, int64_t N)
{
    if (!(band > 0)) return -1;
    if (band >= 1) return M * N;     // every cell: |i N - j M| < M N
    return (int64_t)floor(band * (double)M * (double)N);
}

void launch_setup(const SetupParams& sp, cudaStream_t st);

// Scan a[0..na) and b[0..nb) (either may be null) for a non-finite value (NaN
// or +-inf, Sec. 3.1 removes missing values before alignment); if one is
// found, set hdr->status = kDevBadInput and hdr->abort = 1, so that every
// kernel of the call leaves before doing any work.  sms sizes the grid.
cudaError_t launch_check_finite(const float* a, int64_t na, const float* b, int64_t nb, WsHeader* hdr, int sms,
                                cudaStream_t st);

}  // namespace wts
