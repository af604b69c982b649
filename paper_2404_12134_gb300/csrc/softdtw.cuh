// Soft-DTW forward (Eqs. 3-5, R stored) and backward (E recursion, Eq. 6).
#pragma once

#include "plan.cuh"
#include "wts_common.cuh"

namespace wts {

struct SoftParams {
    const PairDesc* pairs;
    const int32_t* order;
    const int32_t* prefix;
    int P;
    int n_items;
    int d;
    float gamma;
    WsHeader* hdr;
    float* hbuf;         // forward hand-off rows (r of a band's bottom row); pre-filled with NaN
    float* ebuf;         // backward hand-off rows: {r, delta} {e, 0} of a band's top row, 16 bytes
                         // per column; pre-filled with NaN
    float* rstore;       // R, per band [(N+31) steps][R/4][32 lanes][4]
    float* value_out;    // [P] Soft-DTW value per pair (forward)
    float* gpart;        // [P][M][d] per-pair gradient sum_j e_ij * d delta_ij / d b_i (backward):
                         // 2 (b_i - y_j), or (b_i - y_j) / delta_ij for the l2 norm
    // checkpoint mode: R is kept only for bands [band_lo, band_lo + band_cnt)
    // (band b at R offset b - band_lo); the forward then recomputes those
    // bands from their stored top rows (recompute = 1, no hand-off writes)
    int store_r;         // forward: write R
    int recompute;
    int band_lo, band_cnt;
    int rbuf_band0;      // checkpoint mode: R of band b is kept in band slot b - band_lo + rbuf_band0
                         // (two buffers of ckpt_bands slots per pair, used by alternate groups)
    // checkpoint mode, backward launches: items n_items .. n_items + n_rec - 1
    // recompute R of the next group up (bands [rec_band_lo, rec_band_lo +
    // rec_band_cnt), into slots from rec_rbuf_band0) while the backward items
    // run; they read only the stored hand-off rows, so they never wait
    int n_rec, rec_band_lo, rec_band_cnt, rec_rbuf_band0;
    // checkpoint mode without a band: column checkpoints instead of R groups.
    // The full forward writes them (ckcol != null), and the backward (fused = 1)
    // recomputes R a few steps at a time inside each band's warp
    // Pairs whose PairDesc::keep_r is set (store_pairs) keep R instead: the
    // fused backward runs their items through the backward that reads it.
    float* ckcol;
    int fused;
    long long spin_limit;    // polls before a wait gives up
    int skip_handoff;        // fault injection (tests): producers do not write hand-off rows
    int banded;              // pairs carry a Sakoe-Chiba band (PairDesc::band_bound); items run band-major
    int cost_kind;           // LocalCost
    int rows;                // rows per lane R: 8, or 4 under a narrow band
    int m_aligned;           // the prototype's M is a multiple of the rows per lane (every lane's rows
                             // lie all inside the matrix or all past it)
};

// Rows held per lane by the soft-DTW kernels (8 for every padded channel
// count: measured best against 4 and 16).
inline int soft_rows(int /*D*/) { return 8; }
// Under a Sakoe-Chiba band narrower than this fraction the soft-DTW passes
// run 4 rows per lane: the band's lower edge is a chain of row bands, each
// starting when the one above has covered its first 32 R + 62 columns, so
// the time barely falls with the band's width at 8 rows; at 4 the chain's
// steps are half as long (64 pairs of 10k, forward + backward: w = 0.3
// 18.5 -> 15.8 ms, w = 0.1 18.0 -> 14.0 ms; at w = 0.6 8 rows stay faster,
// 18.1 against 19.8 ms).
constexpr double kSoftNarrowBand = 0.45;

cudaError_t launch_softdtw_fwd(int D, const SoftParams& p, int grid, int block, cudaStream_t st);
cudaError_t launch_softdtw_bwd(int D, const SoftParams& p, int grid, int block, cudaStream_t st);
int softdtw_max_blocks_per_sm(int D, int backward, int block, int banded = 0, int cost_kind = 0, int fused = 0,
                              int rows = 8);

// grad_B[i][c] = sum_k g[k] * gpart[k][i][c] (FP64 sum, k ascending); g == null
// takes g[k] = 1 / N_k (Eq. 7 with lambda_k = 1) from the cycle offsets
cudaError_t launch_softdtw_grad_reduce(const float* gpart, const float* g, const int64_t* offsets, int T, int64_t M,
                                       int d, float* grad_B, cudaStream_t st);

// One Adam step on n parameters (m, v: first / second moments, t >= 1).
cudaError_t launch_adam(float* x, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                        float beta2, float eps, int t, cudaStream_t st);

}  // namespace wts
