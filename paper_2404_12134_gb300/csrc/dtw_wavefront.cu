// Hard-min band wavefront for DTW (Eq. 1, computed by the recursion Eq. 5
// with gamma = 0; the alignment path of Definition "Alignment path").
//
//   r(0,0) = 0, r(i,0) = r(0,j) = +inf,
//   r(i,j) = delta(i,j) + min(r(i-1,j-1), r(i-1,j), r(i,j-1)),
//   delta(i,j) = sum_c (b_ic - y_jc)^2   (squared Euclidean local cost).
//
// Ties between predecessors resolve diag first, then up (i-1,j), then left
// (i,j-1); the CPU oracle takes the same decision in the same float
// arithmetic (subtract, then one fused multiply-add per channel from 0, then
// one add), so paths match bit for bit.
//
// One warp owns a band of 32*R rows of one pair; lane t holds R rows, their
// prototype samples and their last column of r in registers.  Lanes are
// skewed by one column (lane t is at column s - t in step s), so the value
// above a lane's first row comes from lane t-1 by __shfl_up_sync, and the
// cycle sample y_j enters at lane 0 and walks down the lanes with it.  Lane 0
// of band b > 0 reads the bottom row of band b-1 from a hand-off row in global
// memory (L2), 32 columns at a time, after the producer has published them.
// Each warp takes (pair, band) items in order from a global cursor, so the
// producer of any item it waits for was started earlier: no deadlock, with or
// without co-residency.  Every wait is bounded (wait_progress).
#include "dtw_wavefront.cuh"

namespace wts {

namespace {

template <int D, int R, int MODE>
__device__ __forceinline__ void run_band(const DPParams& p, const PairDesc& pd, int band, int lane)
{
    constexpr int BR = 32 * R;
    constexpr int W = R / 16;                      // direction words per lane per step
    const int M = pd.M, N = pd.N, d = p.d;
    const int i0 = band * BR + lane * R;
    const bool top = band == 0;
    const bool last = band == pd.nbands - 1;
    const float INF = inf_f();

    float b[R][D];
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int c = 0; c < D; ++c)
            b[k][c] = (i0 + k < M && c < d) ? __ldg(pd.X + (int64_t)(i0 + k) * d + c) : 0.f;

    float col[R];
    int cnt[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { col[k] = INF; cnt[k] = 0; }

    float y[D], ybuf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { y[c] = 0.f; ybuf[c] = 0.f; }

    float topv = INF;
    int topc = 0;
    // value and path count of r(i0-1, j-1) for the first row of this lane:
    // r(0,0) = 0 (0 cells) for the first row of the matrix, +inf otherwise
    float prev_up = (top && lane == 0) ? 0.f : INF;
    int prev_upc = 0;

    const float* hprev = top ? nullptr : p.hbuf + pd.hbuf_off + (int64_t)(band - 1) * N;
    float* hcur = last ? nullptr : p.hbuf + pd.hbuf_off + (int64_t)band * N;
    const int* cprev = (MODE == kModePlen && !top) ? p.hcnt + pd.hbuf_off + (int64_t)(band - 1) * N : nullptr;
    int* ccur = (MODE == kModePlen && !last) ? p.hcnt + pd.hbuf_off + (int64_t)band * N : nullptr;
    const int* fprev = top ? nullptr : p.flags + pd.flag_off + band - 1;
    int* fcur = p.flags + pd.flag_off + band;
    uint32_t* dout = (MODE == kModeDirs) ? p.dirs + pd.dir_off + (int64_t)band * (N + 31) * 32 * W : nullptr;

    const int steps = N + 31;
    for (int s = 0; s < steps; ++s) {
        if ((s & 31) == 0 && s < N) {
            // the next 32 columns of the lane-0 feeds: cycle samples and the
            // bottom row of the band above
            const int jj = s + lane;
#pragma unroll
            for (int c = 0; c < D; ++c)
                ybuf[c] = (jj < N && c < d) ? __ldg(pd.Y + (int64_t)jj * d + c) : 0.f;
            if (!top) {
                const int need = min(s + 32, N);
                if (!wait_progress(fprev, need, p.hdr, 1)) return;
                topv = jj < N ? __ldcg(hprev + jj) : INF;
                if (MODE == kModePlen) topc = jj < N ? __ldcg(cprev + jj) : 0;
            }
        }
        const int src = s & 31;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float fresh = __shfl_sync(FULL, ybuf[c], src);
            const float moved = __shfl_up_sync(FULL, y[c], 1);
            y[c] = lane == 0 ? fresh : moved;
        }
        const float above = __shfl_up_sync(FULL, col[R - 1], 1);
        const float tv = __shfl_sync(FULL, topv, src);
        const float up_in = lane == 0 ? (top ? INF : tv) : above;
        const float dg_in = prev_up;
        prev_up = up_in;
        int upc_in = 0, dgc_in = 0;
        if (MODE == kModePlen) {
            const int abovec = __shfl_up_sync(FULL, cnt[R - 1], 1);
            const int tc = __shfl_sync(FULL, topc, src);
            upc_in = lane == 0 ? tc : abovec;
            dgc_in = prev_upc;
            prev_upc = upc_in;
        }

        const int j = s - lane;
        uint32_t word[W > 0 ? W : 1];
#pragma unroll
        for (int w = 0; w < (W > 0 ? W : 1); ++w) word[w] = 0u;
        if (j >= 0 && j < N) {
            float dg = dg_in, up = up_in;
            int cdg = dgc_in, cup = upc_in;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float lf = col[k];
                float t = __fsub_rn(b[k][0], y[0]);
                float acc = __fmul_rn(t, t);
#pragma unroll
                for (int c = 1; c < D; ++c) {
                    t = __fsub_rn(b[k][c], y[c]);
                    acc = __fmaf_rn(t, t, acc);
                }
                const float m1 = fminf(up, lf);
                const float m = fminf(dg, m1);
                const float r = __fadd_rn(acc, m);
                if (MODE != kModeCost) {
                    const bool is_dg = dg <= m1;
                    const bool is_up = up <= lf;
                    if (MODE == kModeDirs) {
                        const uint32_t code = is_dg ? 0u : (is_up ? 1u : 2u);
                        word[k >> 4] |= code << (2 * (k & 15));
                    } else {
                        const int cl = cnt[k];
                        const int cn = 1 + (is_dg ? cdg : (is_up ? cup : cl));
                        cdg = cl;
                        cup = cn;
                        cnt[k] = cn;
                    }
                }
                dg = lf;
                up = r;
                col[k] = r;
            }
            if (hcur != nullptr && lane == 31) {
                __stcg(hcur + j, col[R - 1]);
                if (MODE == kModePlen) __stcg(ccur + j, cnt[R - 1]);
                if (((j + 1) & 31) == 0 || j == N - 1) st_release(fcur, j + 1);
            }
        }
        if (MODE == kModeDirs) {
            if (W == 1) {
                __stcs(dout + (int64_t)s * 32 + lane, word[0]);
            } else {
                uint2 v = make_uint2(word[0], word[W > 1 ? 1 : 0]);
                __stcs(reinterpret_cast<uint2*>(dout) + (int64_t)s * 32 + lane, v);
            }
        }
    }

    if (last) {
        const int ilast = M - 1 - band * BR;
        if (lane == ilast / R) {
            const int kk = ilast % R;
            float v = col[0];
            int c = cnt[0];
#pragma unroll
            for (int k = 1; k < R; ++k)
                if (k == kk) { v = col[k]; c = cnt[k]; }
            if (p.cost_out) p.cost_out[pd.out] = v;
            if (MODE == kModePlen) {
                if (p.plen_out) p.plen_out[pd.out] = c;
                if (p.score_out) p.score_out[pd.out] = __fdiv_rn(v, (float)c);
            }
            if (p.cost_matrix) {
                int a = 0, rem = pd.out;
                while (rem >= p.T - 1 - a) { rem -= p.T - 1 - a; ++a; }
                const int bb = a + 1 + rem;
                p.cost_matrix[(int64_t)a * p.T + bb] = v;
                p.cost_matrix[(int64_t)bb * p.T + a] = v;
            }
        }
    }
}

template <int D, int R, int MODE>
__global__ void __launch_bounds__(256) dtw_wavefront_kernel(DPParams p)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.hdr->item_counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= p.n_items) break;
        if (ld_volatile(&p.hdr->abort)) break;
        const int q = find_slot(p.prefix, p.P, item);
        const PairDesc pd = p.pairs[p.order[q]];
        run_band<D, R, MODE>(p, pd, item - p.prefix[q], lane);
    }
}

template <int D, int R>
cudaError_t launch_mode(int mode, const DPParams& p, int grid, int block, cudaStream_t st)
{
    switch (mode) {
        case kModeCost: dtw_wavefront_kernel<D, R, kModeCost><<<grid, block, 0, st>>>(p); break;
        case kModePlen: dtw_wavefront_kernel<D, R, kModePlen><<<grid, block, 0, st>>>(p); break;
        case kModeDirs: dtw_wavefront_kernel<D, R, kModeDirs><<<grid, block, 0, st>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int D, int R>
int occ_mode(int mode, int block)
{
    int n = 0;
    switch (mode) {
        case kModeCost: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dtw_wavefront_kernel<D, R, kModeCost>, block, 0); break;
        case kModePlen: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dtw_wavefront_kernel<D, R, kModePlen>, block, 0); break;
        case kModeDirs: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dtw_wavefront_kernel<D, R, kModeDirs>, block, 0); break;
        default: break;
    }
    return n;
}

}  // namespace

#define WTS_DISPATCH_DR(FN, ...)                                              \
    if (R == 16) {                                                           \
        switch (D) {                                                         \
            case 1: return FN<1, 16>(__VA_ARGS__);                           \
            case 2: return FN<2, 16>(__VA_ARGS__);                           \
            case 3: return FN<3, 16>(__VA_ARGS__);                           \
            case 4: return FN<4, 16>(__VA_ARGS__);                           \
            case 6: return FN<6, 16>(__VA_ARGS__);                           \
            case 8: return FN<8, 16>(__VA_ARGS__);                           \
            case 12: return FN<12, 16>(__VA_ARGS__);                         \
            case 16: return FN<16, 16>(__VA_ARGS__);                         \
            default: break;                                                  \
        }                                                                    \
    } else if (R == 32) {                                                    \
        switch (D) {                                                         \
            case 1: return FN<1, 32>(__VA_ARGS__);                           \
            case 2: return FN<2, 32>(__VA_ARGS__);                           \
            case 3: return FN<3, 32>(__VA_ARGS__);                           \
            default: break;                                                  \
        }                                                                    \
    }

cudaError_t launch_dtw_wavefront(int mode, int D, int R, const DPParams& p, int grid, int block, cudaStream_t st)
{
    WTS_DISPATCH_DR(launch_mode, mode, p, grid, block, st)
    return cudaErrorInvalidValue;
}

int dtw_wavefront_max_blocks_per_sm(int mode, int D, int R, int block)
{
    WTS_DISPATCH_DR(occ_mode, mode, block)
    return 0;
}

}  // namespace wts
