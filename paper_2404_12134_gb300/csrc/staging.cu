// Batch staging (Sec. 3.1): time steps with a missing value (NaN in any
// channel) are removed and the cycles re-packed, giving the irregularly
// sampled series the alignment works on.
//
// keep[t] = no NaN in row t; pos = exclusive prefix sum of keep over the whole
// packed batch (block sums, one-block scan of the block sums, add back);
// out[pos[t]] = in[t] for kept rows; out_offsets[k] = pos[in_offsets[k]].
// Row order is preserved, so the result does not depend on scheduling.
//
// Two re-layouts for the paper's own forms of the data: last-value padding
// (Sec. 4.1: every cycle extended with its last sample to a common length, as
// the paper's Soft-DTW runs need) and the selection of one channel (the paper
// aligns, averages and scores each joint on its own, Sec. 5).
#include <cstdint>

#include <cuda_runtime.h>

#include "wts_common.cuh"

namespace wts {

namespace {

constexpr int kScanBlock = 1024;

__global__ void keep_kernel(const float* __restrict__ in, int64_t rows, int d, int64_t* __restrict__ pos,
                            int64_t* __restrict__ block_sums)
{
    __shared__ int64_t warp_tot[32];
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    int64_t keep = 0;
    if (t < rows) {
        keep = 1;
        for (int c = 0; c < d; ++c)
            if (isnan(in[t * d + c])) keep = 0;
    }
    // block-exclusive scan
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = keep;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    const int64_t excl = (wid ? warp_tot[wid - 1] : 0) + x - keep;
    if (t < rows) pos[t] = keep ? excl : -1 - excl;     // negative: dropped (encodes the position too)
    if (threadIdx.x == 0) block_sums[blockIdx.x] = warp_tot[31];
}

// One block: exclusive scan of the block sums, in place; total at [nblocks].
__global__ void scan_blocks_kernel(int64_t* block_sums, int64_t nblocks)
{
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t base = 0; base < nblocks; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < nblocks ? block_sums[i] : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int64_t w = warp_tot[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int64_t excl = carry + (wid ? warp_tot[wid - 1] : 0) + x - v;
        if (i < nblocks) block_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[nblocks] = carry;
}

__global__ void scatter_kernel(const float* __restrict__ in, int64_t rows, int d, const int64_t* __restrict__ pos,
                               const int64_t* __restrict__ block_sums, float* __restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * kScanBlock + threadIdx.x;
    if (t >= rows) return;
    const int64_t p = pos[t];
    if (p < 0) return;
    const int64_t o = block_sums[blockIdx.x] + p;
    for (int c = 0; c < d; ++c) out[o * d + c] = in[t * d + c];
}

__global__ void offsets_kernel(const int64_t* __restrict__ in_offsets, int T, int64_t rows,
                               const int64_t* __restrict__ pos, const int64_t* __restrict__ block_sums,
                               int64_t nblocks, int64_t* __restrict__ out_offsets)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > T) return;
    const int64_t t = in_offsets[k];
    if (t >= rows) { out_offsets[k] = block_sums[nblocks]; return; }
    const int64_t p = pos[t];
    const int64_t local = p >= 0 ? p : -1 - p;       // kept rows before t inside its block
    out_offsets[k] = block_sums[t / kScanBlock] + local;
}

// out[k][j][c] = in[offsets[k] + min(j, N_k - 1)][c]: one thread per output
// float, consecutive threads on consecutive floats (coalesced writes; the
// reads are the same rows, or the one last row, of one cycle).
__global__ void pad_last_kernel(const float* __restrict__ in, const int64_t* __restrict__ offsets, int T, int d,
                                int64_t L, float* __restrict__ out)
{
    const int64_t per = L * d;
    const int64_t n = per * T;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = q / per;
        const int64_t r = q - k * per;
        const int64_t j = r / d;
        const int c = (int)(r - j * d);
        const int64_t o = __ldg(offsets + k), N = __ldg(offsets + k + 1) - o;
        out[q] = __ldg(in + (o + (j < N ? j : N - 1)) * d + c);
    }
}

// out[t] = in[t][c] over every sample of the packed batch.
__global__ void select_channel_kernel(const float* __restrict__ in, int64_t rows, int d, int c,
                                      float* __restrict__ out)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < rows; t += (int64_t)gridDim.x * blockDim.x)
        out[t] = __ldg(in + t * d + c);
}

unsigned grid_for_elems(int64_t n)
{
    const int64_t g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

cudaError_t launch_pad_last(const float* in, const int64_t* offsets, int T, int d, int64_t L, float* out,
                            cudaStream_t st)
{
    pad_last_kernel<<<grid_for_elems(L * d * T), 256, 0, st>>>(in, offsets, T, d, L, out);
    return cudaGetLastError();
}

cudaError_t launch_select_channel(const float* in, int64_t rows, int d, int c, float* out, cudaStream_t st)
{
    select_channel_kernel<<<grid_for_elems(rows), 256, 0, st>>>(in, rows, d, c, out);
    return cudaGetLastError();
}

size_t compact_workspace_bytes(int64_t rows)
{
    const int64_t nblocks = (rows + kScanBlock - 1) / kScanBlock;
    return (size_t)(rows + nblocks + 1) * sizeof(int64_t);
}

cudaError_t launch_compact_nan(const float* in, const int64_t* in_offsets, int T, int d, int64_t rows, float* out,
                               int64_t* out_offsets, void* ws, cudaStream_t st)
{
    const int64_t nblocks = (rows + kScanBlock - 1) / kScanBlock;
    int64_t* pos = static_cast<int64_t*>(ws);
    int64_t* bsum = pos + rows;
    if (nblocks > 0) {
        keep_kernel<<<(unsigned)nblocks, kScanBlock, 0, st>>>(in, rows, d, pos, bsum);
    }
    scan_blocks_kernel<<<1, kScanBlock, 0, st>>>(bsum, nblocks);
    if (nblocks > 0) scatter_kernel<<<(unsigned)nblocks, kScanBlock, 0, st>>>(in, rows, d, pos, bsum, out);
    offsets_kernel<<<(T + 1 + 255) / 256, 256, 0, st>>>(in_offsets, T, rows, pos, bsum, nblocks, out_offsets);
    return cudaGetLastError();
}

}  // namespace wts
