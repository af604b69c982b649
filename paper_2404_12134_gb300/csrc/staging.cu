// Batch staging (Sec. 3.1): time steps with a missing value (NaN in any
// channel) are removed and the cycles re-packed, giving the irregularly
// sampled series the alignment works on.
//
// keep[t] = no NaN in row t; pos = exclusive prefix sum of keep over the whole
// packed batch (block sums, one-block scan of the block sums, add back);
// out[pos[t]] = in[t] for kept rows; out_offsets[k] = pos[in_offsets[k]].
// Row order is preserved, so the result does not depend on scheduling.
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

}  // namespace

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
