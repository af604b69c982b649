// Setup kernel: per-pair descriptors, longest-first order and item prefix.
#include "plan.cuh"

namespace wts {

namespace {

constexpr int kSetupThreads = 1024;

// Exclusive block scan of one int64 per thread; returns the block total.
__device__ int64_t block_exclusive_scan(int64_t v, int64_t* out_excl)
{
    __shared__ int64_t warp_tot[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        warp_tot[lane] = w;            // inclusive over warps
    }
    __syncthreads();
    int64_t base = wid ? warp_tot[wid - 1] : 0;
    *out_excl = base + x - v;
    int64_t total = warp_tot[31];
    __syncthreads();
    return total;
}

__device__ void decode_pair(int p, int T, int* a, int* b)
{
    // pairs (a, b), a < b, enumerated a-major
    int aa = 0, rem = p;
    while (rem >= T - 1 - aa) { rem -= T - 1 - aa; ++aa; }
    *a = aa;
    *b = aa + 1 + rem;
}

__global__ void __launch_bounds__(kSetupThreads) setup_kernel(SetupParams sp)
{
    const int P = sp.P;
    // pass 1: descriptors and storage offsets in pair order
    int64_t run_h = 0, run_d = 0, run_r = 0;
    for (int base = 0; base < P; base += kSetupThreads) {
        const int p = base + threadIdx.x;
        PairDesc pd{};
        int64_t nb = 0, h = 0, dw = 0, rs = 0;
        if (p < P) {
            int64_t M, N;
            if (sp.op == kOpPairwise) {
                int a, b;
                decode_pair(p, sp.T, &a, &b);
                pd.X = sp.data + sp.offsets[a] * sp.d;
                M = sp.offsets[a + 1] - sp.offsets[a];
                pd.Y = sp.data + sp.offsets[b] * sp.d;
                N = sp.offsets[b + 1] - sp.offsets[b];
            } else {
                pd.X = sp.B;
                M = sp.M;
                pd.Y = sp.data + sp.offsets[p] * sp.d;
                N = sp.offsets[p + 1] - sp.offsets[p];
            }
            nb = cdiv(M, sp.BR);
            pd.M = (int32_t)M;
            pd.N = (int32_t)N;
            pd.nbands = (int32_t)nb;
            pd.out = p;
            pd.band_bound = band_bound_of(sp.band, M, N);
            h = pair_hbuf_slots(nb, N);
            if (sp.op == kOpAlign || sp.op == kOpDba || sp.op == kOpSubdtw)
                dw = pair_dir_words(sp.group_bands > 0 ? min((int64_t)sp.group_bands, nb) : nb, N, sp.R);
            if (sp.op == kOpSoft) {    // checkpoint mode: column checkpoints, or (band) two R buffers of groups
                if (sp.store_pairs > 0) {
                    // column checkpoints, but the first store_pairs pairs of the
                    // work list's order keep R (the rank as in pass 2)
                    int rank = p;
                    if (sp.sort) {
                        rank = 0;
                        for (int q = 0; q < P; ++q)
                            rank += longer_first(M * (sp.offsets[q + 1] - sp.offsets[q]), q, M * N, p);
                    }
                    pd.keep_r = rank < sp.store_pairs ? 1 : 0;
                }
                rs = sp.group_bands <= 0 || pd.keep_r ? pair_rstore_floats(nb, N, sp.R)
                     : sp.band > 0                    ? pair_rstore_floats(min(2 * (int64_t)sp.group_bands, nb), N, sp.R)
                                                      : nb * band_ckcol_floats(N, sp.R);
            }
        }
        int64_t eh, ed, er;
        int64_t th = block_exclusive_scan(h, &eh);
        int64_t td = block_exclusive_scan(dw, &ed);
        int64_t tr = block_exclusive_scan(rs, &er);
        if (p < P) {
            pd.hbuf_off = run_h + eh;
            pd.dir_off = run_d + ed;
            pd.aux_off = run_r + er;
            sp.pairs[p] = pd;
        }
        run_h += th; run_d += td; run_r += tr;
    }
    __syncthreads();
    // pass 2: order (longest first by cells, ties by index) via rank counting
    for (int p = threadIdx.x; p < P; p += kSetupThreads) {
        if (!sp.sort) { sp.order[p] = p; continue; }
        const int64_t cp = (int64_t)sp.pairs[p].M * sp.pairs[p].N;
        int rank = 0;
        for (int q = 0; q < P; ++q) rank += longer_first((int64_t)sp.pairs[q].M * sp.pairs[q].N, q, cp, p);
        sp.order[rank] = p;
    }
    __syncthreads();
    // pass 3: item prefix in that order
    int64_t run = 0;
    for (int base = 0; base < P; base += kSetupThreads) {
        const int q = base + threadIdx.x;
        int64_t nb = q < P ? sp.pairs[sp.order[q]].nbands : 0;
        int64_t ex;
        int64_t tot = block_exclusive_scan(nb, &ex);
        if (q < P) sp.prefix[q] = (int32_t)(run + ex);
        run += tot;
    }
    if (threadIdx.x == 0) sp.prefix[P] = (int32_t)run;
}

// true if the float with these bits is NaN or +-inf
__device__ __forceinline__ bool nonfinite_bits(uint32_t u) { return (u & 0x7f800000u) == 0x7f800000u; }

// Grid-stride scan of two arrays; 16-byte loads where the pointer allows.
__device__ bool scan_nonfinite(const float* x, int64_t n, int64_t tid, int64_t nthr)
{
    if (x == nullptr || n <= 0) return false;
    bool bad = false;
    const int64_t head = min(n, (int64_t)(((16 - ((uintptr_t)x & 15)) & 15) >> 2));
    for (int64_t i = tid; i < head; i += nthr) bad |= nonfinite_bits(__float_as_uint(x[i]));
    const int64_t n4 = (n - head) >> 2;
    const uint4* x4 = reinterpret_cast<const uint4*>(x + head);
    for (int64_t i = tid; i < n4; i += nthr) {
        const uint4 v = __ldcs(x4 + i);
        bad |= nonfinite_bits(v.x) | nonfinite_bits(v.y) | nonfinite_bits(v.z) | nonfinite_bits(v.w);
    }
    for (int64_t i = head + 4 * n4 + tid; i < n; i += nthr) bad |= nonfinite_bits(__float_as_uint(x[i]));
    return bad;
}

__global__ void __launch_bounds__(256) check_finite_kernel(const float* a, int64_t na, const float* b, int64_t nb,
                                                           WsHeader* hdr)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const bool bad = scan_nonfinite(a, na, tid, nthr) | scan_nonfinite(b, nb, tid, nthr);
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0) {
        atomicExch(&hdr->status, kDevBadInput);
        atomicExch(&hdr->abort, 1);
    }
}

}  // namespace

cudaError_t launch_check_finite(const float* a, int64_t na, const float* b, int64_t nb, WsHeader* hdr, int sms,
                                cudaStream_t st)
{
    const int64_t n = (na > 0 ? na : 0) + (nb > 0 ? nb : 0);
    int64_t blocks = (n / 4 + 255) / 256;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    check_finite_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, na, b, nb, hdr);
    return cudaGetLastError();
}

void launch_setup(const SetupParams& sp, cudaStream_t st)
{
    setup_kernel<<<1, kSetupThreads, 0, st>>>(sp);
}

}  // namespace wts
