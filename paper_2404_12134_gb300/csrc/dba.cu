// Backtrack of the tie-rule path, DBA averaging, and initial barycenters.
#include "dba.cuh"

namespace wts {

namespace {

constexpr int kBtWarps = 2;      // warps per backtrack CTA
constexpr int kBtWords = 4096;   // 16 KB of direction words cached per warp
constexpr long long kBtSpin = 1ll << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase)
{
    for (long long it = 0; it < kBtSpin; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(phase) : "memory");
        if (ok) return true;
    }
    return false;
}

// Walk the stored predecessor codes back from (M-1, N-1) to (0, 0).
// A cell (i, j) of band b sits in lane t = (i mod BR) / R at step s = j + t,
// as bit k = i mod R ("not diag") and bit R + k ("not up") of the lane's 2R
// code bits of that step.  For R >= 16 those are the W = R / 16 words at
// dirs[dir_off + b*(N+31)*32*W + (s*32 + t)*W + w]; for R = 8 and 4 the word
// dirs[dir_off + b*band_dir_words(N, R) + (s/S)*32 + t] holds the S = 32/(2R)
// steps S*(s/S) .. of the lane (2R bits each, the earliest in the lowest
// bits).  Along the walk s only decreases inside a
// band, so a window of kBtWords / 32 consecutive word rows (one contiguous
// block of global memory) is brought into shared memory by one bulk
// asynchronous copy (completion on an mbarrier, bounded wait) and the walk
// reads it; every lane walks the same path, and the lanes look ahead along a
// run of equal moves (one vote per run).
// Row i's range is [jlo(i), jhi(i)]: jhi when the walk enters the row, jlo
// when it leaves it (Definition "Alignment path": monotone, so each row's
// columns are contiguous).
template <int R>
__global__ void __launch_bounds__(32 * kBtWarps) backtrack_kernel(BTParams p)
{
    constexpr int W = R >= 16 ? R / 16 : 1;         // words per (word row, lane)
    constexpr int SPW = R >= 16 ? 1 : 32 / (2 * R); // steps per word row
    constexpr int LOG_R = R == 4 ? 2 : (R == 8 ? 3 : (R == 16 ? 4 : 5));
    constexpr int kBtRows = kBtWords / (32 * W);    // word rows of one band in the window
    __shared__ __align__(128) uint32_t win_all[kBtWarps][kBtWords];
    __shared__ __align__(8) uint64_t bars[kBtWarps];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    // the call's DP left early (a non-finite sample, or a wait that gave up):
    // its codes and b* were never written, so there is nothing to walk
    if (p.hdr != nullptr && ld_volatile(&p.hdr->abort)) return;
    uint32_t* win = win_all[wid];
    uint64_t* bar = &bars[wid];
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    uint32_t phase = 0;
    bool failed = false;
    const int units = p.nseg > 0 ? p.P * p.nseg : p.P;
    for (int u = blockIdx.x * kBtWarps + wid; u < units && !failed; u += gridDim.x * kBtWarps) {
        const int q = p.nseg > 0 ? u / p.nseg : u;
        const PairDesc pd = p.pairs[q];
        const int N = pd.N;
        int32_t* jlo = p.jlo + (int64_t)pd.out * p.M;
        int32_t* jhi = p.jhi + (int64_t)pd.out * p.M;
        int i, j, len;
        int i_lo = p.band_lo * 32 * R;
        int32_t* sg = p.nseg > 0 ? p.seg + 4 * (int64_t)u : nullptr;
        const int cur = p.round & 1;
        bool mergeable = false, merged = false;
        int prev_exit = -1;
        if (p.nseg > 0) {
            // segment sk: rows [sk * seg_rows, top]; the last one holds (M-1, N-1)
            const int sk = u - q * p.nseg;
            const int top = min(pd.M, (sk + 1) * p.seg_rows) - 1;
            i_lo = sk * p.seg_rows;
            int start;
            if (top == pd.M - 1) {
                if (p.round > 0) {                   // walked from the path's end in round 0
                    if (lane == 0) sg[1 + cur] = sg[2 - cur];
                    continue;
                }
                start = N - 1;
            } else if (p.round == 0) {
                // a guess: the column this row was entered at by the previous
                // walk of this pair (the ranges of an earlier call on the same
                // arrays; any value is safe), else the diagonal
                start = jhi[top];
                if (start < 0 || start >= N) start = (int)((int64_t)top * (N - 1) / max(pd.M - 1, 1));
            } else {
                start = p.seg[4 * (int64_t)(u + 1) + 2 - cur];     // exit of the segment above, last round
                if (start == sg[0]) {                // unchanged: the walk recorded stands
                    if (lane == 0) sg[1 + cur] = sg[2 - cur];
                    continue;
                }
            }
            if (start < 0 || start >= N) {           // the segment above failed
                if (lane == 0) { sg[0] = start; sg[1 + cur] = -1; sg[3] = 1; }
                continue;
            }
            // A re-walk (round > 0) stops where it enters the previous walk of
            // this segment, whose ranges the arrays hold: from a shared cell
            // the walks are the same.  Row top of that walk is [jlo(top), old
            // start].
            mergeable = p.round > 0 && sg[3] == 0;
            prev_exit = sg[2 - cur];
            if (mergeable && jlo[top] <= start && start <= sg[0]) {
                __syncwarp();
                if (lane == 0) { jhi[top] = start; sg[0] = start; sg[1 + cur] = prev_exit; }
                continue;
            }
            i = top; j = start; len = 0;
            if (lane == 0) { jhi[i] = j; sg[0] = start; }
        } else if (p.state == nullptr || p.first) {
            i = pd.M - 1; j = p.subseq ? p.bstar[pd.out] : N - 1; len = 0;
            if (j < 0 || j >= N) {                    // b* is not a column of this cycle: no walk
                if (lane == 0) {
                    if (p.astar) p.astar[pd.out] = -1;
                    if (p.plen) p.plen[pd.out] = -1;
                }
                continue;
            }
            if (lane == 0) jhi[i] = j;
        } else {
            i = p.state[3 * q]; j = p.state[3 * q + 1]; len = p.state[3 * q + 2];
            if (i < 0 || len < 0) continue;          // finished, or failed earlier
        }
        int band = -1, wlo = 0, whi = -1;           // word rows in the window
        bool left_group = false;
        for (;;) {
            ++len;
            if (i == 0 && j == 0) break;
            const int b = i >> (LOG_R + 5);
            const int row = (j + ((i >> LOG_R) & 31)) / SPW;     // word row of step s = j + t
            if (b != band || row < wlo || row > whi) {
                band = b;
                whi = row;
                wlo = max(0, row - kBtRows + 1);
                const uint32_t* src = p.dirs + pd.dir_off + (int64_t)(b - p.band_lo) * band_dir_words(N, R) +
                                      (int64_t)wlo * 32 * W;
                const uint32_t bytes = (uint32_t)(whi - wlo + 1) * 32 * W * 4;
                __syncwarp();
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                                 :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(smem_u32(win)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
                }
                const bool ok = mbar_wait(bar, phase);
                phase ^= 1u;
                if (!ok) {
                    // the copy did not land in time: give up on this pair,
                    // wait (bounded) for the copy still in flight, stop
                    mbar_wait(bar, phase ^ 1u);
                    len = -1;
                    failed = true;
                    break;
                }
            }
            // cell (ii, jj) of the window: lane t = (ii mod BR) / R, row k =
            // ii mod R, step s = jj + t; plane 0 ("not diag") is bit k, plane 1
            // ("not up") bit R + k of the step's code bits of lane t
            auto code_at = [&](int ii, int jj, uint32_t& nd, uint32_t& nu) {
                const int tt = (ii >> LOG_R) & 31;
                const int kk = ii & (R - 1);
                const int ss = jj + tt;
                const uint32_t* wp = win + ((ss / SPW - wlo) * 32 + tt) * W;
                const uint32_t w0 = R < 16 ? wp[0] >> ((ss % SPW) * 2 * R) : wp[0];
                nd = (w0 >> kk) & 1u;
                nu = R <= 16 ? (w0 >> (R + kk)) & 1u : (wp[W - 1] >> kk) & 1u;
            };
            uint32_t nd, nu;
            code_at(i, j, nd, nu);
            // codes: diag (nd = 0) moves up-left, up (nd = 1, nu = 0) moves up,
            // left (nd = nu = 1) moves left
            const int di = (nd == 0u || nu == 0u) ? 1 : 0;
            const int dj = (nd == 0u || nu == 1u) ? 1 : 0;
            // Sub-DTW: a move up from row 0 reaches the free start
            if (p.subseq && i == 0 && di) break;
            // a valid code matrix only moves left on row 0 and only up on
            // column 0; anything else is reported as |pi| = -1
            if ((i == 0 && di) || (j == 0 && dj)) { len = -1; break; }
            // Runs: lane u > 0 reads the cell c_u = (i - u di, j - u dj) that u
            // more moves of the same kind would reach, and agrees if that cell
            // is in the window, codes the same move, and the move from it is an
            // ordinary one (not the path's start, not out of the grid, not out
            // of the rows loaded).  The moves of c_0 .. c_{run-1} are then
            // taken at once, run = the first lane that does not agree: the same
            // walk as one cell at a time, with one shared-memory round trip and
            // one vote per run; lane u writes the rows that c_u leaves.
            const int iu = i - lane * di, ju = j - lane * dj;
            bool agree = false;
            if (lane > 0 && iu >= 0 && ju >= 0 && (iu | ju) != 0 && (iu >> (LOG_R + 5)) == band) {
                const int ru = (ju + ((iu >> LOG_R) & 31)) / SPW;
                if (ru >= wlo && ru <= whi) {
                    uint32_t ndu, nuu;
                    code_at(iu, ju, ndu, nuu);
                    const int diu = (ndu == 0u || nuu == 0u) ? 1 : 0;
                    const int dju = (ndu == 0u || nuu == 1u) ? 1 : 0;
                    agree = diu == di && dju == dj && !(iu == 0 && di) && !(ju == 0 && dj) && iu - di >= i_lo;
                }
            }
            const uint32_t votes = __ballot_sync(FULL, agree) | 1u;
            int run = votes == FULL ? 32 : __ffs(~votes) - 1;
            // a re-walk: does the move of c_u enter a row at a cell of the
            // previous walk (read before this run's writes)?
            uint32_t mv = 0u;
            if (mergeable) {                         // warp-uniform
                bool mg = false;
                if (di && lane < run && iu - 1 >= i_lo) {
                    const int je = ju - dj;
                    mg = jlo[iu - 1] <= je && je <= jhi[iu - 1];
                }
                mv = __ballot_sync(FULL, mg);
                if (mv) run = __ffs(mv);             // up to and including the first such move
            }
            if (di && lane < run) {
                jlo[iu] = ju;
                jhi[iu - 1] = ju - dj;
            }
            i -= run * di;
            j -= run * dj;
            len += run - 1;
            if (mv) { merged = true; break; }
            if (i < i_lo) { left_group = true; break; }    // the rest lies in bands not loaded
        }
        if (sg != nullptr) {
            if (lane == 0) {
                if (merged) {
                    sg[1 + cur] = prev_exit;          // the rest is the previous walk's
                } else {
                    sg[1 + cur] = left_group ? j : -1;    // the path's column in the row below
                    sg[3] = len < 0 ? 1 : 0;
                    if (!left_group && i == 0 && j == 0 && len > 0) jlo[0] = 0;
                }
            }
            continue;
        }
        if (left_group) {
            if (lane == 0) { p.state[3 * q] = i; p.state[3 * q + 1] = j; p.state[3 * q + 2] = len; }
            continue;
        }
        if (lane == 0) {
            if (p.subseq) {
                if (len > 0) jlo[0] = j;
                p.astar[pd.out] = len > 0 ? j : -1;
            } else if (i == 0 && j == 0 && len > 0) {
                jlo[0] = 0;
            }
            if (p.plen) p.plen[pd.out] = len;
            if (p.state) { p.state[3 * q] = -1; p.state[3 * q + 2] = len; }
        }
    }
}

// One warp per pair, after the last round of a segmented walk: the segments
// must join up (each one's start = the exit of the one above) and none may
// have failed; then |pi| = sum_i (jhi(i) - jlo(i) + 1), the cells of a monotone
// path being row by row contiguous.
__global__ void __launch_bounds__(128) bt_seg_final_kernel(BTParams p)
{
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (q >= p.P) return;
    if (p.hdr != nullptr && ld_volatile(&p.hdr->abort)) return;      // nothing was walked
    const PairDesc pd = p.pairs[q];
    const int last = (p.round & 1);                  // exit slot of the last round
    const int nseg = (int)((pd.M + p.seg_rows - 1) / p.seg_rows);
    bool bad = false;
    for (int k = lane; k < nseg; k += 32) {
        const int32_t* sg = p.seg + 4 * ((int64_t)q * p.nseg + k);
        if (sg[3] != 0) bad = true;
        if (k + 1 < nseg && sg[0] != p.seg[4 * ((int64_t)q * p.nseg + k + 1) + 1 + last]) bad = true;
    }
    bad = __any_sync(FULL, bad);
    const int32_t* jlo = p.jlo + (int64_t)pd.out * p.M;
    const int32_t* jhi = p.jhi + (int64_t)pd.out * p.M;
    long long cells = 0;
    for (int i = lane; i < pd.M; i += 32) cells += (long long)(jhi[i] - jlo[i] + 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cells += __shfl_xor_sync(FULL, cells, o);
    if (lane == 0 && p.plen) p.plen[pd.out] = bad ? -1 : (int32_t)cells;
}

// One thread per (prototype row i, channel c); the sum of channel c of row i
// is taken in double, cycles in ascending order, samples in ascending order,
// then one division and one rounding to float (the thread of channel 0 also
// writes the count).  The ranges of the next kPre cycles are loaded ahead so
// that the dependent range -> sample loads of successive cycles overlap.
constexpr int kPre = 8;

__global__ void __launch_bounds__(256) dba_average_kernel(const float* __restrict__ data,
                                                          const int64_t* __restrict__ offsets, int T, int d,
                                                          int64_t M, const int32_t* __restrict__ jlo,
                                                          const int32_t* __restrict__ jhi,
                                                          const float* __restrict__ costs, float* __restrict__ B_out,
                                                          int32_t* __restrict__ counts, double* cost_before)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < M * d) {
        const int64_t i = q / d;
        const int c = (int)(q - i * d);
        double acc = 0.0;
        int64_t cnt = 0;
        for (int k0 = 0; k0 < T; k0 += kPre) {
            int a[kPre], b[kPre];
            int64_t o[kPre];
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                const int k = k0 + u;
                if (k < T) {
                    o[u] = __ldg(offsets + k);
                    const int n = (int)(__ldg(offsets + k + 1) - o[u]);
                    // ranges come from the backtrack; clamping keeps every read
                    // inside the cycle even if a range were never written
                    a[u] = max(__ldg(jlo + (int64_t)k * M + i), 0);
                    b[u] = min(__ldg(jhi + (int64_t)k * M + i), n - 1);
                } else {
                    o[u] = 0; a[u] = 0; b[u] = -1;
                }
            }
            float first[kPre];
#pragma unroll
            for (int u = 0; u < kPre; ++u)
                first[u] = b[u] >= a[u] ? __ldg(data + (o[u] + a[u]) * d + c) : 0.f;
#pragma unroll
            for (int u = 0; u < kPre; ++u) {
                if (b[u] < a[u]) continue;
                acc = __dadd_rn(acc, (double)first[u]);
                for (int j = a[u] + 1; j <= b[u]; ++j)
                    acc = __dadd_rn(acc, (double)__ldg(data + (o[u] + j) * d + c));
                cnt += b[u] - a[u] + 1;
            }
        }
        B_out[q] = __double2float_rn(__ddiv_rn(acc, (double)(cnt > 0 ? cnt : 1)));
        if (counts && c == 0) counts[i] = (int32_t)cnt;
    }
    if (q == 0 && cost_before) {
        double s = 0.0;
        for (int k = 0; k < T; ++k) s = __dadd_rn(s, (double)costs[k]);
        *cost_before = s;
    }
}

__global__ void score_divide_kernel(const float* __restrict__ cost, const int32_t* __restrict__ plen,
                                    float* __restrict__ score, int T)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < T) {
        const int32_t c = plen[k];
        score[k] = c > 0 ? __fdiv_rn(cost[k], (float)c) : __int_as_float(0x7fc00000);
    }
}

// Linear resampling: p = m (N-1)/(M-1), i = floor(p), x_i + (p - i)(x_{i+1} - x_i),
// in double with every operation rounded separately, then rounded to float.
__device__ __forceinline__ float resample_at(const float* x, int64_t N, int d, int c, int64_t m, int64_t M)
{
    const double pos = M > 1 ? __ddiv_rn((double)(m * (N - 1)), (double)(M - 1)) : 0.0;
    int64_t i = (int64_t)floor(pos);
    if (i > N - 1) i = N - 1;
    const double f = __dsub_rn(pos, (double)i);
    const double xi = (double)x[i * d + c];
    double v = xi;
    if (i + 1 < N) v = __dadd_rn(xi, __dmul_rn(f, __dsub_rn((double)x[(i + 1) * d + c], xi)));
    return __double2float_rn(v);
}

__global__ void resample_kernel(const float* x, int64_t N, int d, float* out, int64_t M)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < M * d) out[q] = resample_at(x, N, d, (int)(q % d), q / d, M);
}

__global__ void euclid_mean_kernel(const float* data, const int64_t* offsets, int T, int d, int64_t M, float* out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M * d) return;
    const int c = (int)(q % d);
    const int64_t m = q / d;
    double acc = 0.0;
    for (int k = 0; k < T; ++k) {
        const int64_t o = offsets[k];
        acc = __dadd_rn(acc, (double)resample_at(data + o * d, offsets[k + 1] - o, d, c, m, M));
    }
    out[q] = __double2float_rn(__ddiv_rn(acc, (double)T));
}

// Row sums of the symmetric pairwise cost matrix in double (ascending column),
// then the first index of the smallest sum.
__global__ void medoid_kernel(const float* C, int T, int32_t* index_out, double* sums)
{
    for (int a = threadIdx.x; a < T; a += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < T; ++b) s = __dadd_rn(s, (double)C[(int64_t)a * T + b]);
        sums[a] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int a = 1; a < T; ++a)
            if (sums[a] < sums[best]) best = a;
        *index_out = best;
    }
}

}  // namespace

cudaError_t launch_backtrack(const BTParams& p, cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int units = p.nseg > 0 ? p.P * p.nseg : p.P;
    const int need = (units + kBtWarps - 1) / kBtWarps;
    const int cap = (p.nseg > 0 ? 8 : 4) * sms;
    const int grid = need < cap ? need : cap;
    if (p.R == 4) backtrack_kernel<4><<<grid, 32 * kBtWarps, 0, st>>>(p);
    else if (p.R == 8) backtrack_kernel<8><<<grid, 32 * kBtWarps, 0, st>>>(p);
    else if (p.R == 16) backtrack_kernel<16><<<grid, 32 * kBtWarps, 0, st>>>(p);
    else if (p.R == 32) backtrack_kernel<32><<<grid, 32 * kBtWarps, 0, st>>>(p);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_backtrack_seg_final(const BTParams& p, cudaStream_t st)
{
    const int warps = 4;
    bt_seg_final_kernel<<<(p.P + warps - 1) / warps, 32 * warps, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_dba_average(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               const int32_t* jlo, const int32_t* jhi, const float* costs,
                               float* B_out, int32_t* counts, double* cost_before, cudaStream_t st)
{
    const int block = 256;
    const int64_t n = M * d;
    const int grid = (int)((n + block - 1) / block);
    dba_average_kernel<<<grid, block, 0, st>>>(data, offsets, T, d, M, jlo, jhi, costs, B_out, counts, cost_before);
    return cudaGetLastError();
}

cudaError_t launch_score_divide(const float* cost, const int32_t* plen, float* score, int T, cudaStream_t st)
{
    score_divide_kernel<<<(T + 255) / 256, 256, 0, st>>>(cost, plen, score, T);
    return cudaGetLastError();
}

cudaError_t launch_resample(const float* x, int64_t N, int d, float* out, int64_t M, cudaStream_t st)
{
    const int64_t n = M * d;
    resample_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, N, d, out, M);
    return cudaGetLastError();
}

cudaError_t launch_euclid_mean(const float* data, const int64_t* offsets, int T, int d, int64_t M,
                               float* out, cudaStream_t st)
{
    const int64_t n = M * d;
    euclid_mean_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(data, offsets, T, d, M, out);
    return cudaGetLastError();
}

cudaError_t launch_medoid(const float* C, int T, int32_t* index_out, double* sums, cudaStream_t st)
{
    medoid_kernel<<<1, 256, 0, st>>>(C, T, index_out, sums);
    return cudaGetLastError();
}

}  // namespace wts
