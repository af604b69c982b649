// Soft-DTW on the band wavefront.
//
// Forward (Eqs. 3-5): r(i,j) = delta(i,j) + min^gamma(r(i-1,j-1), r(i-1,j), r(i,j-1)),
//   min^gamma(a,b,c) = m - gamma ln(sum exp(-(v - m)/gamma)),  m = min(a,b,c)
// (the exact rewrite of Eq. 3 with exp(-m/gamma) factored out).  The diagonal
// and left values are known before the row above is, so their part is taken
// first: with m2 = min(dg, lf), S2 = 1 + 2^(-|dg - lf| k) (k = log2(e)/gamma)
// and z = 2^(-|up - m2| k),
//   sum = S2 + z          (up >= m2, m = m2)
//   sum = S2 z + 1        (up <  m2, m = up)
// and min^gamma = m - (gamma ln 2) log2(sum), with the hardware ex2 / lg2
// approximations (flush-to-zero forms): two ex2 and one lg2 per cell, one ex2
// and the lg2 on the serial path down the rows.  Every r is stored (FP32) so
// the backward pass can read it.
//
// Backward (Eq. 6 with E from the reverse recursion of Cuturi and Blondel,
// which the paper cites): e(M,N) = 1 and
//   e(i,j) = sum over successors s of exp(((r(s) - r(i,j)) - delta(s)) / gamma) e(s),
// successors beyond the matrix contributing 0, then
//   d/db_ic sum_j ... = sum_j e(i,j) 2 (b_ic - y_jc)
// for the squared l2 local cost, and sum_j e(i,j) (b_ic - y_jc) / delta(i,j)
// (0 where delta = 0) for the l2 norm (COST = kCostL2: delta is the IEEE square
// root of the same sum).
// The difference r(s) - r(i,j) of neighbouring cells is taken first (exact in
// floating point when the two are within a factor of two), then delta(s) is
// subtracted: the exponent keeps the accuracy of the small quantity it is.
//
// Geometry is the hard-min kernel's: one warp per band of 32*R rows, lane t
// owns R rows.  Forward: lane t at column j = s - t in step s, bands top to
// bottom.  Backward: lane t at column j = N-1-s + (31-t) in step s (the lowest
// lane leads), bands bottom to top; the cell a lane needs at backward step s
// was written at forward step N+30-s by every lane, so each backward step
// reads one contiguous block of R.  R layout per band:
// [(N+31) steps][R/4][32 lanes][4 floats].
#include "softdtw.cuh"

#include <type_traits>

namespace wts {

namespace {

// 2^x and log2(x) by the MUFU approximations, flushing subnormals: a term
// below 2^-126 next to a sum of at least 1 changes nothing, and log2 is only
// taken of sums in [1, 3].  (The non-flushing forms cost extra instructions.)
__device__ __forceinline__ float ex2a(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ float lg2a(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 16-byte asynchronous global -> shared copies (L2 only), in commit groups
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Backward steps whose R blocks are in flight at once (shared-memory ring per warp)
constexpr int kRPre = 8;

// float4 words of shared memory per backward warp: the R ring (without a
// band followed by two chunks of hand-off slots and samples, 2 x (16 + 4D)
// bytes per lane), or (fused checkpoint mode) the kCk-step buffer and the
// staged inputs of the next recompute chunk (R + 2 + 2D floats per lane)
template <int D, int R>
__host__ __device__ constexpr int soft_warp_f4(bool fused, bool banded)
{
    return fused ? kCk * (R / 4) * 32 + (R + 2 + 2 * D) * 8 : kRPre * (R / 4) * 32 + (banded ? 0 : 64 + 16 * D);
}

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

template <int D, int R>
__device__ __forceinline__ void load_rows(float (&b)[R][D], const float* X, int i0, int M, int d)
{
#pragma unroll
    for (int k = 0; k < R; ++k)
#pragma unroll
        for (int c = 0; c < D; ++c)
            b[k][c] = (i0 + k < M && c < d) ? __ldg(X + (int64_t)(i0 + k) * d + c) : 0.f;
}

// delta(b_i, y_j): the squared l2 norm, or (COST = kCostL2) its IEEE square root
template <int D, int COST>
__device__ __forceinline__ float local_cost(const float* bk, const float* y, float* t)
{
    t[0] = __fsub_rn(bk[0], y[0]);
    float acc = __fmul_rn(t[0], t[0]);
#pragma unroll
    for (int c = 1; c < D; ++c) {
        t[c] = __fsub_rn(bk[c], y[c]);
        acc = __fmaf_rn(t[c], t[c], acc);
    }
    return COST == kCostL2 ? __fsqrt_rn(acc) : acc;
}

// One cell of the forward recursion: r = delta + min^gamma(dg, up, lf), the
// soft minimum taken relative to min(dg, lf) (see the file comment);
// kk = log2(e) / gamma, gl = gamma ln 2.  It is split in two: soft_pre takes
// what does not depend on r of the row above (delta, m2 = min(dg, lf) and
// S2 = 1 + 2^(-|dg - lf| kk)), soft_chain the rest.  A lane's rows form a
// serial chain through `up` within a step; computing every row's soft_pre
// before the chain keeps that work out of the chain's latency.
struct SoftPre {
    float delta, m2, S2;
};

template <int D, int COST>
__device__ __forceinline__ SoftPre soft_pre(const float* bk, const float* y, float dg, float lf, float kk)
{
    float t[D];
    SoftPre q;
    q.delta = local_cost<D, COST>(bk, y, t);
    q.m2 = fminf(dg, lf);
    q.S2 = __fadd_rn(1.f, ex2a(__fmul_rn(-fabsf(__fsub_rn(dg, lf)), kk)));
    return q;
}

__device__ __forceinline__ float soft_chain(const SoftPre& q, float up, float kk, float gl)
{
    const float du = __fsub_rn(up, q.m2);
    const float z = ex2a(__fmul_rn(-fabsf(du), kk));
    const float S = du >= 0.f ? __fadd_rn(q.S2, z) : __fmaf_rn(q.S2, z, 1.f);
    return __fmaf_rn(-gl, lg2a(S), __fadd_rn(q.delta, fminf(q.m2, up)));
}

// Column checkpoints (kCk, band_ckcol_floats: plan.cuh): chunk c of a band
// holds its lanes' state after forward step c kCk - 1 - the R rows of the
// lane's last column and r of the row above at the column before - so that
// the backward can recompute any kCk steps of the band on its own.

// One band of the forward pass; rslot: the band's slot in the R store (when
// store_r), recompute: start from the stored top row and write no hand-off row.
template <int D, int R, bool BANDED, int COST>
__device__ __forceinline__ void fwd_band(const SoftParams& p, const PairDesc& pd, int band, int lane, int rslot,
                                         bool recompute, bool store_r)
{
    constexpr int BR = 32 * R;
    const int M = pd.M, N = pd.N, d = p.d;
    const int i0 = band * BR + lane * R;
    const bool top = band == 0;
    const bool last = band == pd.nbands - 1;
    // r outside the matrix: a large finite value instead of +inf, so that the
    // difference of two such values is 0, not NaN (every cell of the matrix
    // has a finite neighbour, and 2^(-(1e30 - r) k) is 0 as 2^(-inf) is)
    const float INF = 1e30f;
    const float kk = kLog2e / p.gamma;
    const float gl = p.gamma * kLn2;

    float b[R][D];
    load_rows<D, R>(b, pd.X, i0, M, d);
    float col[R];
#pragma unroll
    for (int k = 0; k < R; ++k) col[k] = INF;
    float y[D], ybuf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { y[c] = 0.f; ybuf[c] = 0.f; }
    float topv = INF;
    float prev_up = (top && lane == 0) ? 0.f : INF;

    const float* hprev = top ? nullptr : p.hbuf + pd.hbuf_off + (int64_t)(band - 1) * N;
    float* hcur = (last || recompute || p.skip_handoff) ? nullptr : p.hbuf + pd.hbuf_off + (int64_t)band * N;
    // what the band keeps: every step's R (store_r), or every kCk steps its
    // lanes' state (the full forward in checkpoint mode without a band)
    const bool ck_mode = !BANDED && !store_r && p.ckcol != nullptr && !recompute;
    float* rs = store_r   ? p.rstore + pd.aux_off + (int64_t)rslot * (N + 31) * 32 * R
                : ck_mode ? p.ckcol + pd.aux_off + (int64_t)band * band_ckcol_floats(N, R) : nullptr;

    // Sakoe-Chiba band (as in the hard-min wavefront): the band's columns
    // [jlo, jhi], the row above's [jtop_lo, jtop_hi] (the only columns its
    // producer writes), and the lane's columns with every row inside
    const int64_t bnd = BANDED ? pd.band_bound : -1;
    int jlo = 0, jhi = N - 1, jtop_lo = 0, jtop_hi = N - 1, full_lo = 0, full_hi = N - 1;
    if (BANDED) {
        const int64_t r0 = (int64_t)band * BR, r1 = min(r0 + BR, (int64_t)M) - 1;
        jlo = band_lo(r0, bnd, M, N);
        jhi = band_hi(r1, bnd, M, N);
        if (!top) { jtop_lo = band_lo(r0 - 1, bnd, M, N); jtop_hi = band_hi(r0 - 1, bnd, M, N); }
        if (i0 < M) { full_lo = band_lo(min(i0 + R - 1, M - 1), bnd, M, N); full_hi = band_hi(i0, bnd, M, N); }
    }
    // from a multiple of 32 at or before jlo - 1 (lane 0's first diagonal is
    // the row above one column before the band starts)
    const int s_begin = BANDED ? max(0, (jlo - 1) & ~31) : 0;
    const int s_end = BANDED ? jhi + 32 : N + 31;
    // the lane's rows inside the band at its column s - lane, kept step by step
    BandRows brow{};
    if (BANDED) brow.init(s_begin - lane, bnd, M, N);

    // lane-0 feeds one chunk of 32 columns ahead (the top row is NaN until written)
    float ynext[D];
    float tnext = INF;
    auto load_y = [&](int jj) {
#pragma unroll
        for (int c = 0; c < D; ++c) ynext[c] = (jj < N && c < d) ? __ldg(pd.Y + (int64_t)jj * d + c) : 0.f;
    };
    load_y(s_begin + lane);
    if (!top && s_begin + lane < N) tnext = __ldcv(hprev + s_begin + lane);

#pragma unroll 2
    for (int s = s_begin; s < s_end; ++s) {
        if (ck_mode && s > 0 && (s % kCk) == 0) {
            float* ck = rs + (int64_t)(s / kCk) * (R + 1) * 32 + lane;
#pragma unroll
            for (int k = 0; k < R; ++k) ck[k * 32] = col[k];
            ck[R * 32] = prev_up;
        }
        if ((s & 31) == 0 && s <= jhi) {
            const int jj = s + lane;
#pragma unroll
            for (int c = 0; c < D; ++c) ybuf[c] = ynext[c];
            if (!top) {
                const bool need = jj >= jtop_lo && jj <= jtop_hi;
                float t = tnext;
                const bool ok = wait_filled(need && isnan(t), [&]() { t = __ldcv(hprev + jj); return isnan(t); },
                                            p.hdr, 3, p.spin_limit);
                if (!ok) return;
                topv = need ? t : INF;
                tnext = jj + 32 < N ? __ldcv(hprev + jj + 32) : INF;
            }
            load_y(jj + 32);
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

        const int j = s - lane;
        // the lane's column; MASK: only rows k in [klo, khi] lie in the band
        auto column = [&](auto mask) {
            constexpr bool MASK = decltype(mask)::value;
            const int klo = MASK ? brow.qa - i0 : 0, khi = MASK ? brow.qb - i0 : R - 1;
            SoftPre q[R];
#pragma unroll
            for (int k = 0; k < R; ++k) q[k] = soft_pre<D, COST>(b[k], y, k == 0 ? dg_in : col[k - 1], col[k], kk);
            float up = up_in;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                float r = soft_chain(q[k], up, kk, gl);
                if (MASK && (k < klo || k > khi)) r = INF;      // outside the band
                up = r;
                col[k] = r;
            }
        };
        if (j >= jlo && j <= jhi) {
            if (BANDED && (j < full_lo || j > full_hi))
                column(std::true_type{});
            else
                column(std::false_type{});
            // NaN (from finite samples whose squared differences overflow) is
            // stored as -inf: a slot is NaN only while it is unwritten
            if (hcur != nullptr && lane == 31) __stcg(hcur + j, fmaxf(col[R - 1], -inf_f()));
        }
        if (store_r) {
            float4* dst = reinterpret_cast<float4*>(rs + (int64_t)s * 32 * R);
#pragma unroll
            for (int k4 = 0; k4 < R / 4; ++k4)
                dst[k4 * 32 + lane] = make_float4(col[4 * k4], col[4 * k4 + 1], col[4 * k4 + 2], col[4 * k4 + 3]);
        }
        if (BANDED) brow.next(N);
    }

    if (last && !recompute) {
        const int ilast = M - 1 - band * BR;
        if (lane == ilast / R) {
            const int kk2 = ilast % R;
            float v = col[0];
#pragma unroll
            for (int k = 1; k < R; ++k)
                if (k == kk2) v = col[k];
            p.value_out[pd.out] = v;
        }
    }
}

// FUSED (checkpoint mode without a band): R is not stored; every kCk
// backward steps the warp recomputes the kCk forward steps they read from the
// band's column checkpoint into `ring` (kCk blocks of R/4 x 32 float4: each
// lane writes and later reads only its own rows, so no synchronisation).
// ALIGNED (no band, M a multiple of R): a lane's rows lie all inside the
// matrix or all past it, so every column runs unchecked: the lanes past the
// matrix skip their columns (their state stays (-inf, 0, 0), what the lane
// above must see below the last row), and the seed e(M-1, N-1) = 1 enters as
// a diagonal successor with r(M-1, N-1), delta 0 and e = 1 (its weight
// 2^0 = 1): the same e, bit for bit, without the checked column's registers.
template <int D, int R, bool BANDED, int COST, bool FUSED, bool ALIGNED = false>
__device__ __forceinline__ void bwd_band(const SoftParams& p, const PairDesc& pd, int band, int lane, float4* ring,
                                         int rslot)
{
    constexpr int BR = 32 * R;
    const int M = pd.M, N = pd.N, d = p.d;
    const int i0 = band * BR + lane * R;
    const bool top = band == 0;
    const bool last = band == pd.nbands - 1;
    const float NINF = -inf_f();
    const float kk = kLog2e / p.gamma;

    float b[R][D];
    load_rows<D, R>(b, pd.X, i0, M, d);
    // lanes whose rows reach the matrix's last row (or pass it); ALIGNED: the
    // lane whose last row is the matrix's
    const bool edge = last && i0 + R >= M;
    const bool seed_lane = last && i0 + R == M;
    // state of each row at the column to the right (r, delta k, e) with
    // k = log2(e) / gamma; beyond the matrix: (-inf, 0, 0)
    float rp[R], dp[R], ep[R];
    float g[R][D];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        rp[k] = NINF; dp[k] = 0.f; ep[k] = 0.f;
#pragma unroll
        for (int c = 0; c < D; ++c) g[k][c] = 0.f;
    }
    float y[D], ybuf[D];
#pragma unroll
    for (int c = 0; c < D; ++c) { y[c] = 0.f; ybuf[c] = 0.f; }
    float cr = NINF, cd = 0.f, ce = 0.f;          // chunk of the row below the band
    float pbr = NINF, pbd = 0.f, pbe = 0.f;       // row below, one column to the right

    // boundary slot b holds the top row of band b+1: per column two 8-byte
    // words {r, delta k} and {e, 0}, each NaN until written
    const u64* enext = last ? nullptr : reinterpret_cast<const u64*>(p.ebuf) + 2 * (pd.hbuf_off + (int64_t)band * N);
    u64* emine = (top || p.skip_handoff) ? nullptr
                                         : reinterpret_cast<u64*>(p.ebuf) + 2 * (pd.hbuf_off + (int64_t)(band - 1) * N);
    const float* rs = FUSED ? nullptr : p.rstore + pd.aux_off + (int64_t)rslot * (N + 31) * 32 * R;

    // Sakoe-Chiba band: the band's columns [jlo, jhi], the row below's
    // [jbot_lo, jbot_hi] (the only columns its producer waits for here), the
    // lane's columns with every row inside.  Lane t is at column
    // N-1-s+(31-t): steps from a multiple of 32 at or before the step where
    // lane 31 is one column right of jhi (its first below-right value), to the
    // step where lane 0 reaches jlo.
    const int64_t bnd = BANDED ? pd.band_bound : -1;
    int jlo = 0, jhi = N - 1, jbot_lo = 0, jbot_hi = N - 1, full_lo = 0, full_hi = N - 1;
    if (BANDED) {
        const int64_t r0 = (int64_t)band * BR, r1 = min(r0 + BR, (int64_t)M) - 1;
        jlo = band_lo(r0, bnd, M, N);
        jhi = band_hi(r1, bnd, M, N);
        if (!last) { jbot_lo = band_lo(r1 + 1, bnd, M, N); jbot_hi = band_hi(r1 + 1, bnd, M, N); }
        if (i0 < M) { full_lo = band_lo(min(i0 + R - 1, M - 1), bnd, M, N); full_hi = band_hi(i0, bnd, M, N); }
    }
    const int s_begin = BANDED ? max(0, (N - 2 - jhi) & ~31) : 0;
    const int steps = BANDED ? N + 31 - jlo : N + 31;
    // the lane's rows inside the band at its column N-1-s+(31-lane)
    BandRows brow{};
    if (BANDED) brow.init(N - 1 - s_begin + (31 - lane), bnd, M, N);

    // R of this lane's rows at the column of step ss (written by forward step
    // N+30-ss) is copied into ring slot ss mod kRPre kRPre steps ahead of its
    // use (one commit group per step, empty past the end), so that a step's
    // wait covers the copies issued kRPre steps earlier
    // (without a band every lane's slot of every step exists, as the forward
    // stores all N + 31 steps: no range check, and the source walks down one
    // step of R per call)
    const float4* rsrc = (FUSED || BANDED)
                             ? nullptr
                             : reinterpret_cast<const float4*>(rs + (int64_t)(N + 30 - s_begin) * 32 * R) + lane;
    auto issue_r = [&](int ss) {
        if (FUSED) return;
        if (!BANDED) {
            if (ss < steps) {
                float4* dst = ring + (ss & (kRPre - 1)) * (R / 4) * 32 + lane;
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4) cp_async16(dst + k4 * 32, rsrc + k4 * 32);
            }
            rsrc -= (R / 4) * 32;
        } else {
            const int jj = N - 1 - ss + (31 - lane);
            if (ss < steps && jj >= jlo && jj <= jhi) {
                const float4* src4 = reinterpret_cast<const float4*>(rs + (int64_t)(N + 30 - ss) * 32 * R);
                float4* dst = ring + (ss & (kRPre - 1)) * (R / 4) * 32;
#pragma unroll
                for (int k4 = 0; k4 < R / 4; ++k4) cp_async16(dst + k4 * 32 + lane, src4 + k4 * 32 + lane);
            }
        }
        cp_async_commit();
    };

    // FUSED: recompute forward steps [f0, f1) of this band into `ring` from
    // the column checkpoint (the same cell arithmetic and inputs as the full
    // forward, so R is bit-identical); the band's top row comes from the
    // forward's hand-off rows, all written before this launch
    const float* ckb = FUSED ? p.ckcol + pd.aux_off + (int64_t)band * band_ckcol_floats(N, R) : nullptr;
    const float* hprev = (FUSED && !top) ? p.hbuf + pd.hbuf_off + (int64_t)(band - 1) * N : nullptr;
    const float FINF = 1e30f;                      // the forward's finite sentinel
    // A chunk's inputs (the checkpoint's R + 1 values, the samples of its first
    // column and of its 32-column block, the top row's value) are staged in
    // shared memory by asynchronous copies one chunk ahead, after the kCk-step
    // buffer: kStage floats per lane, [value][lane]
    float* stage = FUSED ? reinterpret_cast<float*>(ring + kCk * (R / 4) * 32) + lane : nullptr;
    auto stage_chunk = [&](int f0) {
        if (f0 == 0) {
#pragma unroll
            for (int k = 0; k < R; ++k) stage[k * 32] = FINF;
            stage[R * 32] = (top && lane == 0) ? 0.f : FINF;
        } else {
            const float* ck = ckb + (int64_t)(f0 / kCk) * (R + 1) * 32 + lane;
#pragma unroll
            for (int k = 0; k <= R; ++k) cp_async4(stage + k * 32, ck + k * 32);
        }
        const int jy = f0 - 1 - lane, fb = f0 & ~31;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float* a = stage + (R + 1 + c) * 32;
            float* bq = stage + (R + 1 + D + c) * 32;
            if (jy >= 0 && jy < N && c < d) cp_async4(a, pd.Y + (int64_t)jy * d + c); else *a = 0.f;
            if (fb + lane < N && c < d) cp_async4(bq, pd.Y + (int64_t)(fb + lane) * d + c); else *bq = 0.f;
        }
        float* tq = stage + (R + 1 + 2 * D) * 32;
        if (top || fb + lane >= N) *tq = FINF; else cp_async4(tq, hprev + fb + lane);
        cp_async_commit();
    };
    auto recompute = [&](int f0, int f1, bool first) {
        const float gl = p.gamma * kLn2;
        if (first) stage_chunk(f0);
        cp_async_wait<0>();
        float fcol[R];
#pragma unroll
        for (int k = 0; k < R; ++k) fcol[k] = stage[k * 32];
        float fprev = stage[R * 32];
        float fy[D], fyb[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            fy[c] = stage[(R + 1 + c) * 32];
            fyb[c] = stage[(R + 1 + D + c) * 32];
        }
        const float ftop = stage[(R + 1 + 2 * D) * 32];
        if (f0 >= kCk) stage_chunk(f0 - kCk);        // the next chunk down, while this one runs
        for (int ff = f0; ff < f1; ++ff) {
            const int src = ff & 31;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const float fresh = __shfl_sync(FULL, fyb[c], src);
                const float moved = __shfl_up_sync(FULL, fy[c], 1);
                fy[c] = lane == 0 ? fresh : moved;
            }
            const float above = __shfl_up_sync(FULL, fcol[R - 1], 1);
            const float tv = __shfl_sync(FULL, ftop, src);
            const float up_in = lane == 0 ? (top ? FINF : tv) : above;
            const float dg_in = fprev;
            fprev = up_in;
            const int jf = ff - lane;
            if (jf >= 0 && jf < N) {
                SoftPre q[R];
#pragma unroll
                for (int k = 0; k < R; ++k)
                    q[k] = soft_pre<D, COST>(b[k], fy, k == 0 ? dg_in : fcol[k - 1], fcol[k], kk);
                float up = up_in;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float r = soft_chain(q[k], up, kk, gl);
                    up = r;
                    fcol[k] = r;
                }
            }
            float4* dst = ring + (ff - f0) * (R / 4) * 32;
#pragma unroll
            for (int k4 = 0; k4 < R / 4; ++k4)
                dst[k4 * 32 + lane] = make_float4(fcol[4 * k4], fcol[4 * k4 + 1], fcol[4 * k4 + 2], fcol[4 * k4 + 3]);
        }
    };
    // lane-31 feeds one chunk ahead: lane l holds column N-1-s-l.  With R
    // stored and no band, each chunk's hand-off slots (16 B: r, delta k, e) and samples are
    // copied by cp.async, one chunk ahead and in the step's commit group, into
    // one of two shared-memory buffers after the R ring, and read there every
    // step by lane 31 (the ring's wait seven groups behind has them complete
    // long before their chunk starts); no register holds a chunk, which lets
    // the one-channel loop without a band be unrolled by two within 96
    // registers (the column state then alternates registers instead of being
    // copied each step).  Fused or banded, the chunks are loaded into registers
    // and broadcast by shuffles.
    constexpr bool SPF = !FUSED && !BANDED;
    float4* ech = SPF ? ring + kRPre * (R / 4) * 32 : nullptr;           // [2][32]
    float* ych = SPF ? reinterpret_cast<float*>(ech + 64) : nullptr;    // [2][D][32]
    float ynext[D];
    u64 wa = 0, wb = 0;
    auto load_y = [&](int jj, int buf) {
#pragma unroll
        for (int c = 0; c < D; ++c) {
            if (SPF) {
                float* dst = ych + (buf * D + c) * 32 + lane;
                if (jj >= 0 && c < d) cp_async4(dst, pd.Y + (int64_t)jj * d + c);
                else *dst = 0.f;
            } else {
                ynext[c] = (jj >= 0 && c < d) ? __ldg(pd.Y + (int64_t)jj * d + c) : 0.f;
            }
        }
    };
    auto load_e = [&](int jj, int buf) {
        if (jj >= 0) {
            if (SPF) {
                cp_async16(ech + buf * 32 + lane, enext + 2 * jj);
            } else {
                wa = __ldcv(enext + 2 * jj);
                wb = __ldcv(enext + 2 * jj + 1);
            }
        }
    };
    load_y(N - 1 - s_begin - lane, (s_begin >> 5) & 1);
    if (!last) load_e(N - 1 - s_begin - lane, (s_begin >> 5) & 1);
    // the first chunk's group, then the ring's first kRPre steps: the first
    // step's wait (all but the newest kRPre - 1 groups) covers both
    if (SPF) cp_async_commit();
    if (!FUSED)
#pragma unroll 1
        for (int ss = s_begin; ss < s_begin + kRPre; ++ss) issue_r(ss);

#pragma unroll(D == 1 && !BANDED && !FUSED ? 2 : 1)
    for (int s = s_begin; s < steps; ++s) {
        float4 rcur[R / 4];
        if (FUSED) {
            // forward step f of this backward step; a new chunk of kCk forward
            // steps (read backwards) starts at its last step
            const int f = N + 30 - s;
            const int fr = f % kCk;
            if (s == s_begin || fr == kCk - 1) recompute(f - fr, min(f - fr + kCk, N + 31), s == s_begin);
#pragma unroll
            for (int k4 = 0; k4 < R / 4; ++k4) rcur[k4] = ring[fr * (R / 4) * 32 + k4 * 32 + lane];
        } else {
            cp_async_wait<kRPre - 1>();
#pragma unroll
            for (int k4 = 0; k4 < R / 4; ++k4) rcur[k4] = ring[(s & (kRPre - 1)) * (R / 4) * 32 + k4 * 32 + lane];
        }
        const int cbuf = (s >> 5) & 1;
        if ((s & 31) == 0 && s < N) {
            const int jj = N - 1 - s - lane;
            if (!SPF) {
#pragma unroll
                for (int c = 0; c < D; ++c) ybuf[c] = ynext[c];
            }
            if (!last) {
                // only the row below's columns inside the band are written (and
                // waited for); a slot found unwritten is polled from global memory
                const bool need = jj >= jbot_lo && jj <= jbot_hi;
                if (SPF && need) {
                    const float4 v = ech[cbuf * 32 + lane];
                    wa = pack2(v.x, v.y);
                    wb = pack2(v.z, v.w);
                }
                bool polled = false;
                const bool ok = wait_filled(need && (is_nan_bits((uint32_t)wa) || is_nan_bits((uint32_t)wb)),
                                            [&]() {
                                                wa = __ldcv(enext + 2 * jj);
                                                wb = __ldcv(enext + 2 * jj + 1);
                                                polled = true;
                                                return is_nan_bits((uint32_t)wa) || is_nan_bits((uint32_t)wb);
                                            },
                                            p.hdr, 4, p.spin_limit);
                if (!ok) {
                    cp_async_wait<0>();
                    return;
                }
                if (need) {
                    cr = __uint_as_float((uint32_t)wa);
                    cd = __uint_as_float((uint32_t)(wa >> 32));
                    ce = __uint_as_float((uint32_t)wb);
                } else {
                    cr = NINF; cd = 0.f; ce = 0.f;
                }
                if (SPF && (polled || !need)) ech[cbuf * 32 + lane] = make_float4(cr, cd, ce, 0.f);
            }
            if (SPF) {
                // this chunk's slots visible to lane 31, the other buffer's last
                // chunk read by every lane, before the next chunk's copies
                __syncwarp();
                if (!last) load_e(jj - 32, cbuf ^ 1);
            } else if (!last) {
                load_e(jj - 32, 0);
            }
            load_y(jj - 32, cbuf ^ 1);
        }
        const int src = s & 31;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const float fresh = SPF ? ych[(cbuf * D + c) * 32 + src] : __shfl_sync(FULL, ybuf[c], src);
            const float moved = __shfl_down_sync(FULL, y[c], 1);
            y[c] = lane == 31 ? fresh : moved;
        }
        float br = __shfl_down_sync(FULL, rp[0], 1);
        float bd = __shfl_down_sync(FULL, dp[0], 1);
        float be = __shfl_down_sync(FULL, ep[0], 1);
        float fr, fd, fe;
        if (SPF) {
            const float4 v = last ? make_float4(NINF, 0.f, 0.f, 0.f) : ech[cbuf * 32 + src];
            fr = v.x; fd = v.y; fe = v.z;
        } else {
            fr = __shfl_sync(FULL, cr, src);
            fd = __shfl_sync(FULL, cd, src);
            fe = __shfl_sync(FULL, ce, src);
        }
        if (lane == 31) {
            br = last ? NINF : fr;
            bd = last ? 0.f : fd;
            be = last ? 0.f : fe;
        }
        float xr = pbr, xd = pbd, xe = pbe;        // below, column j+1
        pbr = br; pbd = bd; pbe = be;
        if (ALIGNED && seed_lane && s == 31 - lane) {  // this lane's first column, j = N-1
            xr = rcur[R / 4 - 1].w;
            xd = 0.f;
            xe = 1.f;
        }

        const int j = N - 1 - s + (31 - lane);
        // one column of the lane's rows, bottom to top; CHECKED: rows past the
        // matrix and the seed e(M-1, N-1) = 1 (only the lanes at the matrix's
        // last rows, and only at column N-1, take that path)
        auto column = [&](auto checked) {
            constexpr bool CHECKED = decltype(checked)::value;
            // checked with a band: only rows k in [klo, khi] lie in the band
            const int klo = CHECKED && BANDED ? brow.qa - i0 : 0;
            const int khi = CHECKED && BANDED ? brow.qb - i0 : R - 1;
            float nr = br, nd = bd, ne = be;       // below, column j
#pragma unroll
            for (int k4 = R / 4 - 1; k4 >= 0; --k4) {
                const float4 v4 = rcur[k4];
                const float rv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int kq = 3; kq >= 0; --kq) {
                    const int k = 4 * k4 + kq;
                    const float rr = rp[k], rd = dp[k], re = ep[k];
                    float rn = NINF, dn = 0.f, en = 0.f;
                    if (!CHECKED || (i0 + k < M && k >= klo && k <= khi)) {
                        const float r = rv[kq];
                        float t[D];
                        const float delta = local_cost<D, COST>(b[k], y, t);
                        // successor s: 2^((r(s) - r) k - delta(s) k), the difference
                        // exact, then one fused multiply-add with delta(s) k kept per cell
                        const float a = ex2a(__fmaf_rn(__fsub_rn(nr, r), kk, -nd));
                        const float bb = ex2a(__fmaf_rn(__fsub_rn(rr, r), kk, -rd));
                        const float cc = ex2a(__fmaf_rn(__fsub_rn(xr, r), kk, -xd));
                        // the row below's e (ne) is the only input computed in
                        // this step: it enters last, so the serial chain down the
                        // rows is one fused multiply-add per row
                        float e = __fmaf_rn(a, ne, __fmaf_rn(cc, xe, __fmul_rn(bb, re)));
                        if (CHECKED && i0 + k == M - 1 && j == N - 1) e = 1.f;
                        if (COST != kCostL2) {
#pragma unroll
                            for (int c = 0; c < D; ++c) g[k][c] = __fmaf_rn(e, t[c], g[k][c]);
                        } else {
                            // d delta / d b = t / delta (0 where delta = 0), an IEEE division
                            const float w = delta > 0.f ? __fdiv_rn(e, delta) : 0.f;
#pragma unroll
                            for (int c = 0; c < D; ++c) g[k][c] = __fmaf_rn(w, t[c], g[k][c]);
                        }
                        rn = r; dn = __fmul_rn(delta, kk); en = e;
                    }
                    xr = rr; xd = rd; xe = re;
                    nr = rn; nd = dn; ne = en;
                    rp[k] = rn; dp[k] = dn; ep[k] = en;
                }
            }
        };
        if (j >= jlo && j <= jhi && (!ALIGNED || i0 < M)) {
            if (ALIGNED)
                column(std::false_type{});
            else if ((edge && (i0 + R > M || j == N - 1)) || (BANDED && (j < full_lo || j > full_hi)))
                column(std::true_type{});
            else
                column(std::false_type{});
            if (emine != nullptr && lane == 0) {
                // (NaN from overflowing samples stored as -inf, as in the forward)
                __stcg(emine + 2 * j, pack2(fmaxf(rp[0], NINF), dp[0]));
                __stcg(emine + 2 * j + 1, pack2(fmaxf(ep[0], NINF), 0.f));
            }
        }
        // the slot just read (its values are consumed) takes step s + kRPre
        issue_r(s + kRPre);
        if (BANDED) brow.prev(N);
    }
    cp_async_wait<0>();

    float* gout = p.gpart + (int64_t)pd.out * M * d;
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (i0 + k < M)
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (c < d) gout[(int64_t)(i0 + k) * d + c] = COST == kCostL2 ? g[k][c] : __fmul_rn(2.f, g[k][c]);
}

// The persistent item loop shared by the kernels below.
template <int D, int R, bool BWD, bool BANDED, int COST, bool FUSED, bool ALIGNED = false>
__device__ __forceinline__ void soft_items(const SoftParams& p)
{
    extern __shared__ float4 rring_all[];
    const int lane = threadIdx.x & 31;
    const int n_all = p.n_items + (BWD ? p.n_rec : 0);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.hdr->item_counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= n_all) break;
        if (ld_volatile(&p.hdr->abort)) break;
        if (BWD && item >= p.n_items) {
            // recompute of the next group up, beside this group's backward
            const int r = item - p.n_items;
            const int qr = r / p.rec_band_cnt, kr = r % p.rec_band_cnt;
            const PairDesc pr = p.pairs[p.order[qr]];
            fwd_band<D, R, BANDED, COST>(p, pr, p.rec_band_lo + kr, lane, p.rec_rbuf_band0 + kr, true, true);
            continue;
        }
        int q, k;
        if (BANDED) {
            // band-major (every pair's k-th band, then k + 1): under a band a
            // pair has few bands ready at a time; band k - 1 of a pair is always
            // earlier in the list.  Every pair has the same bands (one prototype).
            q = item % p.P;
            k = item / p.P;
        } else if (p.band_cnt > 0) {          // a band range of every pair
            q = item / p.band_cnt;
            k = item % p.band_cnt;
        } else {
            q = find_slot(p.prefix, p.P, item);
            k = item - p.prefix[q];
        }
        const PairDesc pd = p.pairs[p.order[q]];
        if (BWD) {
            // bands bottom-up: the whole pair, or the range's last band first
            const int band = p.band_cnt > 0 ? p.band_lo + p.band_cnt - 1 - k : pd.nbands - 1 - k;
            float4* wring = rring_all + (threadIdx.x >> 5) * soft_warp_f4<D, R>(FUSED, BANDED);
            if constexpr (FUSED && !BANDED) {
                static_assert(soft_warp_f4<D, R>(true, false) >= soft_warp_f4<D, R>(false, false),
                              "the fused warp's shared memory holds the R ring");
                // a pair that kept R (store_pairs) beside checkpointed ones: the
                // backward that reads R, in this warp's part of shared memory
                // (the fused layout is the larger)
                if (pd.keep_r) {
                    bwd_band<D, R, BANDED, COST, false>(p, pd, band, lane, wring, band - p.band_lo + p.rbuf_band0);
                    continue;
                }
            }
            bwd_band<D, R, BANDED, COST, FUSED, ALIGNED>(p, pd, band, lane, wring, band - p.band_lo + p.rbuf_band0);
        } else {
            const int band = p.band_cnt > 0 ? p.band_lo + k : k;
            fwd_band<D, R, BANDED, COST>(p, pd, band, lane, band - p.band_lo + p.rbuf_band0, p.recompute != 0,
                                         p.store_r != 0 || pd.keep_r != 0);
        }
    }
}

// g == null: Eq. 7's weights lambda_k / m_k with lambda_k = 1, i.e. 1 / N_k
// (N_k from the offsets), rounded to FP32 as a caller's FP32 weights would be.
// Blocks of at most 4 warps.
template <int D, int R, bool BWD, bool BANDED, int COST, bool FUSED>
__global__ void __launch_bounds__(256) softdtw_kernel(SoftParams p)
{
    soft_items<D, R, BWD, BANDED, COST, FUSED>(p);
}

// The backward for one channel without a band, its step loop unrolled by two,
// held to 128 registers: four blocks of 4 warps per SM (2,432 warps on the
// GPU; the 2,560 (pair, band) items of 64 pairs of 10k then almost all run at
// once).  Held to 96 registers (five blocks, every item at once) it ran 1.5 %
// slower on that workload, the unrolled loop at the edge of its registers.
// ALIGNED (M a multiple of R) needs no checked columns.
template <int D, int R, bool BANDED, int COST, bool FUSED, bool ALIGNED = false>
__global__ void __launch_bounds__(128, 4) softdtw_bwd_narrow_kernel(SoftParams p)
{
    soft_items<D, R, true, BANDED, COST, FUSED, ALIGNED>(p);
}

// the kernel that runs (D, BWD, FUSED)
template <int D, int R, bool BWD, bool BANDED, int COST, bool FUSED>
constexpr auto soft_kernel()
{
    if constexpr (BWD && D == 1 && !BANDED)
        return softdtw_bwd_narrow_kernel<D, R, BANDED, COST, FUSED>;
    else
        return softdtw_kernel<D, R, BWD, BANDED, COST, FUSED>;
}

// dynamic shared memory per block: the backward's R ring (or, FUSED, its
// kCk-step buffer of recomputed R and the staged inputs of the next chunk)
template <int D, int R>
constexpr size_t soft_smem(bool bwd, bool fused, bool banded, int block)
{
    return bwd ? (size_t)(block / 32) * soft_warp_f4<D, R>(fused, banded) * sizeof(float4) : 0;
}

__global__ void grad_reduce_kernel(const float* __restrict__ gpart, const float* __restrict__ g,
                                   const int64_t* __restrict__ offsets, int T, int64_t M, int d,
                                   float* __restrict__ out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = M * d;
    if (q >= n) return;
    double acc = 0.0;
    for (int k = 0; k < T; ++k) {
        const float gk = g ? __ldg(g + k)
                           : __double2float_rn(__ddiv_rn(1.0, (double)(__ldg(offsets + k + 1) - __ldg(offsets + k))));
        acc = __fma_rn((double)gk, (double)__ldg(gpart + (int64_t)k * n + q), acc);
    }
    out[q] = __double2float_rn(acc);
}

__global__ void adam_kernel(float* x, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                            float beta2, float eps, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = grad[i];
    const float mi = __fmaf_rn(beta1, m[i], __fmul_rn(1.f - beta1, gi));
    const float vi = __fmaf_rn(beta2, v[i], __fmul_rn(1.f - beta2, __fmul_rn(gi, gi)));
    m[i] = mi;
    v[i] = vi;
    const float mh = __fdiv_rn(mi, bc1);
    const float vh = __fdiv_rn(vi, bc2);
    x[i] = __fsub_rn(x[i], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(sqrtf(vh), eps)));
}

template <int D, int R, bool BWD, bool BANDED, int COST, bool FUSED = false>
cudaError_t launch_dbr(const SoftParams& p, int grid, int block, cudaStream_t st)
{
    const size_t smem = soft_smem<D, R>(BWD, FUSED, BANDED, block);
    auto run = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, block, smem, st>>>(p);
        return cudaGetLastError();
    };
    if constexpr (BWD && D == 1 && !BANDED) {
        if (p.m_aligned) return run(softdtw_bwd_narrow_kernel<D, R, BANDED, COST, FUSED, true>);
    }
    return run(soft_kernel<D, R, BWD, BANDED, COST, FUSED>());
}

// 8 rows per lane, or 4 under a narrow band (kSoftNarrowBand)
template <int D, bool BWD, bool BANDED, int COST, bool FUSED = false>
cudaError_t launch_db(const SoftParams& p, int grid, int block, cudaStream_t st)
{
    if constexpr (BANDED) {
        if (p.rows == 4) return launch_dbr<D, 4, BWD, BANDED, COST, FUSED>(p, grid, block, st);
    }
    return launch_dbr<D, 8, BWD, BANDED, COST, FUSED>(p, grid, block, st);
}

template <int D, bool BWD>
cudaError_t launch_d(const SoftParams& p, int grid, int block, cudaStream_t st)
{
    if (BWD && p.fused && !p.banded)
        return p.cost_kind == kCostL2 ? launch_db<D, BWD, false, kCostL2, BWD>(p, grid, block, st)
                                      : launch_db<D, BWD, false, kCostSqEuclid, BWD>(p, grid, block, st);
    if (p.cost_kind == kCostL2)
        return p.banded ? launch_db<D, BWD, true, kCostL2>(p, grid, block, st)
                        : launch_db<D, BWD, false, kCostL2>(p, grid, block, st);
    return p.banded ? launch_db<D, BWD, true, kCostSqEuclid>(p, grid, block, st)
                    : launch_db<D, BWD, false, kCostSqEuclid>(p, grid, block, st);
}

template <int D, int R, bool BWD, bool BANDED, int COST, bool FUSED = false>
int occ_dbr(int block)
{
    const size_t smem = soft_smem<D, R>(BWD, FUSED, BANDED, block);
    int n = 0;
    auto kern = soft_kernel<D, R, BWD, BANDED, COST, FUSED>();
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, block, smem);
    return n;
}

template <int D, bool BWD, bool BANDED, int COST, bool FUSED = false>
int occ_db(int block, int rows)
{
    if constexpr (BANDED) {
        if (rows == 4) return occ_dbr<D, 4, BWD, BANDED, COST, FUSED>(block);
    }
    return occ_dbr<D, 8, BWD, BANDED, COST, FUSED>(block);
}

template <int D, bool BWD>
int occ_d(int block, int banded, int cost_kind, int fused, int rows)
{
    if (BWD && fused && !banded)
        return cost_kind == kCostL2 ? occ_db<D, BWD, false, kCostL2, BWD>(block, rows)
                                    : occ_db<D, BWD, false, kCostSqEuclid, BWD>(block, rows);
    if (cost_kind == kCostL2)
        return banded ? occ_db<D, BWD, true, kCostL2>(block, rows) : occ_db<D, BWD, false, kCostL2>(block, rows);
    return banded ? occ_db<D, BWD, true, kCostSqEuclid>(block, rows)
                  : occ_db<D, BWD, false, kCostSqEuclid>(block, rows);
}

}  // namespace

#define WTS_SOFT_DISPATCH(FN, BWD, ...)          \
    switch (D) {                                 \
        case 1: return FN<1, BWD>(__VA_ARGS__);  \
        case 2: return FN<2, BWD>(__VA_ARGS__);  \
        case 3: return FN<3, BWD>(__VA_ARGS__);  \
        case 4: return FN<4, BWD>(__VA_ARGS__);  \
        case 6: return FN<6, BWD>(__VA_ARGS__);  \
        case 8: return FN<8, BWD>(__VA_ARGS__);  \
        default: break;                          \
    }

cudaError_t launch_softdtw_fwd(int D, const SoftParams& p, int grid, int block, cudaStream_t st)
{
    WTS_SOFT_DISPATCH(launch_d, false, p, grid, block, st)
    return cudaErrorInvalidValue;
}

cudaError_t launch_softdtw_bwd(int D, const SoftParams& p, int grid, int block, cudaStream_t st)
{
    WTS_SOFT_DISPATCH(launch_d, true, p, grid, block, st)
    return cudaErrorInvalidValue;
}

int softdtw_max_blocks_per_sm(int D, int backward, int block, int banded, int cost_kind, int fused, int rows)
{
    if (backward) {
        WTS_SOFT_DISPATCH(occ_d, true, block, banded, cost_kind, fused, rows)
    } else {
        WTS_SOFT_DISPATCH(occ_d, false, block, banded, cost_kind, fused, rows)
    }
    return 0;
}

cudaError_t launch_softdtw_grad_reduce(const float* gpart, const float* g, const int64_t* offsets, int T, int64_t M,
                                       int d, float* grad_B, cudaStream_t st)
{
    const int64_t n = M * d;
    grad_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gpart, g, offsets, T, M, d, grad_B);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* x, const float* grad, float* m, float* v, int64_t n, float lr, float beta1,
                        float beta2, float eps, int t, cudaStream_t st)
{
    double b1t = 1.0, b2t = 1.0;
    for (int i = 0; i < t; ++i) { b1t *= beta1; b2t *= beta2; }
    adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, grad, m, v, n, lr, beta1, beta2, eps,
                                                              (float)(1.0 - b1t), (float)(1.0 - b2t));
    return cudaGetLastError();
}

}  // namespace wts
