// Kernel templates of the hard-min band wavefront for DTW (Eq. 1, computed by
// the recursion Eq. 5 with gamma = 0; the alignment path of Definition
// "Alignment path").  Each dtw_wavefront_*.cu file instantiates one set of
// them (rows per lane R, local cost, with or without a band), so that the
// sets compile in parallel; dtw_wavefront.cu dispatches between the sets.
//
//   r(0,0) = 0, r(i,0) = r(0,j) = +inf,
//   r(i,j) = delta(i,j) + min(r(i-1,j-1), r(i-1,j), r(i,j-1)),
//   delta(i,j) = sum_c (b_ic - y_jc)^2   (squared Euclidean local cost), or
//   its square root (COST = kCostL2: the l2 norm, Sec. 3.2's wording).
//
// Ties between predecessors resolve diag first, then up (i-1,j), then left
// (i,j-1).  With m = min(dg, up, lf): the predecessor is diag iff dg == m,
// else up iff up == m, else left.  The CPU oracle takes the same decision in
// the same float arithmetic (subtract, then one fused multiply-add per channel
// from 0, the IEEE square root for the l2 norm, then one add), so paths match
// bit for bit.
//
// One warp owns a band of 32*R rows of one pair; lane t holds R rows, their
// prototype samples (as row pairs, for the packed f32x2 arithmetic) and their
// last column of r in registers.  Lanes are skewed by one column (lane t is at
// column s - t in step s), so the value above a lane's first row comes from
// lane t-1 by __shfl_up_sync.  Cycle samples are staged per warp in a
// 128-column shared-memory ring as duplicated pairs {y, y}, refilled every 32
// steps from registers loaded ahead.  Lane 0 of band b > 0 reads the bottom row
// of band b-1 from a hand-off row in global memory (L2), 32 columns at a time,
// also one chunk ahead; each slot is NaN until its producer has written it
// (the row is pre-filled before the launch), so the consumer re-reads only the
// slots that are not there yet.
// Each warp takes (pair, band) items in order from a global cursor, so the
// producer of any item it waits for was started earlier: no deadlock, with or
// without co-residency.  Every wait is bounded (wait_progress).
//
// Predecessor codes (kModeDirs) are two bit-planes per lane and step: bit
// p*R + k of the lane's W = R/16 words is plane p of row k, plane 0 = "not
// diag", plane 1 = "not up" (meaningful only when plane 0 is set).  With R = 8
// (R = 4) a step has 16 (8) bits and two (four) consecutive steps share one
// word, the earliest step in the lowest bits.
#pragma once

#include "dtw_wavefront.cuh"

namespace wts {

namespace {

typedef unsigned long long u64;

__device__ __forceinline__ u64 pack2(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ u64 fsub2(u64 a, u64 b)
{
    u64 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 fmul2(u64 a, u64 b)
{
    u64 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ u64 ffma2(u64 a, u64 b, u64 c)
{
    u64 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ float min3f(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// all ones if a != b, else 0
__device__ __forceinline__ uint32_t ne_mask(float a, float b)
{
    uint32_t r;
    asm("set.ne.u32.f32 %0, %1, %2;" : "=r"(r) : "f"(a), "f"(b));
    return r;
}

constexpr int kRing = 128;   // columns of cycle samples staged per warp
constexpr int kSlot = 4;     // u64 words after a warp's ring: its band's columns and the band



// c[k] for a k known only at run time, by a binary tree of selects on the bits
// of k (R - 1 selects, no local memory)
template <int R>
__device__ __forceinline__ float pick_row(const float (&c)[R], int k)
{
    float v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = c[q];
#pragma unroll
    for (int w = R / 2; w >= 1; w /= 2) {
        const bool hi = (k & w) != 0;
#pragma unroll
        for (int q = 0; q < w; ++q) v[q] = hi ? v[q + w] : v[q];
    }
    return v[0];
}

template <int D, int R, int MODE, bool BANDED, int COST>
struct Band {
    static constexpr int BR = 32 * R;
    static constexpr int W = R / 16;        // code words per lane per step (0: part of a word)
    static constexpr int SPW = R >= 16 ? 1 : 32 / (2 * R);     // steps per code word
    static constexpr int Q = R / 2;         // row pairs

    u64 bp[Q][D];                           // prototype rows as pairs
    float col[R];                           // r at the lane's last column
    float dl[R];                            // local costs of the lane's next column
    int cnt[R];                             // path cells (kModePlen)
    float prev_up;                          // r(i0-1, j-1) for the first row
    int prev_upc;
    float topv;                             // lane l: r(band top - 1, s0 + l)
    int topc;
    uint32_t half;                          // R < 16: codes of the word's earlier steps
    // kModeSubDirs, matrix's last band: running minimum of r(M-1, j) over the
    // lane's columns (row kk of the lane), and its first column
    bool track;
    int kk;
    float best;
    int bestj;
    static constexpr bool CODES = MODE == kModeDirs || MODE == kModeSubDirs;

    // Local costs of column jc for the lane's rows, pair q (two rows at once).
    __device__ __forceinline__ void cost_pair(const u64* yy, int q)
    {
        u64 t = fsub2(bp[q][0], yy[0]);
        u64 acc = fmul2(t, t);
#pragma unroll
        for (int c = 1; c < D; ++c) {
            t = fsub2(bp[q][c], yy[c]);
            acc = ffma2(t, t, acc);
        }
        unpack2(acc, dl[2 * q], dl[2 * q + 1]);
        if (COST == kCostL2) {                   // the norm itself: IEEE square root
            dl[2 * q] = __fsqrt_rn(dl[2 * q]);
            dl[2 * q + 1] = __fsqrt_rn(dl[2 * q + 1]);
        }
    }

    __device__ __forceinline__ void load_samples(const u64* ring, int jc, u64* yy)
    {
        const u64* yr = ring + (jc & (kRing - 1));
#pragma unroll
        for (int c = 0; c < D; ++c) yy[c] = yr[c * kRing];
    }

    // One step: the lane's column j = s - lane (in range when FULLCHUNK).
    // dl holds the local costs of column j on entry and those of column j+1 on
    // exit: the next column's costs are computed between the links of this
    // column's min-plus chain, which is serial down the rows.
    template <bool FULLCHUNK, bool MASK = false>
    __device__ __forceinline__ void step(const u64* ring, int s, int src, int lane, int N, bool top,
                                         void* hcur, uint32_t* dout)
    {
        const float INF = inf_f();
        const float above = __shfl_up_sync(FULL, col[R - 1], 1);
        const float tv = __shfl_sync(FULL, topv, src);
        // above the matrix: +inf (DTW), 0 for Sub-DTW (a path may start in any column)
        const float top_in = MODE == kModeSubDirs ? 0.f : INF;
        const float up_in = lane == 0 ? (top ? top_in : tv) : above;
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
        u64 yy[D];
        load_samples(ring, j + 1, yy);
        uint32_t word[W > 0 ? W : 1];
#pragma unroll
        for (int w = 0; w < (W > 0 ? W : 1); ++w) word[w] = 0u;
        // partial chunks with a band read the band's columns (and the band)
        // from the warp's slot after the sample ring:
        // [jlo | jhi << 32, row0 | M << 32, bnd]
        const u64* slot = ring + D * kRing;
        bool valid = true;
        int klo = 0, khi = R - 1;
        if (!FULLCHUNK && !BANDED) valid = j >= 0 && j < N;
        if (!FULLCHUNK && BANDED) {
            const u64 cols = slot[0];
            valid = j >= (int)(uint32_t)cols && j <= (int)(cols >> 32);
            if (MASK) {
                // rows k in [klo, khi] lie in the band at column j
                const u64 im = slot[1];
                const int64_t bnd = (int64_t)slot[2];
                const int i0 = (int)(uint32_t)im + lane * R;
                const int64_t jm = (int64_t)j * (int64_t)(im >> 32);
                klo = (int)max((int64_t)-1, ceil_div64(jm - bnd, N) - i0);
                khi = (int)min((int64_t)R, floor_div64(jm + bnd, N) - i0);
            }
        }
        if (FULLCHUNK || valid) {
            float dg = dg_in, up = up_in;
            int cdg = dgc_in, cup = upc_in;
#pragma unroll
            for (int k = 0; k < R; ++k) {
                const float lf = col[k];
                const float m = min3f(dg, up, lf);
                float r = __fadd_rn(dl[k], m);
                if (MASK && (k < klo || k > khi)) r = INF;     // outside the band
                if (CODES) {
                    word[k >> 5] |= ne_mask(dg, m) & (1u << (k & 31));
                    word[(R + k) >> 5] |= ne_mask(up, m) & (1u << ((R + k) & 31));
                } else if (MODE == kModePlen) {
                    const int cl = cnt[k];
                    const int cn = 1 + (dg == m ? cdg : (up == m ? cup : cl));
                    cdg = cl;
                    cup = cn;
                    cnt[k] = cn;
                }
                dg = lf;
                up = r;
                col[k] = r;
                if (k & 1) cost_pair(yy, k >> 1);      // rows k-1, k of column j+1
            }
            if (MODE == kModeSubDirs && track) {
                const float v = pick_row<R>(col, kk);
                if (v < best) { best = v; bestj = j; }
            }
            if (lane == 31 && hcur != nullptr) {
                if (MODE == kModePlen)
                    __stcg(reinterpret_cast<u64*>(hcur) + j, pack2(col[R - 1], __int_as_float(cnt[R - 1])));
                else
                    __stcg(reinterpret_cast<float*>(hcur) + j, col[R - 1]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < Q; ++q) cost_pair(yy, q);
        }
        if (CODES) {
            if (W == 0 && SPW == 2) {
                if ((s & 1) == 0)
                    half = word[0];
                else
                    __stcs(dout + (int64_t)(s >> 1) * 32 + lane, __byte_perm(half, word[0], 0x5410));
            } else if (W == 0) {
                const int sl = s & (SPW - 1);
                half = sl == 0 ? word[0] : (half | (word[0] << (sl * 2 * R)));
                if (sl == SPW - 1) __stcs(dout + (int64_t)(s / SPW) * 32 + lane, half);
            } else if (W == 1) {
                __stcs(dout + (int64_t)s * 32 + lane, word[0]);
            } else {
                __stcs(reinterpret_cast<uint2*>(dout) + (int64_t)s * 32 + lane,
                       make_uint2(word[0], word[W > 1 ? 1 : 0]));
            }
        }
    }
};

template <int D, int R, int MODE, bool BANDED, int COST>
__device__ __forceinline__ void run_band(const DPParams& p, const PairDesc& pd, int band, int lane, u64* ring)
{
    using BandT = Band<D, R, MODE, BANDED, COST>;
    constexpr int BR = BandT::BR;
    constexpr int W = BandT::W;
    const int M = pd.M, N = pd.N, d = p.d;
    const int i0 = band * BR + lane * R;
    const bool top = band == 0;
    const bool last = band == pd.nbands - 1;
    const float INF = inf_f();

    BandT st;
#pragma unroll
    for (int q = 0; q < BandT::Q; ++q)
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int ia = i0 + 2 * q, ib = ia + 1;
            const float va = (ia < M && c < d) ? __ldg(pd.X + (int64_t)ia * d + c) : 0.f;
            const float vb = (ib < M && c < d) ? __ldg(pd.X + (int64_t)ib * d + c) : 0.f;
            st.bp[q][c] = pack2(va, vb);
        }
#pragma unroll
    for (int k = 0; k < R; ++k) { st.col[k] = INF; st.cnt[k] = 0; }
    // r(i0-1, j-1) at j = 0: r(0,0) = 0 (0 cells) for the matrix's first row, +inf otherwise
    st.prev_up = (top && lane == 0) ? 0.f : INF;
    st.prev_upc = 0;
    st.topv = INF;
    st.topc = 0;
    st.half = 0u;
    st.track = MODE == kModeSubDirs && last;
    st.kk = M - 1 - i0;
    st.best = INF;
    st.bestj = 0;

    // Sakoe-Chiba band: row i keeps columns [lo(i), hi(i)] with
    // lo(i) = ceil((i N - bnd) / M), hi(i) = floor((i N + bnd) / M), both
    // nondecreasing in i.  The band's columns run from lo(first row) to
    // hi(last row); the row above is +inf outside [lo, hi] of that row; a lane
    // needs no masking where all its rows are in: [lo(last row), hi(first row)].
    const int64_t bnd = BANDED ? pd.band_bound : -1;
    int jlo_b = 0, jhi_b = N - 1, jtop_lo = 0, jtop_hi = N - 1, full_lo = 0, full_hi = N - 1;
    if (BANDED) {
        auto lo_of = [&](int64_t i) { return (int)max((int64_t)0, ceil_div64(i * N - bnd, M)); };
        auto hi_of = [&](int64_t i) { return (int)min((int64_t)N - 1, floor_div64(i * N + bnd, M)); };
        const int64_t r0 = (int64_t)band * BR, r1 = min(r0 + BR, (int64_t)M) - 1;
        jlo_b = lo_of(r0);
        jhi_b = hi_of(r1);
        if (!top) { jtop_lo = lo_of(r0 - 1); jtop_hi = hi_of(r0 - 1); }
        if (i0 < M) { full_lo = lo_of(min(i0 + R - 1, M - 1)); full_hi = hi_of(i0); }
    }
    if (BANDED) {
        u64* slot = ring + D * kRing;
        __syncwarp();
        if (lane == 0) {
            slot[0] = (u64)(uint32_t)jlo_b | ((u64)(uint32_t)jhi_b << 32);
            slot[1] = (u64)(uint32_t)(band * BR) | ((u64)(uint32_t)M << 32);
            slot[2] = (u64)bnd;
        }
        __syncwarp();
    }
    // chunks of 32 steps from a multiple of 32, starting at or before column
    // jlo_b - 1: lane 0 takes its first diagonal, r(r0 - 1, jlo_b - 1), from
    // the row above at the step before its first column (that cell may be
    // inside the band)
    const int s_begin = max(0, (jlo_b - 1) & ~31);
    const int s_end = jhi_b + 32;           // one past the last step (column jhi_b in lane 31)

    // hand-off rows: slot size 4 bytes (r), or 8 bytes ({r, cells}) with |pi|
    constexpr int SLOT = MODE == kModePlen ? 8 : 4;
    char* hb = static_cast<char*>(p.hbuf);
    const char* hprev = top ? nullptr : hb + (pd.hbuf_off + (int64_t)(band - 1) * N) * SLOT;
    // a recomputed band reads its stored top row and produces no hand-off row
    void* hcur = (last || p.recompute || p.skip_handoff) ? nullptr : hb + (pd.hbuf_off + (int64_t)band * N) * SLOT;
    uint32_t* dout = BandT::CODES ? p.dirs + pd.dir_off + (int64_t)(band - p.band_lo) * band_dir_words(N, R)
                                         : nullptr;

    // Cycle samples go through the ring two chunks of 32 columns ahead of the
    // step that first reads them (a step also reads the next column), loaded
    // into registers one chunk before that; the bottom row of the band above
    // (NaN until its producer has written it) is read one chunk ahead.
    float ynext[D];
    u64 tnext = 0;
    auto load_y = [&](int jj) {
#pragma unroll
        for (int c = 0; c < D; ++c) ynext[c] = (jj < N && c < d) ? __ldg(pd.Y + (int64_t)jj * d + c) : 0.f;
    };
    auto put_y = [&](int jj) {
#pragma unroll
        for (int c = 0; c < D; ++c) ring[c * kRing + (jj & (kRing - 1))] = pack2(ynext[c], ynext[c]);
    };
    auto load_t = [&](int jj) -> u64 {
        if (jj >= N) return 0;
        if (SLOT == 8) return __ldcv(reinterpret_cast<const u64*>(hprev) + jj);
        return (u64)__float_as_uint(__ldcv(reinterpret_cast<const float*>(hprev) + jj));
    };
    __syncwarp();
    load_y(s_begin + lane);
    put_y(s_begin + lane);
    load_y(s_begin + lane + 32);
    put_y(s_begin + lane + 32);
    load_y(s_begin + lane + 64);
    if (!top) tnext = load_t(s_begin + lane);
    __syncwarp();
    {
        // local costs of the lane's first column (j = s_begin - lane)
        u64 yy[D];
        st.load_samples(ring, s_begin - lane, yy);
#pragma unroll
        for (int q = 0; q < BandT::Q; ++q) st.cost_pair(yy, q);
    }

    for (int s0 = s_begin; s0 < s_end; s0 += 32) {
        if (s0 <= jhi_b) {
            const int jj = s0 + lane;
            if (s0 > s_begin) {
                __syncwarp();
                put_y(jj + 32);
                load_y(jj + 64);
                __syncwarp();
            }
            if (!top) {
                // only the row above's columns inside the band are written (and waited for)
                const bool need = jj >= jtop_lo && jj <= jtop_hi;
                u64 t = tnext;
                const bool ok = wait_filled(need && is_nan_bits((uint32_t)t),
                                            [&]() { t = load_t(jj); return is_nan_bits((uint32_t)t); }, p.hdr, 1,
                                            p.spin_limit);
                if (!ok) return;
                st.topv = need ? __uint_as_float((uint32_t)t) : INF;
                if (MODE == kModePlen) st.topc = (int)(t >> 32);
                tnext = load_t(jj + 32);
            }
        }
        // every lane in the band's columns and inside the band all chunk long
        const bool full = BANDED ? (s0 - 31 >= jlo_b && s0 + 31 <= jhi_b &&
                                    __all_sync(FULL, s0 - lane >= full_lo && s0 + 31 - lane <= full_hi))
                                 : (s0 >= 31 && s0 + 32 <= N);
        if (full) {
#pragma unroll 2
            for (int u = 0; u < 32; ++u) st.template step<true>(ring, s0 + u, u, lane, N, top, hcur, dout);
        } else {
            const int n = min(32, s_end - s0);
            if (BANDED) {
                for (int u = 0; u < n; ++u) st.template step<false, true>(ring, s0 + u, u, lane, N, top, hcur, dout);
            } else {
                for (int u = 0; u < n; ++u) st.template step<false>(ring, s0 + u, u, lane, N, top, hcur, dout);
            }
        }
    }

    constexpr int SPW = BandT::SPW;
    if (BandT::CODES && W == 0 && (s_end % SPW) != 0)
        __stcs(dout + (int64_t)((s_end - 1) / SPW) * 32 + lane, st.half);

    if (MODE == kModeSubDirs) {
        if (last && lane == (M - 1 - band * BR) / R) {
            if (p.cost_out) p.cost_out[pd.out] = st.best;
            p.bstar_out[pd.out] = st.bestj;
        }
    } else if (last && !p.recompute) {
        const int ilast = M - 1 - band * BR;
        if (lane == ilast / R) {
            const int kk = ilast % R;
            float v = st.col[0];
            int c = st.cnt[0];
#pragma unroll
            for (int k = 1; k < R; ++k)
                if (k == kk) { v = st.col[k]; c = st.cnt[k]; }
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

// Blocks of at most 4 warps.  R = 16: three resident blocks (12 warps, <= 170
// registers) where the prototype rows fit easily, two otherwise (the
// software-pipelined step keeps enough independent work per warp).  R = 8
// halves the prototype registers: four blocks (16 warps, <= 128 registers) up
// to 6 channels.
template <int D, int R>
constexpr int min_blocks()
{
    return R == 4 ? (D <= 8 ? 4 : 3) : R == 8 ? (D <= 6 ? 4 : (D <= 8 ? 3 : 2)) : ((R == 16 && D <= 4) ? 3 : 2);
}

template <int D, int R, int MODE, bool BANDED, int COST>
__global__ void __launch_bounds__(128, min_blocks<D, R>()) dtw_wavefront_kernel(DPParams p)
{
    extern __shared__ u64 ring_all[];
    const int lane = threadIdx.x & 31;
    u64* ring = ring_all + (threadIdx.x >> 5) * (D * kRing + kSlot);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&p.hdr->item_counter, 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= p.n_items) break;
        if (ld_volatile(&p.hdr->abort)) break;
        int q, band;
        if (p.group_pairs > 0) {
            // groups of G pairs (in the work list's order), band-major within
            // a group: a group's bands start in the order their producers
            // do, and its items about fill the resident warps once (G = P:
            // every pair's band b before any band b + 1, as under a band,
            // where a pair has few bands ready at a time).  Every pair has the
            // same bands here (one prototype); recompute runs the range
            // [band_lo, band_lo + band_cnt) of each.  Band b - 1 of a pair is
            // earlier in the list (no deadlock).
            const int nb = p.recompute ? p.band_cnt : p.prefix[1] - p.prefix[0];
            const int G = p.group_pairs;
            const int g = item / (G * nb), q0 = g * G;
            const int Gg = min(G, p.P - q0);
            const int r = item - q0 * nb;
            q = q0 + r % Gg;
            band = (p.recompute ? p.band_lo : 0) + r / Gg;
        } else if (p.recompute) {
            q = item / p.band_cnt;
            band = p.band_lo + item % p.band_cnt;
        } else {
            q = find_slot(p.prefix, p.P, item);
            band = item - p.prefix[q];
        }
        const PairDesc pd = p.pairs[p.order[q]];
        run_band<D, R, MODE, BANDED, COST>(p, pd, band, lane, ring);
    }
}

template <int D>
constexpr size_t ring_bytes(int block) { return (size_t)(block / 32) * (D * kRing + kSlot) * sizeof(u64); }

template <int D, int R, int MODE, bool BANDED, int COST>
cudaError_t launch_one(const DPParams& p, int grid, int block, cudaStream_t st)
{
    const size_t smem = ring_bytes<D>(block);
    cudaFuncSetAttribute(dtw_wavefront_kernel<D, R, MODE, BANDED, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    dtw_wavefront_kernel<D, R, MODE, BANDED, COST><<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

template <int D, int R, int MODE, bool BANDED, int COST>
int occ_one(int block)
{
    int n = 0;
    const size_t smem = ring_bytes<D>(block);
    cudaFuncSetAttribute(dtw_wavefront_kernel<D, R, MODE, BANDED, COST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dtw_wavefront_kernel<D, R, MODE, BANDED, COST>, block, smem);
    return n;
}

// The three DTW modes for every instance; Sub-DTW (never banded) for R = 8 and 16.
template <int D, int R, bool BANDED, int COST>
cudaError_t launch_mode(int mode, const DPParams& p, int grid, int block, cudaStream_t st)
{
    if constexpr (R == 4) {                  // Sub-DTW windows only (one pair: more, shorter bands)
        if (mode == kModeSubDirs && !BANDED) return launch_one<D, 4, kModeSubDirs, false, COST>(p, grid, block, st);
        return cudaErrorInvalidValue;
    } else {
        switch (mode) {
            case kModeCost: return launch_one<D, R, kModeCost, BANDED, COST>(p, grid, block, st);
            case kModePlen: return launch_one<D, R, kModePlen, BANDED, COST>(p, grid, block, st);
            case kModeDirs: return launch_one<D, R, kModeDirs, BANDED, COST>(p, grid, block, st);
            case kModeSubDirs:
                if constexpr (!BANDED && (R == 16 || R == 8))
                    return launch_one<D, R, kModeSubDirs, false, COST>(p, grid, block, st);
                break;
            default: break;
        }
        return cudaErrorInvalidValue;
    }
}

template <int D, int R, bool BANDED, int COST>
int occ_mode(int mode, int block)
{
    if constexpr (R == 4) {
        if (mode == kModeSubDirs && !BANDED) return occ_one<D, 4, kModeSubDirs, false, COST>(block);
        return 0;
    } else {
        switch (mode) {
            case kModeCost: return occ_one<D, R, kModeCost, BANDED, COST>(block);
            case kModePlen: return occ_one<D, R, kModePlen, BANDED, COST>(block);
            case kModeDirs: return occ_one<D, R, kModeDirs, BANDED, COST>(block);
            case kModeSubDirs:
                if constexpr (!BANDED && (R == 16 || R == 8)) return occ_one<D, R, kModeSubDirs, false, COST>(block);
                break;
            default: break;
        }
        return 0;
    }
}

// One set of instances: every padded channel count D (1, 2, 3 only for R = 32).
#define WTS_WF_SWITCH_D(FN, ...)                                              \
    switch (D) {                                                             \
        case 1: return FN<1, R, BANDED, COST>(__VA_ARGS__);                   \
        case 2: return FN<2, R, BANDED, COST>(__VA_ARGS__);                   \
        case 3: return FN<3, R, BANDED, COST>(__VA_ARGS__);                   \
        default: break;                                                      \
    }                                                                        \
    if constexpr (R < 32) {                                                  \
        switch (D) {                                                         \
            case 4: return FN<4, R, BANDED, COST>(__VA_ARGS__);               \
            case 6: return FN<6, R, BANDED, COST>(__VA_ARGS__);               \
            case 8: return FN<8, R, BANDED, COST>(__VA_ARGS__);               \
            case 12: return FN<12, R, BANDED, COST>(__VA_ARGS__);             \
            case 16: return FN<16, R, BANDED, COST>(__VA_ARGS__);             \
            default: break;                                                  \
        }                                                                    \
    }

template <int R, bool BANDED, int COST>
cudaError_t launch_set(int mode, int D, const DPParams& p, int grid, int block, cudaStream_t st)
{
    WTS_WF_SWITCH_D(launch_mode, mode, p, grid, block, st)
    return cudaErrorInvalidValue;
}

template <int R, bool BANDED, int COST>
int occ_set(int mode, int D, int block)
{
    WTS_WF_SWITCH_D(occ_mode, mode, block)
    return 0;
}

#undef WTS_WF_SWITCH_D

}  // namespace

}  // namespace wts

// Defines the entry points wf_launch_TAG / wf_occ_TAG of one instance set.
#define WTS_WF_ENTRY(TAG, R, BANDED, COST)                                                        \
    namespace wts {                                                                               \
    cudaError_t wf_launch_##TAG(int mode, int D, const DPParams& p, int grid, int block, cudaStream_t st) \
    {                                                                                             \
        return launch_set<R, BANDED, COST>(mode, D, p, grid, block, st);                          \
    }                                                                                             \
    int wf_occ_##TAG(int mode, int D, int block) { return occ_set<R, BANDED, COST>(mode, D, block); } \
    }
