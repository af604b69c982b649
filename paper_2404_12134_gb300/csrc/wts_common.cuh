// Shared device-side definitions of the WETSAND alignment kernels (sm_103a).
//
// Geometry used by every wavefront kernel.  A pair (X, Y) has X on the rows
// (length M: the prototype / barycenter B, Eq. 8 and Eq. 7 put B first) and Y
// on the columns (length N: a cycle).  The M rows are cut into bands of
// BR = 32 * R rows; one warp owns one band, lane t owns rows
// [band*BR + t*R, band*BR + t*R + R).  Lanes are skewed by one column: at step
// s lane t works on column j = s - t, so the row above a lane's first row was
// finished by lane t-1 one step earlier and arrives by a register shuffle.
// Bands of the same pair are chained through a full-row hand-off buffer in
// global memory (the bottom row of band b is the top boundary of band b+1),
// each slot filled once and polled by the consumer (see wait_filled).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wts {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kMaxD = 16;              // channels handled (zero-padded up to the template D)
constexpr long long kSpinLimit = 1ll << 27;   // polls before a wait gives up (~tens of seconds)

// Device status word values (first word of every workspace): a wait gave up,
// or a sample of the inputs is not finite (found before any DP work).
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1, kDevBadInput = 2 };
// local cost delta(b_i, y_j) (Sec. 3.2): the squared l2 norm, or the norm itself
enum LocalCost : int { kCostSqEuclid = 0, kCostL2 = 1 };

// One alignment problem of a batch.
struct PairDesc {
    const float* X;      // rows, [M][d]
    const float* Y;      // columns, [N][d]
    int32_t M, N;
    int32_t nbands;      // ceil(M / BR)
    int32_t out;         // output slot (cycle index, or pair index for pairwise)
    int64_t dir_off;     // first direction word of this pair
    int64_t hbuf_off;    // first slot of this pair's hand-off rows ((nbands-1) * N slots)
    int64_t aux_off;     // first element of per-pair auxiliary storage (R store)
    int64_t band_bound;  // Sakoe-Chiba band: cell (i, j) kept when |i N - j M| <= band_bound; -1 = no band
    int32_t keep_r;      // soft-DTW checkpoint mode: this pair's R is stored (not column checkpoints)
    int32_t spare;
};

// Header at the start of every workspace.
struct WsHeader {
    int status;          // DevStatus; sticky until the next call resets it
    int item_counter;    // work-list cursor of the persistent kernels
    int abort;           // set with status so that waiting warps leave at once
    int timeout_where;   // which wait gave up (diagnostics)
    int pad[60];
};

__device__ __forceinline__ float inf_f() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ int ld_volatile(const int* p)
{
    int v;
    asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Hand-off rows between bands are pre-filled with 0xFF bytes (a NaN pattern)
// before every launch; a producer writes each slot once with a plain store and
// a consumer polls the slot until it is no longer NaN.  Each slot is one
// single-copy-atomic word (4 or 8 bytes), so no flag and no fence is needed.
// Hard-min costs are never NaN for finite inputs (a non-finite sample is
// rejected before the wavefront runs); the soft-DTW kernels also map a NaN
// from overflowing finite inputs to a non-NaN value before storing a slot, so
// no wait can be set off by data.
__device__ __forceinline__ bool is_nan_bits(uint32_t bits) { return (bits & 0x7fffffffu) > 0x7f800000u; }

// Spin (warp-uniform) until no lane reports `missing`; `reload` re-reads the
// lane's slot and returns whether it is still missing.  Bounded: after `limit`
// rounds, or once another warp raised the abort word, records a timeout and
// returns false.
template <typename Reload>
__device__ __forceinline__ bool wait_filled(bool missing, Reload reload, WsHeader* hdr, int where,
                                            long long limit = kSpinLimit)
{
    if (!__any_sync(FULL, missing)) return true;
    long long spins = 0;
    for (;;) {
        __nanosleep(64);
        if (missing) missing = reload();
        if (!__any_sync(FULL, missing)) return true;
        if (ld_volatile(&hdr->abort)) return false;
        if (++spins > limit) {
            if ((threadIdx.x & 31) == 0) {
                atomicExch(&hdr->status, kDevTimeout);
                atomicExch(&hdr->timeout_where, where);
                atomicExch(&hdr->abort, 1);
            }
            return false;
        }
    }
}

// floor(a / b) and ceil(a / b) for b > 0 and any sign of a
__device__ __forceinline__ int64_t floor_div64(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int64_t ceil_div64(int64_t a, int64_t b) { return -floor_div64(-a, b); }

// Sakoe-Chiba band of an M x N pair with bound bnd: row i keeps the columns
// [band_lo(i), band_hi(i)] (clipped to the matrix), both nondecreasing in i.
__device__ __forceinline__ int band_lo(int64_t i, int64_t bnd, int M, int N)
{
    return (int)max((int64_t)0, ceil_div64(i * N - bnd, M));
}
__device__ __forceinline__ int band_hi(int64_t i, int64_t bnd, int M, int N)
{
    return (int)min((int64_t)N - 1, floor_div64(i * N + bnd, M));
}

// The rows inside the band at a column j that moves by one a step, without a
// division per step: row i is in the band at column j iff
// ceil((jM - bnd) / N) <= i <= floor((jM + bnd) / N).  qa and qb are those two
// quotients, ra = qa N - (jM - bnd) and rb = (jM + bnd) - qb N their
// remainders in [0, N); dq, dr = M / N, M % N.  |bnd| <= MN keeps every field
// within 32 bits.
struct BandRows {
    int qa, ra, qb, rb, dq, dr;
    __device__ __forceinline__ void init(int64_t j, int64_t bnd, int M, int N)
    {
        const int64_t A = j * M - bnd, B = j * M + bnd;
        const int64_t a = ceil_div64(A, N), b = floor_div64(B, N);
        qa = (int)a;
        ra = (int)(a * N - A);
        qb = (int)b;
        rb = (int)(B - b * N);
        dq = M / N;
        dr = M % N;
    }
    __device__ __forceinline__ void next(int N)      // j + 1
    {
        const bool ca = dr > ra, cb = rb + dr >= N;
        qa += dq + (int)ca;
        ra += ca ? N - dr : -dr;
        qb += dq + (int)cb;
        rb += cb ? dr - N : dr;
    }
    __device__ __forceinline__ void prev(int N)      // j - 1
    {
        const bool ca = ra + dr >= N, cb = rb < dr;
        qa -= dq + (int)ca;
        ra += ca ? dr - N : dr;
        qb -= dq + (int)cb;
        rb += cb ? N - dr : -dr;
    }
};

// Work list: items are (pair, band) in the order pairs[order[0]], bands 0..,
// pairs[order[1]], ...; prefix[q] = first item of the q-th pair in that order.
__device__ __forceinline__ int find_slot(const int32_t* prefix, int n, int item)
{
    int lo = 0, hi = n;                      // prefix[lo] <= item < prefix[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace wts
