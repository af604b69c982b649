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
// guarded by a per-band progress counter with release/acquire ordering.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wts {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kMaxD = 16;              // channels handled (zero-padded up to the template D)
constexpr long long kSpinLimit = 1ll << 27;   // polls before a wait gives up (~tens of seconds)

// Device status word values (first word of every workspace).
enum DevStatus : int { kDevOk = 0, kDevTimeout = 1 };

// One alignment problem of a batch.
struct PairDesc {
    const float* X;      // rows, [M][d]
    const float* Y;      // columns, [N][d]
    int32_t M, N;
    int32_t nbands;      // ceil(M / BR)
    int32_t out;         // output slot (cycle index, or pair index for pairwise)
    int64_t dir_off;     // first direction word of this pair
    int64_t hbuf_off;    // first float of this pair's hand-off rows ((nbands-1) * N)
    int64_t aux_off;     // first element of per-pair auxiliary storage (R store / flags base)
    int32_t flag_off;    // first progress counter of this pair (nbands counters)
    int32_t pad;
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

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile(const int* p)
{
    int v;
    asm volatile("ld.volatile.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait (warp-uniform) until *flag >= need.  Every lane polls the same word.
// Gives up after kSpinLimit polls or when another warp has raised the abort
// word: then records a timeout and returns false.
__device__ __forceinline__ bool wait_progress(const int* flag, int need, WsHeader* hdr, int where)
{
    if (ld_acquire(flag) >= need) return true;
    long long spins = 0;
    for (;;) {
        __nanosleep(128);
        if (ld_acquire(flag) >= need) return true;
        if (ld_volatile(&hdr->abort)) return false;
        if (++spins > kSpinLimit) {
            if ((threadIdx.x & 31) == 0) {
                atomicExch(&hdr->status, kDevTimeout);
                atomicExch(&hdr->timeout_where, where);
                atomicExch(&hdr->abort, 1);
            }
            return false;
        }
    }
}

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
