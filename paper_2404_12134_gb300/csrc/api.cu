// C ABI entry points: validation, workspace layout, launches.
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/wetsand.h"
#include "dba.cuh"
#include "dtw_wavefront.cuh"
#include "plan.cuh"
#include "softdtw.cuh"

namespace wts {
int run_probe(int which, double* ops_per_s);
size_t compact_workspace_bytes(int64_t rows);
cudaError_t launch_pad_last(const float* in, const int64_t* offsets, int T, int d, int64_t L, float* out,
                            cudaStream_t st);
cudaError_t launch_select_channel(const float* in, int64_t rows, int d, int c, float* out, cudaStream_t st);
cudaError_t launch_compact_nan(const float* in, const int64_t* in_offsets, int T, int d, int64_t rows, float* out,
                               int64_t* out_offsets, void* ws, cudaStream_t st);
namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int ok()
{
    g_err.clear();
    return WTS_OK;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(WTS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Opt-in kernel timing: a CUDA event pair recorded on the launching stream
// around every kernel launch while enabled; read (and cleared) per kernel.
struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
    int kernels;
};
std::mutex g_prof_mu;
bool g_prof = false;
std::vector<ProfRec> g_recs;

struct Prof {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st;
    const char* name;
    int kernels = 1;             // kernel launches inside the region
    Prof(const char* n, cudaStream_t s) : st(s), name(n)
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        if (!g_prof) return;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) { a = b = nullptr; return; }
        cudaEventRecord(a, st);
    }
    ~Prof()
    {
        if (!a) return;
        cudaEventRecord(b, st);
        std::lock_guard<std::mutex> g(g_prof_mu);
        g_recs.push_back({name, a, b, kernels});
    }
};

int pick_D(int d)
{
    static const int Ds[] = {1, 2, 3, 4, 6, 8, 12, 16};
    for (int D : Ds)
        if (D >= d) return D;
    return 0;
}

int pick_R(int D, const wts_options* opt)
{
    if (opt && opt->rows_per_thread) return opt->rows_per_thread;
    return D <= 2 ? 32 : 16;
}

int check_batch(const wts_batch* Y, bool need_device)
{
    if (!Y) return fail(WTS_EINVAL, "batch is NULL");
    if (Y->T < 1) return fail(WTS_EINVAL, "batch has T=%d cycles (need >= 1)", Y->T);
    if (Y->d < 1 || Y->d > kMaxD) return fail(WTS_EINVAL, "d=%d outside 1..%d", Y->d, kMaxD);
    if (!Y->offsets_host) return fail(WTS_EINVAL, "batch offsets_host is NULL");
    if (need_device && (!Y->data || !Y->offsets)) return fail(WTS_EINVAL, "batch data/offsets is NULL");
    if (Y->offsets_host[0] != 0) return fail(WTS_EINVAL, "offsets[0] must be 0");
    for (int k = 0; k < Y->T; ++k) {
        const int64_t n = Y->offsets_host[k + 1] - Y->offsets_host[k];
        if (n < 1) return fail(WTS_EINVAL, "cycle %d has length %lld (need >= 1)", k, (long long)n);
        if (n > (int64_t)1 << 30) return fail(WTS_EINVAL, "cycle %d too long (%lld)", k, (long long)n);
    }
    return WTS_OK;
}

int check_opt(const wts_options* opt, int D)
{
    if (!opt) return WTS_OK;
    if (opt->rows_per_thread && opt->rows_per_thread != 4 && opt->rows_per_thread != 8 &&
        opt->rows_per_thread != 16 && opt->rows_per_thread != 32)
        return fail(WTS_EINVAL, "rows_per_thread must be 0, 4 (Sub-DTW), 8, 16 or 32");
    if (opt->rows_per_thread == 32 && D > 3) return fail(WTS_EINVAL, "rows_per_thread=32 needs d <= 3");
    if (opt->warps_per_block < 0 || opt->warps_per_block > 4) return fail(WTS_EINVAL, "warps_per_block must be 0..4");
    if (opt->max_blocks < 0) return fail(WTS_EINVAL, "max_blocks must be >= 0");
    if (opt->dir_mode < 0 || opt->dir_mode > 1) return fail(WTS_EINVAL, "dir_mode must be 0 or 1");
    if (opt->ckpt_bands < 0) return fail(WTS_EINVAL, "ckpt_bands must be >= 0");
    if (opt->spin_limit < 0) return fail(WTS_EINVAL, "spin_limit must be >= 0");
    if (!(opt->band >= 0.0) || opt->band > 1e6) return fail(WTS_EINVAL, "band must be a finite value >= 0");
    if (opt->cost_kind != WTS_COST_SQEUCLID && opt->cost_kind != WTS_COST_L2)
        return fail(WTS_EINVAL, "cost_kind must be 0 (squared l2) or 1 (l2 norm), got %d", opt->cost_kind);
    if (opt->score_via_codes != 0 && opt->score_via_codes != 1) return fail(WTS_EINVAL, "score_via_codes must be 0 or 1");
    if (opt->store_pairs < 0) return fail(WTS_EINVAL, "store_pairs must be >= 0");
    return WTS_OK;
}

// Layout of the workspace for one call (host side; mirrors the setup kernel).
int compute_layout(int op, int64_t M, const wts_batch* Y, const wts_options* opt, Layout* L)
{
    int rc = check_batch(Y, false);
    if (rc) return rc;
    const int D = pick_D(Y->d);
    rc = check_opt(opt, D);
    if (rc) return rc;
    if (op != kOpPairwise && (M < 1 || M > (int64_t)1 << 30)) return fail(WTS_EINVAL, "M=%lld out of range", (long long)M);
    if (op == kOpPairwise && Y->T < 2) return fail(WTS_EINVAL, "pairwise DTW needs T >= 2");
    if (op == kOpPairwise && Y->T > 4096) return fail(WTS_EINVAL, "pairwise DTW limited to T <= 4096");
    // the score through stored codes: dtw_align's layout (codes, walk state,
    // ranges, costs) plus |pi| per cycle
    const bool via_codes = op == kOpScore && opt && opt->score_via_codes;
    if (via_codes) op = kOpDba;
    *L = Layout{};
    L->op = op;
    L->T = Y->T;
    L->P = op == kOpPairwise ? Y->T * (Y->T - 1) / 2 : Y->T;
    L->d = Y->d;
    L->D = D;
    L->R = pick_R(D, opt);
    if (op != kOpSubdtw && opt && opt->rows_per_thread == 4)
        return fail(WTS_EINVAL, "rows_per_thread = 4 is for Sub-DTW only");
    if (op == kOpSubdtw) {
        if (opt && opt->rows_per_thread && opt->rows_per_thread != 16 && opt->rows_per_thread != 8 &&
            opt->rows_per_thread != 4)
            return fail(WTS_EINVAL, "Sub-DTW runs with rows_per_thread = 4, 8 or 16 (got %d)", opt->rows_per_thread);
        if (opt && opt->dir_mode == 1) return fail(WTS_EINVAL, "Sub-DTW keeps every code (dir_mode must be 0)");
        L->R = (opt && (opt->rows_per_thread == 8 || opt->rows_per_thread == 4)) ? opt->rows_per_thread : 16;
    }
    if (op == kOpSoft) {
        if (D > 8) return fail(WTS_EINVAL, "soft-DTW supports d <= 8 (got %d)", Y->d);
        L->R = soft_rows(D);          // fixed by the channel count (registers)
    }
    if (opt && opt->band > 0) {
        if (op != kOpSoft) {
            if (opt->rows_per_thread && opt->rows_per_thread != 16)
                return fail(WTS_EINVAL, "with a band, rows_per_thread must be 0 or 16 (got %d)", opt->rows_per_thread);
            L->R = 16;
        } else if (opt->band < kSoftNarrowBand) {
            L->R = 4;
        }
        L->banded = 1;
    }
    if (opt && opt->cost_kind == WTS_COST_L2) {
        if (op != kOpSoft) {
            if (opt->rows_per_thread && opt->rows_per_thread != 16)
                return fail(WTS_EINVAL, "with the l2-norm cost, rows_per_thread must be 0 or 16 (got %d)",
                            opt->rows_per_thread);
            L->R = 16;
        }
        L->cost_kind = WTS_COST_L2;
    }
    L->BR = 32 * L->R;
    L->M = M;
    const int64_t* o = Y->offsets_host;
    // soft-DTW column checkpoints: the first store_pairs pairs of the work
    // list's order (longest first, or the batch order) keep R; the setup
    // kernel takes the same ranks
    std::vector<char> keep_r;
    if (opt && opt->store_pairs) {
        if (op != kOpSoft || opt->dir_mode != 1 || opt->band > 0)
            return fail(WTS_EINVAL, "store_pairs applies to soft-DTW with dir_mode = 1 and no band");
        L->store_pairs = opt->store_pairs < L->P ? opt->store_pairs : L->P;
        std::vector<int> idx(L->P);
        for (int p = 0; p < L->P; ++p) idx[p] = p;
        if (!opt->keep_batch_order)
            std::sort(idx.begin(), idx.end(), [&](int q, int p) {
                return longer_first(M * (o[q + 1] - o[q]), q, M * (o[p + 1] - o[p]), p);
            });
        keep_r.assign(L->P, 0);
        for (int r = 0; r < L->store_pairs; ++r) keep_r[idx[r]] = 1;
    }
    int64_t items = 0, h = 0, dw = 0, rs = 0;
    for (int p = 0; p < L->P; ++p) {
        int64_t Mp, Np;
        if (op == kOpPairwise) {
            int a = 0, rem = p;
            while (rem >= L->T - 1 - a) { rem -= L->T - 1 - a; ++a; }
            const int b = a + 1 + rem;
            Mp = o[a + 1] - o[a];
            Np = o[b + 1] - o[b];
        } else {
            Mp = M;
            Np = o[p + 1] - o[p];
        }
        if (opt && opt->band > 0) {
            if (op != kOpScore && op != kOpAlign && op != kOpDba && op != kOpSoft)
                return fail(WTS_EINVAL, "the band applies to the DTW and soft-DTW operations only");
            const int64_t bb = band_bound_of(opt->band, Mp, Np);
            if (bb < (Mp > Np ? Mp : Np))
                return fail(WTS_EINVAL, "band %g too narrow for pair %d (%lld x %lld): floor(band M N) = %lld < "
                            "max(M, N)", opt->band, p, (long long)Mp, (long long)Np, (long long)bb);
        }
        const int64_t nb = cdiv(Mp, L->BR);
        items += nb;
        h += pair_hbuf_slots(nb, Np);
        if (op == kOpAlign || op == kOpDba || op == kOpSubdtw) {
            const int64_t G = (opt && opt->dir_mode == 1) ? (opt->ckpt_bands ? opt->ckpt_bands : 16) : 0;
            dw += pair_dir_words(G > 0 ? (G < nb ? G : nb) : nb, Np, L->R);
        }
        if (op == kOpSoft) {
            // checkpoint mode: column checkpoints of every band (no band), or
            // two buffers of G bands (with a band: one group's R is read while
            // the next group's is recomputed)
            const int64_t G = (opt && opt->dir_mode == 1) ? (opt->ckpt_bands ? opt->ckpt_bands : 16) : 0;
            if (G > 0 && !(opt->band > 0) && !(L->store_pairs && keep_r[p]))
                rs += nb * band_ckcol_floats(Np, L->R);
            else
                rs += pair_rstore_floats(G > 0 && !(L->store_pairs && keep_r[p]) ? (2 * G < nb ? 2 * G : nb) : nb,
                                         Np, L->R);
        }
    }
    if (items >= ((int64_t)1 << 31)) return fail(WTS_EINVAL, "too many work items");
    L->n_items = items;
    L->hbuf_slots = h;
    L->dir_words = dw;
    L->rstore_floats = rs;
    // hand-off slot: r (4 bytes), or {r, path cells} (8 bytes) when |pi| is counted
    L->hbuf_bytes = (size_t)h * (op == kOpScore ? 8 : 4);
    L->ebuf_bytes = op == kOpSoft ? (size_t)h * 16 : 0;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
    L->off_hdr = take(sizeof(WsHeader));
    L->off_pairs = take((size_t)L->P * sizeof(PairDesc));
    L->off_order = take((size_t)L->P * sizeof(int32_t));
    L->off_prefix = take((size_t)(L->P + 1) * sizeof(int32_t));
    L->off_hbuf = take(L->hbuf_bytes);
    if (op == kOpAlign || op == kOpDba || op == kOpSubdtw) {
        L->off_dirs = take((size_t)dw * sizeof(uint32_t));
        if (opt && opt->dir_mode == 1) {
            L->group_bands = opt->ckpt_bands ? opt->ckpt_bands : 16;
            L->off_btstate = take((size_t)L->T * 3 * sizeof(int32_t));
        } else if (op != kOpSubdtw) {
            L->nseg = (int)cdiv(M, kBtSegRows);
            L->off_seg = take((size_t)L->P * L->nseg * 4 * sizeof(int32_t));
        }
    }
    if (op == kOpDba) {
        L->off_jlo = take((size_t)L->T * M * sizeof(int32_t));
        L->off_jhi = take((size_t)L->T * M * sizeof(int32_t));
        L->off_costs = take((size_t)L->T * sizeof(float));
    }
    if (op == kOpSoft) {
        if (opt && opt->dir_mode == 1) L->group_bands = opt->ckpt_bands ? opt->ckpt_bands : 16;
        L->soft_fused = L->group_bands > 0 && !L->banded;
        L->off_rstore = take((size_t)rs * sizeof(float));
        L->off_gpart = take((size_t)L->T * M * D * sizeof(float));
        L->off_ebuf = take(L->ebuf_bytes);
        L->off_pcost = take((size_t)L->T * sizeof(float));
    }
    if (via_codes) L->off_plen = take((size_t)L->T * sizeof(int32_t));
    L->total = off;
    return WTS_OK;
}

int check_ws(const Layout& L, const void* ws, size_t bytes)
{
    if (!ws) return fail(WTS_EINVAL, "workspace is NULL");
    if (((uintptr_t)ws & 255) != 0) return fail(WTS_EINVAL, "workspace must be 256-byte aligned");
    if (bytes < L.total) return fail(WTS_ENOMEM, "workspace has %zu bytes, needs %zu", bytes, L.total);
    return WTS_OK;
}

struct DevInfo {
    int sms = 0;
};

int device_info(DevInfo* di)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    e = cudaDeviceGetAttribute(&di->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    return WTS_OK;
}

// Reset header + progress counters, build the work list.
int prepare(const Layout& L, char* ws, const float* B, const wts_batch* Y, const wts_options* opt,
            cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(ws + L.off_hdr, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace header)");
    // hand-off rows start as NaN: a slot is valid once its producer wrote it
    if (L.hbuf_bytes) {
        e = cudaMemsetAsync(ws + L.off_hbuf, 0xFF, L.hbuf_bytes, st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(hand-off rows)");
    }
    // every sample must be finite (Sec. 3.1 removes missing values first): a
    // non-finite one sets the status and abort words, and every kernel of the
    // call then leaves at once
    DevInfo di;
    int rc = device_info(&di);
    if (rc) return rc;
    {
        Prof pr("setup", st);
        e = launch_check_finite(B, B ? L.M * L.d : 0, Y->data, Y->offsets_host[Y->T] * Y->d,
                                reinterpret_cast<WsHeader*>(ws + L.off_hdr), di.sms, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "input check launch");
    SetupParams sp{};
    sp.op = L.op;
    sp.T = L.T;
    sp.P = L.P;
    sp.d = L.d;
    sp.R = L.R;
    sp.BR = L.BR;
    sp.M = L.M;
    sp.B = B;
    sp.data = Y->data;
    sp.offsets = Y->offsets;
    sp.pairs = reinterpret_cast<PairDesc*>(ws + L.off_pairs);
    sp.order = reinterpret_cast<int32_t*>(ws + L.off_order);
    sp.prefix = reinterpret_cast<int32_t*>(ws + L.off_prefix);
    sp.sort = (opt && opt->keep_batch_order) ? 0 : 1;
    sp.group_bands = L.group_bands;
    sp.band = opt ? opt->band : 0.0;
    sp.store_pairs = L.store_pairs;
    {
        Prof pr("setup", st);
        launch_setup(sp, st);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "setup kernel launch");
    return WTS_OK;
}

int grid_for(int mode, const Layout& L, const wts_options* opt, int* grid, int* block, int64_t n_items = -1)
{
    if (n_items < 0) n_items = L.n_items;
    DevInfo di;
    int rc = device_info(&di);
    if (rc) return rc;
    const int wpb = (opt && opt->warps_per_block) ? opt->warps_per_block : 4;
    *block = 32 * wpb;
    int occ = dtw_wavefront_max_blocks_per_sm(mode, L.D, L.R, *block, L.banded, L.cost_kind);
    if (occ < 1) return fail(WTS_ECUDA, "no resident block for D=%d R=%d block=%d", L.D, L.R, *block);
    int64_t g = (int64_t)occ * di.sms;
    const int64_t need = (n_items + wpb - 1) / wpb;
    if (g > need) g = need;
    if (opt && opt->max_blocks && g > opt->max_blocks) g = opt->max_blocks;
    *grid = (int)(g < 1 ? 1 : g);
    return WTS_OK;
}

long long spin_limit_of(const wts_options* opt)
{
    return (opt && opt->spin_limit > 0) ? (long long)opt->spin_limit : kSpinLimit;
}

DPParams base_params(const Layout& L, char* ws, const wts_options* opt = nullptr)
{
    DPParams p{};
    p.spin_limit = spin_limit_of(opt);
    p.skip_handoff = (opt && opt->fault_skip_handoff) ? 1 : 0;
    p.pairs = reinterpret_cast<const PairDesc*>(ws + L.off_pairs);
    p.order = reinterpret_cast<const int32_t*>(ws + L.off_order);
    p.prefix = reinterpret_cast<const int32_t*>(ws + L.off_prefix);
    p.P = L.P;
    p.n_items = (int)L.n_items;
    p.d = L.d;
    p.hdr = reinterpret_cast<WsHeader*>(ws + L.off_hdr);
    p.hbuf = ws + L.off_hbuf;
    p.dirs = L.off_dirs ? reinterpret_cast<uint32_t*>(ws + L.off_dirs) : nullptr;
    p.T = L.T;
    p.banded = L.banded;
    p.cost_kind = L.cost_kind;
    return p;
}

int launch_dp(int mode, const Layout& L, const DPParams& p0, const wts_options* opt, cudaStream_t st)
{
    int grid = 0, block = 0;
    int rc = grid_for(mode, L, opt, &grid, &block, p0.n_items);
    if (rc) return rc;
    DPParams p = p0;
    // Every pair of a shared-prototype launch has the same bands: take the
    // pairs in groups whose items about fill the resident warps once,
    // band-major within a group (measured: batched DBA, 200 x 25k x 6 ch,
    // wavefront 74.1 -> 70.7 ms against pair after pair).  Under a band
    // every pair's band b comes before any band b + 1 (one group).
    if (L.op != kOpPairwise && L.M > 0) {
        const int64_t nb = p.recompute ? p.band_cnt : cdiv(L.M, L.BR);
        const int64_t warps = (int64_t)grid * (block / 32);
        p.group_pairs = p.banded ? L.P : (int)std::max<int64_t>(1, std::min<int64_t>(L.P, warps / nb));
    }
    cudaError_t e;
    {
        Prof pr(p.recompute ? "wavefront_recompute" : "wavefront", st);
        e = launch_dtw_wavefront(mode, L.D, L.R, p, grid, block, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "wavefront launch");
    return WTS_OK;
}

// Shared body of dtw_align and dba_iterate: directions + backtrack.
int align_into(const Layout& L, char* ws, const float* B, const wts_batch* Y, const wts_options* opt,
               cudaStream_t st, float* cost, int32_t* plen, int32_t* jlo, int32_t* jhi)
{
    int rc = prepare(L, ws, B, Y, opt, st);
    if (rc) return rc;
    DPParams p = base_params(L, ws, opt);
    p.cost_out = cost;
    BTParams bt{};
    bt.pairs = p.pairs;
    bt.P = L.P;
    bt.R = L.R;
    bt.dirs = p.dirs;
    bt.jlo = jlo;
    bt.jhi = jhi;
    bt.plen = plen;
    bt.M = L.M;
    bt.hdr = p.hdr;
    cudaError_t e;
    if (L.group_bands == 0) {
        // every cell's code stored, one backtrack
        rc = launch_dp(kModeDirs, L, p, opt, st);
        if (rc) return rc;
        bt.band_lo = 0;
        bt.band_hi = (int)cdiv(L.M, L.BR);
        // segmented walk: nseg rounds (a round only re-walks the segments
        // whose start changed), then |pi| from the ranges; a single segment
        // is one plain walk per pair
        bt.nseg = L.nseg > 1 ? L.nseg : 0;
        bt.seg_rows = kBtSegRows;
        bt.seg = reinterpret_cast<int32_t*>(ws + L.off_seg);
        if (bt.nseg == 0) {
            Prof pr("backtrack", st);
            e = launch_backtrack(bt, st);
        } else {
            Prof pr("backtrack", st);
            pr.kernels = L.nseg + 1;
            for (int r = 0; r < L.nseg; ++r) {
                bt.round = r;
                e = launch_backtrack(bt, st);
                if (e != cudaSuccess) break;
            }
            if (e == cudaSuccess) e = launch_backtrack_seg_final(bt, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "backtrack launch");
        return WTS_OK;
    }
    // checkpoint mode: a cost-only pass leaves every band's bottom row in the
    // hand-off rows; then, from the last band up, the codes of G bands (all
    // pairs at once) are recomputed from those rows and the walk continues
    // through them
    rc = launch_dp(kModeCost, L, p, opt, st);
    if (rc) return rc;
    const int nb = (int)cdiv(L.M, L.BR);
    const int G = L.group_bands;
    bt.state = reinterpret_cast<int32_t*>(ws + L.off_btstate);
    for (int hi = nb; hi > 0; hi -= G) {
        const int lo = hi - G > 0 ? hi - G : 0;
        DPParams r = p;
        r.recompute = 1;
        r.band_lo = lo;
        r.band_cnt = hi - lo;
        r.n_items = L.P * (hi - lo);
        r.cost_out = nullptr;
        // every launch starts the work-list cursor from zero
        e = cudaMemsetAsync(ws + L.off_hdr + offsetof(WsHeader, item_counter), 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work cursor)");
        rc = launch_dp(kModeDirs, L, r, opt, st);
        if (rc) return rc;
        bt.band_lo = lo;
        bt.band_hi = hi;
        bt.first = hi == nb;
        {
            Prof pr("backtrack", st);
            e = launch_backtrack(bt, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "backtrack launch");
    }
    return WTS_OK;
}

SoftParams soft_params(const Layout& L, char* ws, float gamma, const wts_options* opt = nullptr)
{
    SoftParams p{};
    p.spin_limit = spin_limit_of(opt);
    p.skip_handoff = (opt && opt->fault_skip_handoff) ? 1 : 0;
    p.pairs = reinterpret_cast<const PairDesc*>(ws + L.off_pairs);
    p.order = reinterpret_cast<const int32_t*>(ws + L.off_order);
    p.prefix = reinterpret_cast<const int32_t*>(ws + L.off_prefix);
    p.P = L.P;
    p.n_items = (int)L.n_items;
    p.d = L.d;
    p.gamma = gamma;
    p.hdr = reinterpret_cast<WsHeader*>(ws + L.off_hdr);
    p.hbuf = reinterpret_cast<float*>(ws + L.off_hbuf);
    p.ebuf = reinterpret_cast<float*>(ws + L.off_ebuf);
    p.rstore = reinterpret_cast<float*>(ws + L.off_rstore);
    p.gpart = reinterpret_cast<float*>(ws + L.off_gpart);
    p.banded = L.banded;
    p.cost_kind = L.cost_kind;
    p.rows = L.R;
    p.m_aligned = (L.M % L.R) == 0 ? 1 : 0;
    if (L.soft_fused) {                   // the checkpoint area holds column checkpoints
        p.ckcol = reinterpret_cast<float*>(ws + L.off_rstore);
        p.fused = 1;
    }
    return p;
}

int soft_grid(const Layout& L, int backward, const wts_options* opt, int* grid, int* block, int64_t n_items = -1)
{
    if (n_items < 0) n_items = L.n_items;
    const int fused = L.soft_fused;
    DevInfo di;
    int rc = device_info(&di);
    if (rc) return rc;
    const int wpb = (opt && opt->warps_per_block) ? opt->warps_per_block : 4;
    *block = 32 * wpb;
    const int occ = softdtw_max_blocks_per_sm(L.D, backward, *block, L.banded, L.cost_kind, fused, L.R);
    if (occ < 1) return fail(WTS_ECUDA, "no resident soft-DTW block for D=%d block=%d", L.D, *block);
    int64_t g = (int64_t)occ * di.sms;
    const int64_t need = (n_items + wpb - 1) / wpb;
    if (g > need) g = need;
    if (opt && opt->max_blocks && g > opt->max_blocks) g = opt->max_blocks;
    *grid = (int)(g < 1 ? 1 : g);
    return WTS_OK;
}

// The caller-visible code of a workspace's device status word.
int status_of(const WsHeader& h)
{
    return h.status == kDevTimeout ? WTS_ETIMEOUT : (h.status == kDevBadInput ? WTS_EINVAL : WTS_OK);
}

int check_gamma(float gamma)
{
    if (!(gamma > 0.f) || !(gamma < 1e30f)) return fail(WTS_EINVAL, "gamma must be finite and > 0 (gamma = 0 is DTW)");
    return WTS_OK;
}

}  // namespace
}  // namespace wts

using namespace wts;

extern "C" {

int wts_version(void) { return 100; }

const char* wts_last_error(void) { return g_err.c_str(); }

int wts_profile_enable(int enable)
{
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof = enable != 0;
    return ok();
}

int wts_profile_read(const char* kernel, double* total_ms, int32_t* launches)
{
    if (!kernel || !total_ms || !launches) return fail(WTS_EINVAL, "NULL argument");
    std::vector<ProfRec> mine;
    {
        std::lock_guard<std::mutex> g(g_prof_mu);
        std::vector<ProfRec> keep;
        for (auto& r : g_recs) (r.name == kernel || kernel[0] == 0 ? mine : keep).push_back(r);
        g_recs.swap(keep);
    }
    double tot = 0;
    int err = WTS_OK;
    int32_t kernels = 0;
    for (auto& r : mine) {
        kernels += r.kernels;
        float ms = 0;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess && err == WTS_OK) err = cuda_fail(e, "reading kernel events");
        tot += ms;
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    *total_ms = tot;
    *launches = kernels;
    return err ? err : ok();
}

int wts_peak_probe(int which, double* ops_per_s)
{
    if (!ops_per_s || which < 0 || which > 5) return fail(WTS_EINVAL, "which must be 0..5");
    if (run_probe(which, ops_per_s)) return fail(WTS_ECUDA, "probe kernel failed");
    return ok();
}

namespace {

// After the soft-DTW workspace: values [T], weights [T], gradient [M][d] (FP32).
size_t lbfgs_extra_bytes(int64_t M, const wts_batch* Y)
{
    return 2 * align256((size_t)Y->T * sizeof(float)) + align256((size_t)M * Y->d * sizeof(float));
}

// After the soft-DTW workspace: Adam's moments m, v and the gradient ([M][d]
// each, FP32), then the values of one step [T] when the caller keeps none.
size_t adam_extra_bytes(int64_t M, const wts_batch* Y)
{
    return 3 * align256((size_t)M * Y->d * sizeof(float)) + align256((size_t)Y->T * sizeof(float));
}

}  // namespace

int wts_workspace_size(int op, int64_t M, const wts_batch* Y, const wts_options* opt, size_t* bytes)
{
    if (!bytes) return fail(WTS_EINVAL, "bytes is NULL");
    static const int map[] = {0, kOpScore, kOpAlign, kOpDba, kOpSoft, kOpPairwise, 0, kOpSubdtw, kOpSoft, kOpSoft};
    if (op == WTS_OP_COMPACT_NAN) {
        int rc = check_batch(Y, false);
        if (rc) return rc;
        *bytes = align256(compact_workspace_bytes(Y->offsets_host[Y->T]));
        return ok();
    }
    if (op < 1 || op > 9 || op == WTS_OP_COMPACT_NAN) return fail(WTS_EINVAL, "unknown op %d", op);
    Layout L;
    int rc = compute_layout(map[op], M, Y, opt, &L);
    if (rc) return rc;
    *bytes = L.total;
    if (op == WTS_OP_SOFTDTW_LBFGS) *bytes += lbfgs_extra_bytes(M, Y);
    if (op == WTS_OP_SOFTDTW_ADAM) *bytes += adam_extra_bytes(M, Y);
    return ok();
}

int wts_read_status(const void* workspace, void* stream, int32_t* status)
{
    if (!workspace || !status) return fail(WTS_EINVAL, "NULL argument");
    WsHeader h;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "reading workspace status");
    *status = status_of(h);
    return ok();
}

int anomaly_score(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
                  void* workspace, size_t workspace_bytes, void* stream,
                  float* score, float* cost, int32_t* plen)
{
    Layout L;
    int rc = compute_layout(kOpScore, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!B || !score) return fail(WTS_EINVAL, "B and score must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    if (opt && opt->score_via_codes) {
        // codes + walk: the same DTW cost, |pi| from the walked ranges, the
        // same FP32 division
        float* c = cost ? cost : reinterpret_cast<float*>(ws + L.off_costs);
        int32_t* pl = plen ? plen : reinterpret_cast<int32_t*>(ws + L.off_plen);
        if ((rc = align_into(L, ws, B, Y, opt, st, c, pl, reinterpret_cast<int32_t*>(ws + L.off_jlo),
                             reinterpret_cast<int32_t*>(ws + L.off_jhi))))
            return rc;
        cudaError_t e;
        {
            Prof pr("score_divide", st);
            e = launch_score_divide(c, pl, score, L.T, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "score division launch");
        return ok();
    }
    if ((rc = prepare(L, ws, B, Y, opt, st))) return rc;
    DPParams p = base_params(L, ws, opt);
    p.cost_out = cost;
    p.plen_out = plen;
    p.score_out = score;
    if ((rc = launch_dp(kModePlen, L, p, opt, st))) return rc;
    return ok();
}

int dtw_align(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
              void* workspace, size_t workspace_bytes, void* stream,
              float* cost, int32_t* plen, int32_t* jlo, int32_t* jhi)
{
    Layout L;
    int rc = compute_layout(kOpAlign, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!B || !jlo || !jhi) return fail(WTS_EINVAL, "B, jlo and jhi must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    if ((rc = align_into(L, (char*)workspace, B, Y, opt, (cudaStream_t)stream, cost, plen, jlo, jhi))) return rc;
    return ok();
}

namespace {

// Sub-DTW in two halves: the wavefront (cost, b*) and the backtrack (a*, the
// path), so that the segmentation loop can overlap a window's backtrack with
// the next window's wavefront.
int subdtw_dp_part(const Layout& L, char* ws, const float* X, const wts_batch* Y, const wts_options* opt,
                   cudaStream_t st, float* cost, int32_t* b_star)
{
    int rc = prepare(L, ws, X, Y, opt, st);
    if (rc) return rc;
    DPParams p = base_params(L, ws, opt);
    p.cost_out = cost;
    p.bstar_out = b_star;
    return launch_dp(kModeSubDirs, L, p, opt, st);
}

int subdtw_bt_part(const Layout& L, char* ws, const wts_options* opt, cudaStream_t st, const int32_t* b_star,
                   int32_t* a_star, int32_t* plen, int32_t* jlo, int32_t* jhi)
{
    const DPParams p = base_params(L, ws, opt);
    BTParams bt{};
    bt.pairs = p.pairs;
    bt.P = L.P;
    bt.R = L.R;
    bt.dirs = p.dirs;
    bt.jlo = jlo;
    bt.jhi = jhi;
    bt.plen = plen;
    bt.M = L.M;
    bt.band_lo = 0;
    bt.band_hi = (int)cdiv(L.M, L.BR);
    bt.subseq = 1;
    bt.bstar = b_star;
    bt.astar = a_star;
    bt.hdr = p.hdr;
    cudaError_t e;
    {
        Prof pr("backtrack", st);
        e = launch_backtrack(bt, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "backtrack launch");
    return WTS_OK;
}

}  // namespace

int subdtw_align(const float* X, int64_t M, const wts_batch* Y, const wts_options* opt,
                 void* workspace, size_t workspace_bytes, void* stream,
                 float* cost, int32_t* a_star, int32_t* b_star, int32_t* plen, int32_t* jlo, int32_t* jhi)
{
    Layout L;
    int rc = compute_layout(kOpSubdtw, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!X || !a_star || !b_star || !jlo || !jhi) return fail(WTS_EINVAL, "X, a_star, b_star, jlo and jhi must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = subdtw_dp_part(L, ws, X, Y, opt, st, cost, b_star))) return rc;
    if ((rc = subdtw_bt_part(L, ws, opt, st, b_star, a_star, plen, jlo, jhi))) return rc;
    return ok();
}

namespace {

// Workspace of wts_segment: the Sub-DTW layout of one full window (2M
// columns) followed by the window's offsets and outputs.
struct SegLayout {
    Layout L;
    size_t off_offsets, off_cost, off_ab, off_jlo, off_jhi, total;
};

int segment_layout(int64_t M, int32_t d, const wts_options* opt, SegLayout* S)
{
    if (M < 1 || M > ((int64_t)1 << 29)) return fail(WTS_EINVAL, "M=%lld out of range", (long long)M);
    int64_t offs[2] = {0, 2 * M};
    wts_batch b{};
    b.offsets_host = offs;
    b.T = 1;
    b.d = d;
    int rc = compute_layout(kOpSubdtw, M, &b, opt, &S->L);
    if (rc) return rc;
    size_t off = align256(S->L.total);
    auto take = [&](size_t bytes) { size_t at = off; off = align256(off + bytes); return at; };
    S->off_offsets = take(2 * sizeof(int64_t));
    S->off_cost = take(sizeof(float));
    S->off_ab = take(3 * sizeof(int32_t));          // a*, b*, |pi|
    S->off_jlo = take((size_t)M * sizeof(int32_t));
    S->off_jhi = take((size_t)M * sizeof(int32_t));
    S->total = off;
    return WTS_OK;
}

// One window is one pair: the wavefront has only M / (32 R) warps, so the
// shorter serial chain of 4 rows per lane (four times the warps of 16) is the
// default (16 with the l2-norm cost, whose kernels hold 16 rows per lane).
wts_options segment_options(const wts_options* opt)
{
    wts_options o = opt ? *opt : wts_options{};
    if (o.rows_per_thread == 0) o.rows_per_thread = o.cost_kind == WTS_COST_L2 ? 16 : 4;
    return o;
}

}  // namespace

int wts_segment_workspace_size(int64_t M, int32_t d, const wts_options* opt, size_t* bytes)
{
    if (!bytes) return fail(WTS_EINVAL, "bytes is NULL");
    SegLayout S;
    const wts_options o = segment_options(opt);
    int rc = segment_layout(M, d, &o, &S);
    if (rc) return rc;
    *bytes = 2 * S.total;                  // two window slots (see wts_segment)
    return ok();
}

namespace {

struct SegStreams {
    cudaStream_t bt = nullptr;
    cudaEvent_t dp_done = nullptr, freed[2] = {nullptr, nullptr};
    ~SegStreams()
    {
        if (bt) cudaStreamSynchronize(bt);
        if (dp_done) cudaEventDestroy(dp_done);
        for (cudaEvent_t& e : freed)
            if (e) cudaEventDestroy(e);
        if (bt) cudaStreamDestroy(bt);
    }
};

}  // namespace

// Windows alternate between two workspace slots.  A window's wavefront runs on
// the caller's stream; once its b* is read back (it sets the next window), its
// backtrack runs on a second stream while the next window's wavefront starts
// on the first; a slot is reused only after its backtrack has finished.
int wts_segment(const float* X, int64_t M, const float* Ydata, int64_t N, int32_t d, int64_t alpha,
                const wts_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                int32_t max_segments, int64_t* seg_start, int64_t* seg_end, float* seg_cost, int32_t* n_segments)
{
    if (!X || !Ydata || !n_segments || (max_segments > 0 && (!seg_start || !seg_end)))
        return fail(WTS_EINVAL, "X, Ydata, n_segments (and seg_start/seg_end) must not be NULL");
    if (N < 1) return fail(WTS_EINVAL, "N=%lld (need >= 1)", (long long)N);
    if (max_segments < 0) return fail(WTS_EINVAL, "max_segments must be >= 0");
    if (M < 1) return fail(WTS_EINVAL, "M=%lld (need >= 1)", (long long)M);
    if (alpha < 0) alpha = (int64_t)(0.15 * (double)M);   // Sec. 3.2: alpha = 0.15 M
    SegLayout S;
    const wts_options o = segment_options(opt);
    opt = &o;
    int rc = segment_layout(M, d, opt, &S);
    if (rc) return rc;
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return fail(WTS_EINVAL, "workspace must be 256-byte aligned");
    if (workspace_bytes < 2 * S.total)
        return fail(WTS_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, 2 * S.total);
    cudaStream_t st = (cudaStream_t)stream;
    SegStreams ss;
    cudaError_t e = cudaStreamCreateWithFlags(&ss.bt, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ss.dp_done, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ss.freed[k], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "segmentation stream / events");
    // the backtrack stream starts after everything already queued on the caller's stream
    if ((e = cudaEventRecord(ss.dp_done, st)) != cudaSuccess || (e = cudaStreamWaitEvent(ss.bt, ss.dp_done, 0)) != cudaSuccess)
        return cuda_fail(e, "segmentation stream order");

    int64_t offs[2][2];
    int32_t found = 0;
    int64_t pos = 0;
    // the window whose backtrack is in flight: its slot, start, b*, cost
    int prev_slot = -1;
    int64_t prev_pos = 0;
    int32_t prev_b = 0;
    float prev_cost = 0.f;
    auto finish_prev = [&]() -> int {
        char* base = (char*)workspace + (size_t)prev_slot * S.total;
        int32_t a = -1;
        cudaError_t e2 = cudaEventSynchronize(ss.freed[prev_slot]);
        if (e2 == cudaSuccess) e2 = cudaMemcpy(&a, base + S.off_ab, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e2 != cudaSuccess) return cuda_fail(e2, "window start read-back");
        if (a < 0 || a > prev_b) return fail(WTS_ECUDA, "window at %lld gave an invalid piece [%d, %d]",
                                             (long long)prev_pos, a, prev_b);
        if (found < max_segments) {
            seg_start[found] = prev_pos + a;
            seg_end[found] = prev_pos + prev_b;
            if (seg_cost) seg_cost[found] = prev_cost;
        }
        ++found;
        return WTS_OK;
    };
    for (int64_t k = 0; pos < N; ++k) {
        const int slot = (int)(k & 1);
        char* base = (char*)workspace + (size_t)slot * S.total;
        const int64_t n = (pos + 2 * M < N ? pos + 2 * M : N) - pos;
        int64_t* d_offs = reinterpret_cast<int64_t*>(base + S.off_offsets);
        float* d_cost = reinterpret_cast<float*>(base + S.off_cost);
        int32_t* d_ab = reinterpret_cast<int32_t*>(base + S.off_ab);
        if (k >= 2 && (e = cudaStreamWaitEvent(st, ss.freed[slot], 0)) != cudaSuccess)
            return cuda_fail(e, "slot reuse order");
        offs[slot][0] = 0;
        offs[slot][1] = n;
        e = cudaMemcpyAsync(d_offs, offs[slot], sizeof(offs[slot]), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "window offsets copy");
        wts_batch b{};
        b.data = Ydata + pos * d;
        b.offsets = d_offs;
        b.offsets_host = offs[slot];
        b.T = 1;
        b.d = d;
        Layout L;
        if ((rc = compute_layout(kOpSubdtw, M, &b, opt, &L))) return rc;
        if ((rc = check_batch(&b, true))) return rc;
        if ((rc = subdtw_dp_part(L, base, X, &b, opt, st, d_cost, d_ab + 1))) return rc;
        int32_t bstar = 0;
        float c = 0.f;
        WsHeader h;
        e = cudaEventRecord(ss.dp_done, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bstar, d_ab + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&c, d_cost, sizeof(float), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h, base + L.off_hdr, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "window result read-back");
        if (h.status == kDevTimeout) return fail(WTS_ETIMEOUT, "a wait in the window at %lld gave up", (long long)pos);
        if (h.status == kDevBadInput)
            return fail(WTS_EINVAL, "a sample of X or of the window at %lld is not finite", (long long)pos);
        if (bstar < 0 || bstar >= n) return fail(WTS_ECUDA, "window at %lld gave an invalid end %d", (long long)pos, bstar);
        // backtrack of this window on the second stream, after its wavefront
        if ((e = cudaStreamWaitEvent(ss.bt, ss.dp_done, 0)) != cudaSuccess) return cuda_fail(e, "backtrack order");
        if ((rc = subdtw_bt_part(L, base, opt, ss.bt, d_ab + 1, d_ab, d_ab + 2,
                                 reinterpret_cast<int32_t*>(base + S.off_jlo),
                                 reinterpret_cast<int32_t*>(base + S.off_jhi)))) return rc;
        if ((e = cudaEventRecord(ss.freed[slot], ss.bt)) != cudaSuccess) return cuda_fail(e, "backtrack event");
        // the previous window's backtrack ran beside this window's wavefront
        if (prev_slot >= 0 && (rc = finish_prev())) return rc;
        prev_slot = slot;
        prev_pos = pos;
        prev_b = bstar;
        prev_cost = c;
        if (pos + n == N) break;                      // this window reached the end of Y
        const int64_t next = pos + bstar - alpha;
        pos = next > pos ? next : pos + bstar + 1;
    }
    if (prev_slot >= 0 && (rc = finish_prev())) return rc;
    // later work on the caller's stream follows the last backtrack
    if ((e = cudaEventRecord(ss.dp_done, ss.bt)) != cudaSuccess || (e = cudaStreamWaitEvent(st, ss.dp_done, 0)) != cudaSuccess)
        return cuda_fail(e, "segmentation stream order");
    *n_segments = found;
    if (found > max_segments) return fail(WTS_ENOMEM, "%d pieces found, room for %d", found, max_segments);
    return ok();
}

int dba_iterate(const float* B_in, float* B_out, int64_t M, const wts_batch* Y, const wts_options* opt,
                void* workspace, size_t workspace_bytes, void* stream,
                int32_t* counts, double* cost_before, float* cost)
{
    Layout L;
    int rc = compute_layout(kOpDba, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!B_in || !B_out) return fail(WTS_EINVAL, "B_in and B_out must not be NULL");
    if (B_in == B_out) return fail(WTS_EINVAL, "B_out must not alias B_in");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    char* ws = (char*)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t* jlo = reinterpret_cast<int32_t*>(ws + L.off_jlo);
    int32_t* jhi = reinterpret_cast<int32_t*>(ws + L.off_jhi);
    float* costs = reinterpret_cast<float*>(ws + L.off_costs);
    if ((rc = align_into(L, ws, B_in, Y, opt, st, costs, nullptr, jlo, jhi))) return rc;
    cudaError_t e;
    {
        Prof pr("dba_average", st);
        e = launch_dba_average(Y->data, Y->offsets, L.T, L.d, M, jlo, jhi, costs, B_out, counts, cost_before, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "averaging launch");
    if (cost) {
        e = cudaMemcpyAsync(cost, costs, (size_t)L.T * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "cost copy");
    }
    return ok();
}

int wts_pairwise_dtw(const wts_batch* Y, const wts_options* opt, void* workspace, size_t workspace_bytes,
                     void* stream, float* C)
{
    Layout L;
    int rc = compute_layout(kOpPairwise, 0, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!C) return fail(WTS_EINVAL, "C must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    cudaError_t e = cudaMemsetAsync(C, 0, (size_t)L.T * L.T * sizeof(float), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(C)");
    if ((rc = prepare(L, ws, nullptr, Y, opt, st))) return rc;
    DPParams p = base_params(L, ws, opt);
    p.cost_matrix = C;
    if ((rc = launch_dp(kModeCost, L, p, opt, st))) return rc;
    return ok();
}

int softdtw_forward(const float* B, int64_t M, const wts_batch* Y, float gamma, const wts_options* opt,
                    void* workspace, size_t workspace_bytes, void* stream, float* value)
{
    Layout L;
    int rc = compute_layout(kOpSoft, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if ((rc = check_gamma(gamma))) return rc;
    if (!B || !value) return fail(WTS_EINVAL, "B and value must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    if ((rc = prepare(L, ws, B, Y, opt, st))) return rc;
    SoftParams p = soft_params(L, ws, gamma, opt);
    p.value_out = value;
    p.store_r = L.group_bands == 0;      // checkpoint mode keeps only the hand-off rows
    int grid = 0, block = 0;
    if ((rc = soft_grid(L, 0, opt, &grid, &block))) return rc;
    cudaError_t e;
    {
        Prof pr("softdtw_fwd", st);
        e = launch_softdtw_fwd(L.D, p, grid, block, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "soft-DTW forward launch");
    return ok();
}

int softdtw_backward(const float* B, int64_t M, const wts_batch* Y, float gamma, const float* grad_value,
                     const wts_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                     float* grad_B)
{
    Layout L;
    int rc = compute_layout(kOpSoft, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if ((rc = check_gamma(gamma))) return rc;
    if (!B || !grad_B) return fail(WTS_EINVAL, "B and grad_B must not be NULL");
    if ((rc = check_ws(L, workspace, workspace_bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    cudaError_t e = cudaMemsetAsync(ws + L.off_hdr + offsetof(WsHeader, item_counter), 0, sizeof(int), st);
    if (e == cudaSuccess && L.ebuf_bytes) e = cudaMemsetAsync(ws + L.off_ebuf, 0xFF, L.ebuf_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(backward hand-off rows)");
    SoftParams p = soft_params(L, ws, gamma, opt);
    int grid = 0, block = 0;
    if (L.group_bands == 0 || L.soft_fused) {
        // R stored, or (checkpoint mode without a band) recomputed inside
        // each band's warp from the column checkpoints, the pairs that kept R
        // (store_pairs) reading it: one launch
        if ((rc = soft_grid(L, 1, opt, &grid, &block))) return rc;
        {
            Prof pr("softdtw_bwd", st);
            e = launch_softdtw_bwd(L.D, p, grid, block, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "soft-DTW backward launch");
    } else {
        // checkpoint mode: groups of G bands from the last band up.  R of the
        // last group is recomputed first (from the stored hand-off rows); then
        // each launch runs the backward recursion through group q (R buffer
        // q mod 2) and, in the same launch, recomputes group q + 1 into the
        // other buffer: the recompute items read only stored rows and never
        // wait, so they fill the GPU beside the backward's band pipeline.  E
        // hand-off rows persist across launches.
        const int nb = (int)cdiv(M, L.BR);
        const int G = L.group_bands;
        const int Q = (int)cdiv(nb, G);
        auto group = [&](int q, int* lo, int* hi) {
            *hi = nb - q * G;
            *lo = *hi - G > 0 ? *hi - G : 0;
        };
        int lo = 0, hi = 0;
        group(0, &lo, &hi);
        SoftParams r = p;
        r.band_lo = lo;
        r.band_cnt = hi - lo;
        r.n_items = L.P * (hi - lo);
        r.rbuf_band0 = 0;
        r.recompute = 1;
        r.store_r = 1;
        e = cudaMemsetAsync(ws + L.off_hdr + offsetof(WsHeader, item_counter), 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work cursor)");
        if ((rc = soft_grid(L, 0, opt, &grid, &block, r.n_items))) return rc;
        {
            Prof pr("softdtw_fwd_recompute", st);
            e = launch_softdtw_fwd(L.D, r, grid, block, st);
        }
        if (e != cudaSuccess) return cuda_fail(e, "soft-DTW recompute launch");
        for (int q = 0; q < Q; ++q) {
            SoftParams b = p;
            group(q, &lo, &hi);
            b.band_lo = lo;
            b.band_cnt = hi - lo;
            b.n_items = L.P * (hi - lo);
            b.rbuf_band0 = (q & 1) * G;
            b.recompute = 0;
            b.n_rec = 0;
            if (q + 1 < Q) {
                int lo2 = 0, hi2 = 0;
                group(q + 1, &lo2, &hi2);
                b.n_rec = L.P * (hi2 - lo2);
                b.rec_band_lo = lo2;
                b.rec_band_cnt = hi2 - lo2;
                b.rec_rbuf_band0 = ((q + 1) & 1) * G;
            }
            e = cudaMemsetAsync(ws + L.off_hdr + offsetof(WsHeader, item_counter), 0, sizeof(int), st);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(work cursor)");
            if ((rc = soft_grid(L, 1, opt, &grid, &block, (int64_t)b.n_items + b.n_rec))) return rc;
            {
                Prof pr("softdtw_bwd", st);
                e = launch_softdtw_bwd(L.D, b, grid, block, st);
            }
            if (e != cudaSuccess) return cuda_fail(e, "soft-DTW backward launch");
        }
    }
    {
        Prof pr("softdtw_grad", st);
        e = launch_softdtw_grad_reduce(p.gpart, grad_value, Y->offsets, L.T, M, L.d, grad_B, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gradient reduction launch");
    return ok();
}

int wts_adam_step(float* x, const float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                  float eps, int32_t t, void* stream)
{
    if (!x || !grad || !m || !v) return fail(WTS_EINVAL, "NULL argument");
    if (n < 1 || t < 1) return fail(WTS_EINVAL, "n and t must be >= 1");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
        return fail(WTS_EINVAL, "need 0 <= beta < 1 and eps > 0");
    cudaError_t e = launch_adam(x, grad, m, v, n, lr, beta1, beta2, eps, t, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "adam launch");
    return ok();
}

int wts_softdtw_barycenter_adam(float* B, int64_t M, const wts_batch* Y, float gamma, const float* weights,
                                int32_t steps, float lr, float beta1, float beta2, float eps, const wts_options* opt,
                                void* workspace, size_t workspace_bytes, void* stream, float* values)
{
    Layout L;
    int rc = compute_layout(kOpSoft, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if ((rc = check_gamma(gamma))) return rc;
    if (!B) return fail(WTS_EINVAL, "B must not be NULL");
    if (steps < 0) return fail(WTS_EINVAL, "steps must be >= 0");
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
        return fail(WTS_EINVAL, "need 0 <= beta < 1 and eps > 0");
    const size_t need = L.total + adam_extra_bytes(M, Y);
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return fail(WTS_EINVAL, "workspace must be 256-byte aligned");
    if (workspace_bytes < need) return fail(WTS_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    char* extra = ws + L.total;
    const size_t vec = align256((size_t)M * Y->d * sizeof(float));
    float* m = reinterpret_cast<float*>(extra);
    float* v = reinterpret_cast<float*>(extra + vec);
    float* grad = reinterpret_cast<float*>(extra + 2 * vec);
    float* vscratch = reinterpret_cast<float*>(extra + 3 * vec);
    // the moments start at zero (step t = 1 of Adam)
    cudaError_t e = cudaMemsetAsync(m, 0, 2 * vec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(moments)");
    const int64_t n = M * Y->d;
    for (int32_t t = 1; t <= steps; ++t) {
        float* vals = values ? values + (int64_t)(t - 1) * Y->T : vscratch;
        if ((rc = softdtw_forward(B, M, Y, gamma, opt, ws, L.total, stream, vals))) return rc;
        if ((rc = softdtw_backward(B, M, Y, gamma, weights, opt, ws, L.total, stream, grad))) return rc;
        if ((rc = wts_adam_step(B, grad, m, v, n, lr, beta1, beta2, eps, t, stream))) return rc;
    }
    return ok();
}

int wts_autotune(int op, const float* B, int64_t M, const wts_batch* Y, void* workspace, size_t workspace_bytes,
                 void* stream, wts_options* best, float* best_ms)
{
    if (!best) return fail(WTS_EINVAL, "best is NULL");
    int kop, mode;
    switch (op) {
        case WTS_OP_ANOMALY_SCORE: kop = kOpScore; mode = kModePlen; break;
        case WTS_OP_DTW_ALIGN: kop = kOpAlign; mode = kModeDirs; break;
        case WTS_OP_DBA_ITERATE: kop = kOpDba; mode = kModeDirs; break;
        default: return fail(WTS_EINVAL, "autotune supports the score, align and DBA operations");
    }
    int rc = check_batch(Y, true);
    if (rc) return rc;
    if (!B) return fail(WTS_EINVAL, "B is NULL");
    int64_t sumN = Y->offsets_host[Y->T];
    // for the score: does the workspace hold the codes (the result depends on it)
    int codes_fit = 0;
    if (kop == kOpScore) {
        wts_options o{};
        o.score_via_codes = 1;
        Layout Lc;
        codes_fit = compute_layout(kop, M, Y, &o, &Lc) == WTS_OK && check_ws(Lc, workspace, workspace_bytes) == WTS_OK;
    }
    static std::mutex mu;
    static std::map<std::tuple<int, int, int64_t, int, int64_t, int>, std::pair<wts_options, float>> cache;
    const auto key = std::make_tuple(kop, Y->d, M, (int)Y->T, sumN, codes_fit);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *best = it->second.first;
            if (best_ms) *best_ms = it->second.second;
            return ok();
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int D = pick_D(Y->d);
    std::vector<wts_options> cands;
    // the default shape first: another candidate must beat it by more than 1 %
    for (int R : {D <= 2 ? 32 : 16, D <= 2 ? 16 : 32, 8}) {
        if (R == 32 && D > 3) continue;
        for (int wpb : {4, 2, 1}) {
            wts_options o{};
            o.rows_per_thread = R;
            o.warps_per_block = wpb;
            cands.push_back(o);
        }
    }
    // the score through stored codes and the walk (when the workspace holds
    // the codes): the two row counts of the code-writing DP, 4 warps per block
    if (kop == kOpScore)
        for (int R : {D <= 2 ? 32 : 16, D <= 2 ? 16 : 32}) {
            if (R == 32 && D > 3) continue;
            wts_options o{};
            o.rows_per_thread = R;
            o.warps_per_block = 4;
            o.score_via_codes = 1;
            cands.push_back(o);
        }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return fail(WTS_ECUDA, "cudaEventCreate");
    float best_t = 1e30f;
    wts_options best_o{};
    int tried = 0;
    // one run of a candidate: the DP (after its preparation), or for the score
    // through codes the whole call (DP, walk, division; in place in the workspace)
    auto run_once = [&](const wts_options& o, const Layout& L) -> int {
        char* ws = (char*)workspace;
        if (kop == kOpScore && o.score_via_codes) {
            float* c = reinterpret_cast<float*>(ws + L.off_costs);
            int32_t* pl = reinterpret_cast<int32_t*>(ws + L.off_plen);
            int r = align_into(L, ws, B, Y, &o, st, c, pl, reinterpret_cast<int32_t*>(ws + L.off_jlo),
                               reinterpret_cast<int32_t*>(ws + L.off_jhi));
            if (r) return r;
            const cudaError_t e = launch_score_divide(c, pl, c, L.T, st);
            return e == cudaSuccess ? WTS_OK : cuda_fail(e, "score division launch");
        }
        int r = prepare(L, ws, B, Y, &o, st);
        if (r) return r;
        DPParams p = base_params(L, ws, &o);
        return launch_dp(mode, L, p, &o, st);
    };
    for (const wts_options& o : cands) {
        Layout L;
        if (compute_layout(kop, M, Y, &o, &L) != WTS_OK) continue;
        if (check_ws(L, workspace, workspace_bytes) != WTS_OK) continue;
        float t_min = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {             // first run warms up, best of two
            cudaEventRecord(a, st);
            if ((rc = run_once(o, L))) break;
            cudaEventRecord(b, st);
            if (cudaEventSynchronize(b) != cudaSuccess) { rc = fail(WTS_ECUDA, "autotune run failed"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep > 0 && ms < t_min) t_min = ms;
        }
        if (rc) break;
        ++tried;
        if (tried == 1 || t_min < 0.99f * best_t) { best_t = t_min; best_o = o; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc) return rc;
    if (!tried) return fail(WTS_ENOMEM, "no candidate fits the workspace");
    {
        std::lock_guard<std::mutex> g(mu);
        cache[key] = {best_o, best_t};
    }
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    return ok();
}

int wts_pad_last(const wts_batch* Y, int64_t L, void* stream, float* out)
{
    int rc = check_batch(Y, true);
    if (rc) return rc;
    if (!out) return fail(WTS_EINVAL, "out is NULL");
    int64_t longest = 0;
    for (int k = 0; k < Y->T; ++k) {
        const int64_t n = Y->offsets_host[k + 1] - Y->offsets_host[k];
        if (n > longest) longest = n;
    }
    if (L == 0) L = longest;
    if (L < longest) return fail(WTS_EINVAL, "L=%lld is shorter than the longest cycle (%lld)", (long long)L,
                                 (long long)longest);
    if (L > ((int64_t)1 << 40) / ((int64_t)Y->T * Y->d)) return fail(WTS_EINVAL, "L=%lld too large", (long long)L);
    cudaError_t e;
    {
        Prof pr("pad_last", (cudaStream_t)stream);
        e = launch_pad_last(Y->data, Y->offsets, Y->T, Y->d, L, out, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pad_last launch");
    return ok();
}

int wts_select_channel(const wts_batch* Y, int32_t c, void* stream, float* out)
{
    int rc = check_batch(Y, true);
    if (rc) return rc;
    if (!out) return fail(WTS_EINVAL, "out is NULL");
    if (c < 0 || c >= Y->d) return fail(WTS_EINVAL, "channel %d outside 0..%d", c, Y->d - 1);
    cudaError_t e;
    {
        Prof pr("select_channel", (cudaStream_t)stream);
        e = launch_select_channel(Y->data, Y->offsets_host[Y->T], Y->d, c, out, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "select_channel launch");
    return ok();
}

int wts_compact_nan(const wts_batch* Y, void* workspace, size_t workspace_bytes, void* stream, float* out,
                    int64_t* out_offsets)
{
    int rc = check_batch(Y, true);
    if (rc) return rc;
    if (!out || !out_offsets) return fail(WTS_EINVAL, "out and out_offsets must not be NULL");
    const int64_t rows = Y->offsets_host[Y->T];
    if (!workspace) return fail(WTS_EINVAL, "workspace is NULL");
    if (workspace_bytes < compact_workspace_bytes(rows))
        return fail(WTS_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, compact_workspace_bytes(rows));
    cudaError_t e;
    {
        Prof pr("compact_nan", (cudaStream_t)stream);
        e = launch_compact_nan(Y->data, Y->offsets, Y->T, Y->d, rows, out, out_offsets, workspace,
                               (cudaStream_t)stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "compaction launch");
    return ok();
}

int wts_medoid(const float* C, int32_t n, void* stream, double* sums, int32_t* index)
{
    if (!C || !sums || !index) return fail(WTS_EINVAL, "NULL argument");
    if (n < 1) return fail(WTS_EINVAL, "n must be >= 1");
    cudaError_t e = launch_medoid(C, n, index, sums, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "medoid launch");
    return ok();
}

int wts_resample(const float* x, int64_t N, int32_t d, float* out, int64_t M, void* stream)
{
    if (!x || !out) return fail(WTS_EINVAL, "NULL argument");
    if (N < 1 || M < 1 || d < 1 || d > kMaxD) return fail(WTS_EINVAL, "bad shape");
    cudaError_t e = launch_resample(x, N, d, out, M, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "resample launch");
    return ok();
}

int wts_euclid_mean(const wts_batch* Y, int64_t M, float* out, void* stream)
{
    int rc = check_batch(Y, true);
    if (rc) return rc;
    if (!out || M < 1) return fail(WTS_EINVAL, "bad output");
    cudaError_t e = launch_euclid_mean(Y->data, Y->offsets, Y->T, Y->d, M, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "mean launch");
    return ok();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// anomaly_score_noalloc: the same score with a fixed, library-owned scratch
// area instead of a caller workspace, for callers that cannot allocate device
// memory (see include/wetsand.h).  The scratch is a file-scope __device__
// array, so it exists on every GPU that loads this library, until exit.
// ---------------------------------------------------------------------------
namespace wts {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char wts_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// with that device current: on the first call on each device, and again on
// every call made outside stream capture (a cheap host call), so that a
// context torn down and re-created in between (cudaDeviceReset) is followed.
// During capture the address cached by an earlier call is used; a capture with
// no earlier call on that device is refused.
int noalloc_scratch(cudaStream_t st, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(WTS_EINVAL, "device ordinal %d not supported", dev);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, wts_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_noalloc_addr[dev] = p;
    } else if (!g_noalloc_addr[dev]) {
        return fail(WTS_EINVAL, "the first no-allocation call on device %d must come before any stream capture", dev);
    }
    *out = g_noalloc_addr[dev];
    return WTS_OK;
}

}  // namespace
}  // namespace wts

extern "C" int anomaly_score_noalloc(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
                                     void* stream, float* score, float* cost, int32_t* plen)
{
    using namespace wts;
    // the fixed scratch serves the count inside the DP only
    wts_options o = opt ? *opt : wts_options{};
    o.score_via_codes = 0;
    opt = &o;
    Layout L;
    int rc = compute_layout(kOpScore, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if (!B || !score) return fail(WTS_EINVAL, "B and score must not be NULL");
    if (L.total > kNoAllocScratchBytes)
        return fail(WTS_ENOMEM,
                    "anomaly_score_noalloc: this batch needs %zu bytes of scratch but the fixed scratch holds %zu; "
                    "score fewer or shorter cycles per call, or use anomaly_score with a workspace",
                    L.total, kNoAllocScratchBytes);
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    if ((rc = noalloc_scratch(st, &scratch))) return rc;
    char* ws = (char*)scratch;
    // prepare() zeroes the header and progress counters left by the previous call
    if ((rc = prepare(L, ws, B, Y, opt, st))) return rc;
    DPParams p = base_params(L, ws, opt);
    p.cost_out = cost;
    p.plen_out = plen;
    p.score_out = score;
    if ((rc = launch_dp(kModePlen, L, p, opt, st))) return rc;
    return ok();
}

// The status word of the fixed scratch (the header at its start), read like
// wts_read_status reads a workspace's: after the stream has reached every call
// queued on it.
extern "C" int wts_noalloc_read_status(void* stream, int32_t* status)
{
    using namespace wts;
    if (!status) return fail(WTS_EINVAL, "status is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    int rc = noalloc_scratch(st, &scratch);
    if (rc) return rc;
    return wts_read_status(scratch, stream, status);
}

// Detection thresholds and F2 (Sec. 5.3): host arithmetic on the T scores.
int wts_thresholds(const float* scores, int32_t T, double* two_sigma, double* boxplot)
{
    if (!scores || (!two_sigma && !boxplot)) return fail(WTS_EINVAL, "NULL argument");
    if (T < 1) return fail(WTS_EINVAL, "T must be >= 1");
    std::vector<double> v(scores, scores + T);
    for (double x : v)
        if (!std::isfinite(x)) return fail(WTS_EINVAL, "scores must be finite");
    if (two_sigma) {
        double mean = 0.0;
        for (double x : v) mean += x;
        mean /= T;
        double var = 0.0;
        for (double x : v) var += (x - mean) * (x - mean);
        *two_sigma = mean + 2.0 * std::sqrt(var / T);
    }
    if (boxplot) {
        // quartile q at position q (T - 1) of the sorted scores, linear between neighbours
        std::sort(v.begin(), v.end());
        auto quartile = [&](double q) {
            const double pos = q * (T - 1);
            const int64_t lo = (int64_t)std::floor(pos);
            const int64_t hi = lo + 1 < T ? lo + 1 : lo;
            return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
        };
        const double q1 = quartile(0.25), q3 = quartile(0.75);
        *boxplot = q3 + 1.5 * std::fabs(q3 - q1);
    }
    return ok();
}

int wts_f2(const float* scores, const int8_t* labels, int32_t T, double threshold,
           int32_t* tp, int32_t* fp, int32_t* fn, double* f2)
{
    if (!scores || !labels || !f2) return fail(WTS_EINVAL, "NULL argument");
    if (T < 0) return fail(WTS_EINVAL, "T must be >= 0");
    int32_t a = 0, b = 0, c = 0;
    for (int32_t k = 0; k < T; ++k) {
        const bool flag = (double)scores[k] > threshold;
        const bool truth = labels[k] != 0;
        a += flag && truth;
        b += flag && !truth;
        c += !flag && truth;
    }
    if (tp) *tp = a;
    if (fp) *fp = b;
    if (fn) *fn = c;
    // F_beta with beta = 2: (1 + 4) TP / ((1 + 4) TP + 4 FN + FP); 0 when there is nothing to find or flag
    const double den = 5.0 * a + 4.0 * c + b;
    *f2 = den > 0 ? 5.0 * a / den : 0.0;
    return ok();
}

// L-BFGS (see include/wetsand.h for the method and its stopping rules).
int wts_lbfgs_minimize(int64_t n, double* x, wts_objective_fn fn, void* ctx, const wts_lbfgs_params* prm,
                       double* f_out, int32_t* n_iter, int32_t* n_eval, int32_t* reason)
{
    if (!x || !fn) return fail(WTS_EINVAL, "x and fn must not be NULL");
    if (n < 1) return fail(WTS_EINVAL, "n must be >= 1");
    wts_lbfgs_params P{10, 40, 200, 0, 1e-8, 1e-5, 1e-4};
    if (prm) P = *prm;
    if (P.history < 1 || P.max_iter < 0 || P.max_fun < 1 || !(P.gtol >= 0) || !(P.ftol >= 0) || !(P.c1 > 0 && P.c1 < 1))
        return fail(WTS_EINVAL, "bad L-BFGS parameters");
    auto dot = [n](const double* a, const double* b) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
        return s;
    };
    std::vector<double> g(n), d(n), xn(n), gn(n), q(n);
    std::vector<std::vector<double>> S, Yv;
    std::vector<double> rho;
    double f = 0.0;
    int evals = 0, it = 0, why = 0;
    if (fn(x, &f, g.data(), ctx)) return fail(WTS_ECUDA, "objective evaluation failed");
    ++evals;
    for (;;) {
        double gmax = 0.0;
        for (int64_t i = 0; i < n; ++i) gmax = std::max(gmax, std::fabs(g[i]));
        if (gmax <= P.gtol) { why = 1; break; }
        if (it >= P.max_iter) { why = 3; break; }
        // two-loop recursion: d = -H g
        const int h = (int)S.size();
        std::vector<double> a(h);
        for (int64_t i = 0; i < n; ++i) q[i] = g[i];
        for (int k = h - 1; k >= 0; --k) {
            a[k] = rho[k] * dot(S[k].data(), q.data());
            for (int64_t i = 0; i < n; ++i) q[i] -= a[k] * Yv[k][i];
        }
        const double scale = h ? dot(S[h - 1].data(), Yv[h - 1].data()) / dot(Yv[h - 1].data(), Yv[h - 1].data()) : 1.0;
        for (int64_t i = 0; i < n; ++i) q[i] *= scale;
        for (int k = 0; k < h; ++k) {
            const double bk = rho[k] * dot(Yv[k].data(), q.data());
            for (int64_t i = 0; i < n; ++i) q[i] += S[k][i] * (a[k] - bk);
        }
        for (int64_t i = 0; i < n; ++i) d[i] = -q[i];
        double gd = dot(g.data(), d.data());
        double t = 1.0;
        if (h == 0 || !(gd < 0)) {
            // no curvature pairs (or not a descent direction): steepest descent
            S.clear(); Yv.clear(); rho.clear();
            for (int64_t i = 0; i < n; ++i) d[i] = -g[i];
            gd = -dot(g.data(), g.data());
            t = std::min(1.0, 1.0 / std::sqrt(-gd));
        }
        // backtracking (Armijo)
        double fn_new = 0.0;
        bool accepted = false;
        while (evals < P.max_fun) {
            for (int64_t i = 0; i < n; ++i) xn[i] = x[i] + t * d[i];
            if (fn(xn.data(), &fn_new, gn.data(), ctx)) return fail(WTS_ECUDA, "objective evaluation failed");
            ++evals;
            if (fn_new <= f + P.c1 * t * gd) { accepted = true; break; }
            t *= 0.5;
        }
        if (!accepted) { why = 4; break; }
        std::vector<double> s(n), y(n);
        for (int64_t i = 0; i < n; ++i) { s[i] = xn[i] - x[i]; y[i] = gn[i] - g[i]; }
        const double sy = dot(s.data(), y.data());
        if (sy > 1e-10 * std::sqrt(dot(s.data(), s.data()) * dot(y.data(), y.data()))) {
            if ((int)S.size() == P.history) { S.erase(S.begin()); Yv.erase(Yv.begin()); rho.erase(rho.begin()); }
            S.push_back(std::move(s));
            Yv.push_back(std::move(y));
            rho.push_back(1.0 / sy);
        }
        ++it;
        const double rel = (f - fn_new) / std::max(std::max(std::fabs(f), std::fabs(fn_new)), 1.0);
        for (int64_t i = 0; i < n; ++i) { x[i] = xn[i]; g[i] = gn[i]; }
        f = fn_new;
        if (rel <= P.ftol) { why = 2; break; }
    }
    if (f_out) *f_out = f;
    if (n_iter) *n_iter = it;
    if (n_eval) *n_eval = evals;
    if (reason) *reason = why;
    return ok();
}

namespace {

struct SoftObjective {
    float* B;
    int64_t M;
    const wts_batch* Y;
    float gamma;
    const wts_options* opt;
    char* ws;
    size_t soft_bytes;
    cudaStream_t st;
    float* d_values;
    const float* d_weights;
    float* d_grad;
    std::vector<double> w;        // host weights
    std::vector<float> xf, vals, gf;
    int err = WTS_OK;
};

int soft_objective(const double* x, double* f, double* g, void* ctx)
{
    SoftObjective& o = *static_cast<SoftObjective*>(ctx);
    const int64_t n = o.M * o.Y->d;
    for (int64_t i = 0; i < n; ++i) o.xf[i] = (float)x[i];
    cudaError_t e = cudaMemcpyAsync(o.B, o.xf.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice, o.st);
    if (e != cudaSuccess) { o.err = cuda_fail(e, "barycenter copy"); return 1; }
    int rc = softdtw_forward(o.B, o.M, o.Y, o.gamma, o.opt, o.ws, o.soft_bytes, o.st, o.d_values);
    if (rc == WTS_OK)
        rc = softdtw_backward(o.B, o.M, o.Y, o.gamma, o.d_weights, o.opt, o.ws, o.soft_bytes, o.st, o.d_grad);
    if (rc != WTS_OK) { o.err = rc; return 1; }
    e = cudaMemcpyAsync(o.vals.data(), o.d_values, (size_t)o.Y->T * sizeof(float), cudaMemcpyDeviceToHost, o.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(o.gf.data(), o.d_grad, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, o.st);
    WsHeader h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, o.ws, sizeof(h), cudaMemcpyDeviceToHost, o.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(o.st);
    if (e != cudaSuccess) { o.err = cuda_fail(e, "objective read-back"); return 1; }
    if (status_of(h) != WTS_OK) {
        o.err = fail(status_of(h), status_of(h) == WTS_EINVAL ? "a sample of B or of the batch is not finite"
                                                              : "a wait inside the soft-DTW kernels gave up");
        return 1;
    }
    double s = 0.0;
    for (int k = 0; k < o.Y->T; ++k) s += o.w[k] * (double)o.vals[k];
    *f = s;
    for (int64_t i = 0; i < n; ++i) g[i] = (double)o.gf[i];
    return 0;
}

}  // namespace

int wts_softdtw_barycenter_lbfgs(float* B, int64_t M, const wts_batch* Y, float gamma, const float* weights,
                                 const wts_lbfgs_params* prm, const wts_options* opt, void* workspace,
                                 size_t workspace_bytes, void* stream, double* f_out, int32_t* n_iter,
                                 int32_t* n_eval, int32_t* reason)
{
    Layout L;
    int rc = compute_layout(kOpSoft, M, Y, opt, &L);
    if (rc) return rc;
    if ((rc = check_batch(Y, true))) return rc;
    if ((rc = check_gamma(gamma))) return rc;
    if (!B) return fail(WTS_EINVAL, "B must not be NULL");
    const size_t need = L.total + lbfgs_extra_bytes(M, Y);
    if (!workspace || ((uintptr_t)workspace & 255) != 0) return fail(WTS_EINVAL, "workspace must be 256-byte aligned");
    if (workspace_bytes < need) return fail(WTS_ENOMEM, "workspace has %zu bytes, needs %zu", workspace_bytes, need);
    SoftObjective o;
    o.B = B;
    o.M = M;
    o.Y = Y;
    o.gamma = gamma;
    o.opt = opt;
    o.ws = (char*)workspace;
    o.soft_bytes = L.total;
    o.st = (cudaStream_t)stream;
    char* extra = o.ws + L.total;
    o.d_values = reinterpret_cast<float*>(extra);
    float* d_w = reinterpret_cast<float*>(extra + align256((size_t)Y->T * sizeof(float)));
    o.d_grad = reinterpret_cast<float*>(extra + 2 * align256((size_t)Y->T * sizeof(float)));
    const int64_t n = M * Y->d;
    o.xf.resize(n);
    o.gf.resize(n);
    o.vals.resize(Y->T);
    o.w.resize(Y->T);
    std::vector<float> wf(Y->T);
    if (weights) {
        cudaError_t e = cudaMemcpyAsync(wf.data(), weights, (size_t)Y->T * sizeof(float), cudaMemcpyDeviceToHost, o.st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(o.st);
        if (e != cudaSuccess) return cuda_fail(e, "weights read");
    } else {
        for (int k = 0; k < Y->T; ++k) wf[k] = (float)(1.0 / (double)(Y->offsets_host[k + 1] - Y->offsets_host[k]));
    }
    for (int k = 0; k < Y->T; ++k) o.w[k] = (double)wf[k];
    cudaError_t e = cudaMemcpyAsync(d_w, wf.data(), (size_t)Y->T * sizeof(float), cudaMemcpyHostToDevice, o.st);
    if (e != cudaSuccess) return cuda_fail(e, "weights copy");
    o.d_weights = d_w;
    // start from B
    std::vector<double> x(n);
    e = cudaMemcpyAsync(o.xf.data(), B, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, o.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(o.st);
    if (e != cudaSuccess) return cuda_fail(e, "barycenter read");
    for (int64_t i = 0; i < n; ++i) x[i] = (double)o.xf[i];
    rc = wts_lbfgs_minimize(n, x.data(), soft_objective, &o, prm, f_out, n_iter, n_eval, reason);
    if (rc != WTS_OK) return o.err != WTS_OK ? o.err : rc;
    // leave the last accepted iterate in B
    for (int64_t i = 0; i < n; ++i) o.xf[i] = (float)x[i];
    e = cudaMemcpyAsync(B, o.xf.data(), (size_t)n * sizeof(float), cudaMemcpyHostToDevice, o.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(o.st);
    if (e != cudaSuccess) return cuda_fail(e, "barycenter write");
    return ok();
}
