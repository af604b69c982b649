/*
 * wetsand.h - C ABI of the GB300 (sm_103a) alignment hot path of WETSAND
 * ("Warped Time Series Anomaly Detection", arXiv 2404.12134).
 *
 * The hot path is the alignment of many long, uneven cycles against one
 * prototype by Dynamic Time Warping: it feeds DTW Barycenter Averaging (the
 * prototype) and the per-cycle anomaly score, plus Soft-DTW with its gradient
 * for gradient-based barycenters.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Rows index the prototype / barycenter B (length M), columns index a cycle
 *    Y_k (length N_k): DTW(B, C_k) as in Eq. 8, Soft-DTW(B, Y_i) as in Eq. 7.
 *  - Samples are d-channel FP32 vectors, row-major: B is [M][d]; a batch packs
 *    T cycles back to back, cycle k = data[offsets[k]*d .. offsets[k+1]*d).
 *    Time steps with missing values must already be removed (Sec. 3.1): every
 *    sample must be finite.  Every call that runs a DP first scans B and the
 *    batch on the device; a NaN or +-inf sample makes each kernel of the call
 *    leave before doing any work (outputs are then unspecified) and leaves
 *    WTS_EINVAL in the workspace's device status word (wts_read_status).
 *  - Local cost delta(b_i, y_j) = sum_c (b_ic - y_jc)^2 (the Euclidean norm of
 *    Sec. 3.2, squared), or the norm itself with wts_options.cost_kind = 1.
 *  - Equal predecessors resolve diag (i-1,j-1) first, then up (i-1,j), then
 *    left (i,j-1): the path returned is, among all optimal complete alignment
 *    paths, the one whose steps read backwards from (M-1,N-1) are
 *    lexicographically greatest under diag > up > left.
 *  - Every array argument is a DEVICE pointer owned by the caller unless
 *    marked host.  The library never allocates device memory: scratch space is
 *    one caller-owned workspace buffer whose size wts_workspace_size() gives.
 *    A workspace must not be shared by calls in flight at the same time.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Outputs are valid once the stream has reached the call.
 *    Inputs are validated on the host before any launch.
 *  - Return value: WTS_OK or an error code; wts_last_error() gives the text
 *    (thread-local).  What a call can only find on the device is reported in
 *    the workspace's device status word, read by wts_read_status(): a
 *    non-finite sample (WTS_EINVAL), or a wait inside a kernel that gave up
 *    (WTS_ETIMEOUT; it never does in normal operation).
 */
#ifndef WETSAND_H
#define WETSAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    WTS_OK = 0,
    WTS_EINVAL = 1,      /* bad argument: null pointer, shape, length, d, gamma */
    WTS_ENOMEM = 2,      /* workspace smaller than wts_workspace_size() */
    WTS_ECUDA = 3,       /* CUDA runtime error (launch or configuration) */
    WTS_ETIMEOUT = 4,    /* a bounded in-kernel wait gave up (device status) */
};

/* Operation codes for wts_workspace_size(). */
enum {
    WTS_OP_ANOMALY_SCORE = 1,
    WTS_OP_DTW_ALIGN = 2,
    WTS_OP_DBA_ITERATE = 3,
    WTS_OP_SOFTDTW = 4,        /* softdtw_forward + softdtw_backward (R kept in the workspace) */
    WTS_OP_PAIRWISE = 5,
    WTS_OP_COMPACT_NAN = 6,    /* wts_compact_nan (M ignored) */
    WTS_OP_SUBDTW = 7,         /* subdtw_align (M = length of X) */
    WTS_OP_SOFTDTW_LBFGS = 8,  /* wts_softdtw_barycenter_lbfgs */
    WTS_OP_SOFTDTW_ADAM = 9,   /* wts_softdtw_barycenter_adam */
};

/* A packed batch of T cycles (Sec. 3.1: d-channel series of uneven lengths). */
typedef struct wts_batch {
    const float* data;             /* device, [sum_k N_k][d] */
    const int64_t* offsets;        /* device, [T+1]: offsets[0] = 0, N_k = offsets[k+1]-offsets[k] >= 1 */
    const int64_t* offsets_host;   /* host copy of offsets (plans the work, validates lengths) */
    int32_t T;                     /* >= 1 */
    int32_t d;                     /* 1..16 */
} wts_batch;

/* Launch options; a zeroed struct (or NULL) selects the defaults. */
typedef struct wts_options {
    int32_t rows_per_thread;       /* prototype rows held per lane: 0 = default (32 if d <= 2, else 16); 8, 16 or 32 (32 needs d <= 3);
                                      4 for Sub-DTW only.  Soft-DTW does not use it: 8 rows per lane, 4 under a
                                      band narrower than 0.45 */
    int32_t warps_per_block;       /* 0 = 4; 1..4 */
    int32_t max_blocks;            /* 0 = as many as are resident at once (persistent grid); else a cap */
    int32_t keep_batch_order;      /* 0 = schedule the longest pairs first; 1 = batch order */
    int32_t dir_mode;              /* dtw_align / dba_iterate: 0 = store every cell's 2-bit code (M*N/4 bytes
                                      per cycle); 1 = checkpoint + recompute: store only the band hand-off rows,
                                      recompute the codes of ckpt_bands bands at a time during the backtrack
                                      (one extra forward pass, bit-identical paths) */
    int32_t ckpt_bands;            /* bands (of 32*rows_per_thread prototype rows) recomputed per group; 0 = 16.
                                      DTW keeps one group's codes; soft-DTW with a band keeps two groups' R (the
                                      backward of one group runs beside the recompute of the next); soft-DTW
                                      without a band uses column checkpoints instead and ignores it */
    int32_t spin_limit;            /* polls before an in-kernel wait gives up (each ~0.1-1 us); 0 = 2^27 */
    int32_t fault_skip_handoff;    /* fault injection for tests: 1 = producers skip their hand-off rows, so
                                      consumers wait until spin_limit and the call ends with WTS_ETIMEOUT in
                                      the workspace status; never set it otherwise */
    double band;                   /* Sakoe-Chiba band (Table I: a width as a fraction of the signals' length):
                                      0-based cell (i, j) of an M x N pair is kept when
                                      |i N - j M| <= floor(band M N) (|i/M - j/N| <= band); cells outside are
                                      +inf.  0 = no band.  A band narrower than max(M, N) for some pair (it may
                                      hold no complete path) is WTS_EINVAL.  DTW and soft-DTW operations
                                      (anomaly_score, dtw_align, dba_iterate, softdtw_forward / _backward and
                                      the barycenters); for soft-DTW, cells outside the band take no part in the
                                      soft minimum (forward) and carry no weight (backward). */
    int32_t cost_kind;             /* local cost delta(b_i, y_j) (Definition "Distance Matrix", Sec. 3.2):
                                      WTS_COST_SQEUCLID (0, default) = sum_c (b_ic - y_jc)^2;
                                      WTS_COST_L2 (1) = its IEEE square root, the l2 norm.  Every DTW,
                                      Sub-DTW and soft-DTW operation; the DTW kernels then hold 16 rows per
                                      lane (rows_per_thread 0 or 16, else WTS_EINVAL).  The soft-DTW
                                      gradient of the norm is (b_ic - y_jc) / delta, taken as 0 where
                                      delta = 0.  dba_iterate still averages the aligned samples (the mean
                                      minimises the squared cost only, so the DBA cost need not decrease). */
    int32_t score_via_codes;       /* anomaly_score: 0 = count |pi| inside the DP (small workspace); 1 = store
                                      every cell's 2-bit code, walk the paths (dtw_align's segmented walk) and
                                      take |pi| from the row ranges - the same scores, with the dtw_align
                                      workspace; faster where the code-writing DP outruns the counting one
                                      (wts_autotune tries both when the workspace allows).
                                      anomaly_score_noalloc always counts inside the DP. */
    int32_t store_pairs;           /* soft-DTW with dir_mode = 1 and no band (column checkpoints): the first
                                      store_pairs pairs of the work list (longest first, or the batch order
                                      with keep_batch_order) keep every R value in the
                                      workspace, as dir_mode = 0 does, and only the others keep column
                                      checkpoints, so the backward recomputes R for those pairs only.  0 = none;
                                      values >= T store every pair.  Values, gradients and the workspace's
                                      other parts are the same bit for bit; the workspace grows by
                                      (R - checkpoint) bytes of the stored pairs (wts_workspace_size).  For
                                      batches whose whole R (4 bytes per cell) exceeds the device's memory:
                                      the checkpoints take about 0.3 bytes per cell, and the memory left
                                      can hold R of some pairs instead of recomputing it.  Non-zero with
                                      any other operation or mode is WTS_EINVAL. */
    int32_t reserved[3];
} wts_options;

/* Values of wts_options.cost_kind. */
enum { WTS_COST_SQEUCLID = 0, WTS_COST_L2 = 1 };

/* Library version (major * 100 + minor). */
int wts_version(void);

/* Text of the last error returned on this thread ("" if none). */
const char* wts_last_error(void);

/* Bytes of workspace that operation `op` needs for prototype length M and
 * batch Y (M is ignored for WTS_OP_PAIRWISE).  Host-only; no CUDA call. */
int wts_workspace_size(int op, int64_t M, const wts_batch* Y, const wts_options* opt, size_t* bytes);

/* Synchronise `stream` and read the device status word of `workspace` into
 * *status (host): WTS_OK, WTS_EINVAL (a sample of B or of the batch is NaN or
 * +-inf; the call's kernels did no work) or WTS_ETIMEOUT (an in-kernel wait
 * gave up).  The word is reset by the next call on the workspace. */
int wts_read_status(const void* workspace, void* stream, int32_t* status);

/* Kernel timing for measurement: while enabled, every kernel the library
 * launches is bracketed by a pair of CUDA events recorded on the launching
 * stream (library-owned events, created per launch).  Host-only switch. */
int wts_profile_enable(int enable);

/* Sum of the recorded durations (ms) and kernel launches of one stage
 * ("setup", "wavefront", "backtrack", "dba_average", "softdtw_fwd",
 * "softdtw_bwd", "softdtw_grad"; "" = all), then forget those records.  A
 * stage may launch several kernels (the segmented backtrack: one per round
 * and a last one); `launches` counts them all.  Waits for the recorded events
 * to complete. */
int wts_profile_read(const char* kernel, double* total_ms, int32_t* launches);

/* Measured roofline denominators (not part of the method): lane operations
 * per second of the whole GPU for which = 0 FP32 fused multiply-add, 1 FP32
 * min / max, 2 MUFU ex2.approx, 3 MUFU lg2.approx, 4 packed f32x2 fused
 * multiply-add (two lane-ops each), 5 three-input FP32 min; best of
 * four timed launches.  Synchronises the device. */
int wts_peak_probe(int which, double* ops_per_s);

/*
 * anomaly_score - similarity score of Eq. 8 (Sec. 3.4):
 *     d_score(B, C_k) = DTW(B, C_k) / |pi_k|,
 * DTW by Eq. 1 (the recursion Eq. 5 at gamma = 0), |pi_k| = number of index
 * pairs on the tie-rule optimal path (Definition "Alignment path"), counted on
 * the fly without storing the path.  The division is one FP32 division.
 *   B     [M][d]   prototype
 *   score [T]      out: d_score per cycle
 *   cost  [T]      out (may be NULL): DTW(B, C_k)
 *   plen  [T]      out (may be NULL): |pi_k|
 * Workspace: wts_workspace_size(WTS_OP_ANOMALY_SCORE, ...).
 */
int anomaly_score(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
                  void* workspace, size_t workspace_bytes, void* stream,
                  float* score, float* cost, int32_t* plen);

/*
 * dtw_align - DTW (Eq. 1) and its optimal complete alignment path
 * (Definitions "Alignment path" / "Alignment matrix", Sec. 3.2) for every
 * cycle.  The path of cycle k is returned as per-row column ranges: row i of
 * B is aligned to columns jlo[k][i] .. jhi[k][i] of Y_k (a monotone path
 * visits each row on one contiguous run of columns), and |pi_k| = sum_i
 * (jhi - jlo + 1).
 *   cost [T], plen [T]           out (either may be NULL)
 *   jlo  [T][M], jhi [T][M]      out (int32); with every code stored
 *                                (dir_mode 0) the walk reads the jhi values
 *                                found there on entry as guesses of where
 *                                the path enters rows 2048 apart (a repeated
 *                                call on the same arrays walks faster); any
 *                                contents are safe and the result does not
 *                                depend on them
 * A 2-bit predecessor code per cell is kept in the workspace (M*N_k/4 bytes
 * per cycle, plus a skew margin); wts_workspace_size(WTS_OP_DTW_ALIGN, ...).
 */
int dtw_align(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
              void* workspace, size_t workspace_bytes, void* stream,
              float* cost, int32_t* plen, int32_t* jlo, int32_t* jhi);

/*
 * subdtw_align - Sub-DTW (Sec. 3.2): for every cycle ("window") Y_k of the
 * batch, the minimum over 0 <= a <= b < N_k of DTW(X, Y_k[a..b]), the whole
 * reference X (length M, rows) against the best contiguous piece of Y_k.  The
 * recursion of Eq. 5 (gamma = 0) runs with a free start (the row above X is
 * 0 in every column); b* is the first column of minimum cost in X's last row,
 * and the walk back from (M-1, b*) under the tie order diag > up > left stops
 * where it leaves X's first row, at a*.
 *   X    [M][d]                  in (device)
 *   cost [T]                     out, min_b r(M-1, b) (may be NULL)
 *   a_star, b_star [T]           out (int32), 0-based inclusive bounds in Y_k
 *   plen [T]                     out, |pi| (may be NULL)
 *   jlo, jhi [T][M]              out (int32), columns of each row of X
 * rows_per_thread must be 0 (16), 4, 8 or 16 (0 or 16 with cost_kind = 1);
 * dir_mode 1 (checkpointing) is not offered.
 * Workspace: wts_workspace_size(WTS_OP_SUBDTW, M, Y, ...).
 */
int subdtw_align(const float* X, int64_t M, const wts_batch* Y, const wts_options* opt,
                 void* workspace, size_t workspace_bytes, void* stream,
                 float* cost, int32_t* a_star, int32_t* b_star, int32_t* plen, int32_t* jlo, int32_t* jhi);

/*
 * wts_segment - the segmentation of Sec. 3.2: a long d-channel series Y
 * (Ydata [N][d], device) is cut into cycles matching the reference X
 * ([M][d], device).  Window [ws, we) with ws = 0, we = ws + 2M (cut at N);
 * Sub-DTW of X against the window gives [a*, b*]; the piece
 * [ws + a*, ws + b*] is recorded and the next window starts at
 * ws + b* - alpha, while ws < N; alpha < 0 selects the paper's
 * alpha = 0.15 M (rounded down).  Two
 * readings where the paper does not say: the window that reaches the end of
 * Y is the last one, and when b* - alpha would not move the window forward
 * the next one starts at ws + b* + 1.
 *   seg_start, seg_end [max_segments]   out (host, int64, inclusive)
 *   seg_cost [max_segments]             out (host, may be NULL)
 *   n_segments                          out (host): pieces found; if more
 *                                       than max_segments, the first
 *                                       max_segments are stored and
 *                                       WTS_ENOMEM is returned
 * Each window runs the Sub-DTW wavefront on `stream`; its b* is read back
 * (the stream is synchronised once per window) and its backtrack (a*) runs on
 * a second stream of the library's, beside the next window's wavefront; the
 * workspace holds two window slots.  On return `stream` is ordered after all
 * of the call's work.  A window is a single pair, so rows_per_thread = 0
 * means 4 here (four times the warps of 16, a quarter of the serial chain per
 * step; 16 with cost_kind = 1).  Workspace: wts_segment_workspace_size (with
 * the same options).
 */
int wts_segment_workspace_size(int64_t M, int32_t d, const wts_options* opt, size_t* bytes);
int wts_segment(const float* X, int64_t M, const float* Ydata, int64_t N, int32_t d, int64_t alpha,
                const wts_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                int32_t max_segments, int64_t* seg_start, int64_t* seg_end, float* seg_cost, int32_t* n_segments);

/*
 * wts_thresholds - the two detection thresholds of Sec. 5.3 on a set of
 * d_score values (host array scores[T], all finite; no CUDA call):
 *   two_sigma = mean + 2 std   (std with divisor T)
 *   boxplot   = q3 + 1.5 |q3 - q1|, quartile q taken at position q (T - 1) of
 *               the sorted scores, linearly between the two neighbouring values
 * A cycle is flagged abnormal when its score is above the threshold.  Either
 * output may be NULL (not both).
 */
int wts_thresholds(const float* scores, int32_t T, double* two_sigma, double* boxplot);

/*
 * wts_f2 - confusion counts and the F2 score (Sec. 5.3) of the flags
 * "score > threshold" against labels[T] (host, nonzero = abnormal):
 *   F2 = 5 TP / (5 TP + 4 FN + FP), 0 when TP + FN + FP = 0.
 * tp, fp, fn may be NULL.
 */
int wts_f2(const float* scores, const int8_t* labels, int32_t T, double threshold,
           int32_t* tp, int32_t* fp, int32_t* fn, double* f2);

/*
 * L-BFGS (the optimiser of the paper's barycenters, Table I: "L-BFGS",
 * max iter 40, max fun 200, G tol 1e-8, tolerance 1e-5), restated from the
 * standard method (limited-memory BFGS, two-loop recursion):
 *   direction d = -H g, H from the last `history` pairs (s, y) with s.y > 0,
 *   initial scaling (s.y)/(y.y) of the newest pair (no pair: d = -g and a
 *   first step of min(1, 1/||g||_2));
 *   step by backtracking from 1, halving until f(x + t d) <= f + c1 t g.d;
 *   stop when max|g| <= gtol (reason 1), when the relative reduction
 *   (f_k - f_k+1) / max(|f_k|, |f_k+1|, 1) <= ftol (reason 2), after
 *   max_iter iterations (3) or max_fun evaluations (4).
 * All vectors in double on the host.  fn(x, f, g, ctx) evaluates the
 * objective and its gradient and returns 0 (nonzero aborts with
 * WTS_ECUDA).  x [n] is the start on entry and the last accepted iterate on
 * return.  prm may be NULL (history 10, max_iter 40, max_fun 200, gtol 1e-8,
 * ftol 1e-5, c1 1e-4).
 */
typedef int (*wts_objective_fn)(const double* x, double* f, double* g, void* ctx);
typedef struct wts_lbfgs_params {
    int32_t history;
    int32_t max_iter;
    int32_t max_fun;
    int32_t reserved;
    double gtol;
    double ftol;
    double c1;
} wts_lbfgs_params;
int wts_lbfgs_minimize(int64_t n, double* x, wts_objective_fn fn, void* ctx, const wts_lbfgs_params* prm,
                       double* f_out, int32_t* n_iter, int32_t* n_eval, int32_t* reason);

/*
 * wts_softdtw_barycenter_lbfgs - the Soft-DTW barycenter of Eq. 7,
 * argmin_B sum_k w_k Soft-DTW^gamma(B, Y_k) (w_k = lambda_k / m_k, by default
 * 1 / N_k), by wts_lbfgs_minimize; every evaluation is one softdtw_forward
 * and one softdtw_backward on the device (the iterate is copied in and the
 * values and gradient out, the stream synchronised once per evaluation).
 *   B [M][d]          in: the start (device), out: the last accepted iterate
 *   weights [T]       device, or NULL for 1 / N_k
 *   f_out, n_iter, n_eval, reason   host outputs (any may be NULL)
 * Workspace: wts_workspace_size(WTS_OP_SOFTDTW_LBFGS, M, Y, opt, ...).
 */
int wts_softdtw_barycenter_lbfgs(float* B, int64_t M, const wts_batch* Y, float gamma, const float* weights,
                                 const wts_lbfgs_params* prm, const wts_options* opt, void* workspace,
                                 size_t workspace_bytes, void* stream, double* f_out, int32_t* n_iter,
                                 int32_t* n_eval, int32_t* reason);

/*
 * dba_iterate - one iteration of DTW Barycenter Averaging (Petitjean et al.
 * 2011; the paper cites it in Sec. 2 and compares with it in Table II and
 * Fig. 6 without printing a formula):
 *   1. align every cycle Y_k to B_in (dtw_align);
 *   2. B_out[i] = (sum over k, over (i, j) on pi_k, of y_k[j]) / counts[i],
 *      counts[i] = number of samples aligned to row i over all cycles;
 *   3. cost_before = sum_k DTW(B_in, Y_k) (the intraclass inertia of Sec. 4.2
 *      under the squared cost).
 * Sums are accumulated in FP64 in a fixed order (cycle k ascending, sample j
 * ascending), divided in FP64 and rounded once to FP32: the result does not
 * depend on scheduling.
 *   B_in [M][d], B_out [M][d] (must not alias B_in)
 *   counts [M] out (may be NULL), cost_before: one double, out (may be NULL),
 *   cost [T] out (may be NULL): DTW(B_in, Y_k)
 * Workspace: wts_workspace_size(WTS_OP_DBA_ITERATE, ...).  The paths are kept
 * in the workspace; with every code stored (dir_mode 0) the next call on the
 * same workspace and batch starts its walk from them as guesses (faster
 * between DBA iterations, whose paths move little); any workspace contents
 * give the same result.
 */
int dba_iterate(const float* B_in, float* B_out, int64_t M, const wts_batch* Y, const wts_options* opt,
                void* workspace, size_t workspace_bytes, void* stream,
                int32_t* counts, double* cost_before, float* cost);

/*
 * softdtw_forward - Soft-DTW^gamma(B, Y_k) for every cycle (Eq. 4, computed by
 * the recursion Eq. 5 with the soft minimum of Eq. 3, read with the exponent
 * -a_i/gamma).  The soft minimum is evaluated as
 *     m - gamma ln(sum_i exp(-(a_i - m)/gamma)),  m = min_i a_i,
 * with the hardware ex2 / lg2 approximations (flush-to-zero), in FP32.  Every r(i,j) is kept
 * in the workspace for softdtw_backward (4 bytes per cell plus a skew
 * margin: wts_workspace_size(WTS_OP_SOFTDTW, ...)).  With opt->dir_mode = 1
 * R is not kept: without a band, every band keeps its lanes' state every 16
 * steps (column checkpoints, about R/14 of R's size) besides the band hand-off
 * rows, and softdtw_backward recomputes R 16 steps at a time inside each
 * band's warp (one extra forward pass, all bands in flight at once); with a
 * band, only the hand-off rows are kept and R is recomputed for ckpt_bands
 * bands at a time (the recompute of the next group overlaps the backward of
 * the current one, so R of two groups is kept).  Values and gradients are
 * bit-identical to the stored mode.
 *   B [M][d] (d <= 8), gamma > 0 (gamma = 0 is DTW: use anomaly_score),
 *   value [T] out.
 */
int softdtw_forward(const float* B, int64_t M, const wts_batch* Y, float gamma, const wts_options* opt,
                    void* workspace, size_t workspace_bytes, void* stream, float* value);

/*
 * softdtw_backward - gradient of sum_k g_k Soft-DTW^gamma(B, Y_k) with
 * respect to B (Eq. 6): grad_B[i][c] = sum_k g_k sum_j e_k(i,j) 2 (b_ic - y_jc),
 * where E_k is the reverse recursion of Cuturi and Blondel (cited by the
 * paper): e(M,N) = 1, e(i,j) = sum over the successors s of (i,j) of
 * exp(((r(s) - r(i,j)) - delta(s))/gamma) e(s).  With g_k = lambda_k / m_k this
 * is the gradient of the barycenter objective Eq. 7.
 * The workspace must still hold the R written by softdtw_forward for the same
 * B, Y, gamma and options (the call may be repeated with other g).
 *   grad_value [T] in (g_k), or NULL for Eq. 7's weights with lambda_k = 1:
 *   g_k = 1 / N_k (rounded to FP32, computed on the device);
 *   grad_B [M][d] out; the sum over k is in FP64, k ascending.
 */
int softdtw_backward(const float* B, int64_t M, const wts_batch* Y, float gamma, const float* grad_value,
                     const wts_options* opt, void* workspace, size_t workspace_bytes, void* stream,
                     float* grad_B);

/*
 * wts_adam_step - one Adam update (Kingma and Ba) of n parameters x given
 * grad, with first / second moments m, v (zero before step t = 1), used to
 * descend the Eq. 7 objective with the gradient of softdtw_backward.
 */
int wts_adam_step(float* x, const float* grad, float* m, float* v, int64_t n, float lr, float beta1, float beta2,
                  float eps, int32_t t, void* stream);

/*
 * wts_softdtw_barycenter_adam - the Soft-DTW barycenter of Eq. 7,
 * argmin_B sum_k g_k Soft-DTW^gamma(B, Y_k) (g_k = lambda_k / m_k; weights
 * NULL = 1 / N_k), by `steps` Adam steps (Kingma and Ba; the paper's optimiser
 * is L-BFGS, see wts_softdtw_barycenter_lbfgs): step t = 1..steps runs
 * softdtw_forward, softdtw_backward with the weights, and wts_adam_step(t)
 * on B, all queued on `stream` (no synchronisation; the moments start at 0).
 *   B [M][d]              in: the start (device), out: B after the last step
 *   values [steps][T]     out (may be NULL): Soft-DTW^gamma(B_t, Y_k) at the
 *                         start of each step
 * Workspace: wts_workspace_size(WTS_OP_SOFTDTW_ADAM, M, Y, opt, ...).
 */
int wts_softdtw_barycenter_adam(float* B, int64_t M, const wts_batch* Y, float gamma, const float* weights,
                                int32_t steps, float lr, float beta1, float beta2, float eps, const wts_options* opt,
                                void* workspace, size_t workspace_bytes, void* stream, float* values);

/*
 * wts_autotune - pick the launch options (rows per lane, warps per block) of
 * the wavefront for operation op (WTS_OP_ANOMALY_SCORE, WTS_OP_DTW_ALIGN or
 * WTS_OP_DBA_ITERATE) on this batch by timing each candidate that fits in the
 * given workspace (one warm-up and the best of two timed passes each, CUDA
 * events on `stream`; synchronises it; the default shape is kept unless another
 * is more than 1 % faster).  Results are cached per (op, d, M, T, total
 * length); a cached answer costs nothing.  best: out (host); best_ms: out
 * (host, may be NULL), the wavefront time of the chosen options.
 */
int wts_autotune(int op, const float* B, int64_t M, const wts_batch* Y, void* workspace, size_t workspace_bytes,
                 void* stream, wts_options* best, float* best_ms);

/*
 * wts_compact_nan - batch staging of Sec. 3.1: every time step with a missing
 * value (NaN in any channel) is removed and the cycles are re-packed in order,
 * giving the irregularly sampled series Y the alignment uses.
 *   Y: the raw batch (samples may be NaN; lengths >= 1)
 *   out [rows][d] out: compacted samples (at most as many rows as the input)
 *   out_offsets [T+1] out (device): offsets of the compacted cycles; copy them
 *   to the host to build the compacted batch.  A cycle whose every step is
 *   missing comes out empty, which the alignment calls reject.
 * Workspace: wts_workspace_size(WTS_OP_COMPACT_NAN, 0, Y, NULL, &bytes).
 */
int wts_compact_nan(const wts_batch* Y, void* workspace, size_t workspace_bytes, void* stream, float* out,
                    int64_t* out_offsets);

/*
 * wts_pad_last - the equal-length form of Sec. 4.1: every cycle extended with
 * its last sample to a common length L (the paper pads this way for its
 * Soft-DTW runs):  out[k][j][c] = y_k[min(j, N_k - 1)][c],  j < L.
 *   L: 0 = the longest cycle's length; a shorter L than that is WTS_EINVAL
 *   out [T][L][d] out (device); with offsets k * L it is a batch of T cycles
 *   of length L.
 * No workspace; asynchronous on `stream`.
 */
int wts_pad_last(const wts_batch* Y, int64_t L, void* stream, float* out);

/*
 * wts_select_channel - channel c of every cycle (the paper aligns, averages
 * and scores each joint on its own, Sec. 5):  out[t] = data[t][c] for every
 * sample t of the packed batch; with Y's offsets and d = 1, out is the batch
 * of that channel.
 *   c in [0, d); out [sum_k N_k] out (device).
 * No workspace; asynchronous on `stream`.
 */
int wts_select_channel(const wts_batch* Y, int32_t c, void* stream, float* out);

/*
 * wts_pairwise_dtw - DTW between every two cycles of the batch (rows = the
 * lower-index cycle), for the medoid that initialises DBA.
 *   C [T][T] out: symmetric, C[a][a] = 0.
 * Workspace: wts_workspace_size(WTS_OP_PAIRWISE, 0, Y, ...).  T >= 2.
 */
int wts_pairwise_dtw(const wts_batch* Y, const wts_options* opt, void* workspace, size_t workspace_bytes,
                     void* stream, float* C);

/*
 * wts_medoid - argmin_a sum_b C[a][b] (row sums in FP64, b ascending; ties go
 * to the lowest a).  C [n][n] from wts_pairwise_dtw; sums [n] out (double);
 * index: one int32, out.
 */
int wts_medoid(const float* C, int32_t n, void* stream, double* sums, int32_t* index);

/*
 * wts_resample - linear resampling of x [N][d] to out [M][d] over the same
 * span (position m -> m (N-1)/(M-1)), in FP64, rounded to FP32; used to bring
 * an initial barycenter to the barycenter length m_b (Sec. 3.3).
 */
int wts_resample(const float* x, int64_t N, int32_t d, float* out, int64_t M, void* stream);

/*
 * wts_euclid_mean - Euclidean mean of the batch's cycles, each resampled to M
 * (the default barycenter initialisation of Table I): out [M][d].
 */
int wts_euclid_mean(const wts_batch* Y, int64_t M, float* out, void* stream);

/*
 * anomaly_score_noalloc - anomaly_score without a caller workspace.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory - code that runs inside a host whose device
 * memory is owned and budgeted by another allocator, or a scoring loop that
 * must not stall (cudaMalloc and cudaFree can synchronise the device and take
 * unbounded time).  It computes exactly what anomaly_score computes, with the
 * same inputs and outputs (all caller-owned device pointers), but its scratch
 * is a fixed 32 MiB array inside the library: every GPU that loads the library
 * holds those 32 MiB until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *  - A batch whose scratch need (the WTS_OP_ANOMALY_SCORE workspace size)
 *    exceeds 32 MiB is rejected with WTS_ENOMEM before anything is launched;
 *    for M = 25,000 and d > 2 that is about two 30,000-sample cycles per call.
 *  - Each call looks up the array's device address with the current device
 *    current (outside stream capture; a call being captured uses the address
 *    found by an earlier call on that device).  Make the first call on each
 *    device before any stream capture; after a cudaDeviceReset, make one call
 *    outside capture before capturing again.
 *  - All calls share the one array and it keeps the last call's contents; each
 *    call clears what must start at zero.  Calls whose work overlaps on the
 *    GPU (other streams, other host threads, without ordering between them)
 *    race on the array: serialise them.
 *  - The array's device status word (a non-finite sample, or a wait that gave
 *    up) is read by wts_noalloc_read_status; it holds the last call's status.
 */
int anomaly_score_noalloc(const float* B, int64_t M, const wts_batch* Y, const wts_options* opt,
                          void* stream, float* score, float* cost, int32_t* plen);

/*
 * wts_noalloc_read_status - synchronise `stream` and read the device status
 * word of the fixed scratch of anomaly_score_noalloc on the current device
 * into *status (host): WTS_OK, WTS_EINVAL (a non-finite sample) or
 * WTS_ETIMEOUT, as wts_read_status reports them for a workspace.  Call it
 * after the anomaly_score_noalloc call it should report on, on the same
 * stream, before the next one.  No allocation.
 */
int wts_noalloc_read_status(void* stream, int32_t* status);

#ifdef __cplusplus
}
#endif

#endif /* WETSAND_H */
