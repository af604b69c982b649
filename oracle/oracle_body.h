/*
 * Body of the CPU oracle, written once and instantiated twice by
 * wetsand_oracle.c: REAL = double (the reference precision) and REAL = float
 * (the FP32 mirror, whose operation order is fixed so that a warping path,
 * which is an integer decision taken from float comparisons, is decided in the
 * same precision as on the GPU).
 *
 * TEST INFRASTRUCTURE ONLY: nothing on the product path links this code.
 *
 * Conventions (paper Sec. 3.2-3.4): rows i index the prototype / barycenter B
 * (length M), columns j index the cycle Y (length N); samples are d-channel
 * vectors stored row-major ([M][d], [N][d]).  Internally the recursion uses the
 * paper's 1-based indices with a padded row 0 and column 0 (Eq. 5); outputs
 * are 0-based.
 *
 * Required macros: REAL, FMA(a,b,c), EXP(x), LOG(x), SQRT(x), SFX(name).
 *
 * The ORACLE_PLANT_* switches are mutation hooks, off in every normal build:
 * the pin tests compile the oracle once per switch, each planting one
 * plausible mistake (a dropped cost term, a wrong index, a wrong sign, a
 * transposed operand, a different tie order), and check that at least one pin
 * fails for each.
 */

/* delta(b_i, y_j) (Definition "Distance Matrix", Sec. 3.2).  The sum
 * s = sum_c (b_c - y_c)^2 is accumulated channel by channel from 0 with one
 * fused multiply-add per channel.  cost_kind 0: delta = s, the squared l2 norm
 * (the default reading); cost_kind 1: delta = sqrt(s), the l2 norm itself (the
 * paper's wording), rounded once in the working precision. */
static REAL SFX(finish_cost)(REAL acc, int cost_kind)
{
#ifdef ORACLE_PLANT_L2_NO_SQRT
    (void)cost_kind;
    return acc;
#else
    return cost_kind ? SQRT(acc) : acc;
#endif
}

static REAL SFX(local_cost)(const float* b, const float* y, int d, int cost_kind)
{
    REAL acc = 0;
    for (int c = 0; c < d; ++c) {
        REAL t = (REAL)b[c] - (REAL)y[c];
#ifdef ORACLE_PLANT_DROP_CHANNEL
        if (c == d - 1 && d > 1) break;
#endif
        acc = FMA(t, t, acc);
    }
    return SFX(finish_cost)(acc, cost_kind);
}

/* Same cost with a REAL-typed prototype row (DBA keeps B in REAL). */
static REAL SFX(local_cost_r)(const REAL* b, const float* y, int d, int cost_kind)
{
    REAL acc = 0;
    for (int c = 0; c < d; ++c) {
        REAL t = b[c] - (REAL)y[c];
#ifdef ORACLE_PLANT_DROP_CHANNEL
        if (c == d - 1 && d > 1) break;
#endif
        acc = FMA(t, t, acc);
    }
    return SFX(finish_cost)(acc, cost_kind);
}

/*
 * DTW (Eq. 1) by the cumulative cost recursion Eq. 5 with gamma = 0:
 *   r(0,0) = 0, r(i,0) = r(0,j) = +inf, r(i,j) = delta(i,j) + min(r(i-1,j-1), r(i-1,j), r(i,j-1)).
 * Each cell also records which predecessor gave the minimum; equal values are
 * resolved diag first, then up (i-1,j), then left (i,j-1).  Walking those
 * choices back from (M,N) gives the optimal complete alignment path
 * (Definition "Alignment path"): among all optimal paths, the one whose
 * reversed step sequence is lexicographically greatest under
 * diag > up > left.
 *
 * B is REAL-typed (so that DBA can iterate in the working precision).
 * Outputs (any may be NULL): cost = r(M,N); plen = |pi|; jlo/jhi[M] = first and
 * last column of row i on the path; pi_i/pi_j[M+N-1] = the path from (0,0).
 * Returns 0, or -1 on allocation failure.
 */
static int SFX(dtw_core)(const REAL* B, int64_t M, const float* Y, int64_t N, int d,
                         REAL* cost, int32_t* plen, int32_t* jlo, int32_t* jhi,
                         int32_t* pi_i, int32_t* pi_j, double band, int cost_kind)
{
    /* Sakoe-Chiba band (Table I: a width given as a fraction of the signals'
     * length; reading for unequal lengths): 0-based cell (i, j) is inside when
     * |i N - j M| <= floor(band M N), i.e. |i/M - j/N| <= band in normalised
     * time.  band <= 0: no band.  Outside cells are +inf.  A band narrower
     * than max(M, N) may hold no path: refused (-3). */
    const int64_t bound = band > 0 ? (int64_t)floor(band * (double)M * (double)N) : -1;
    if (band > 0 && bound < (M > N ? M : N)) return -3;
    REAL* prev = (REAL*)malloc((size_t)(N + 1) * sizeof(REAL));
    REAL* cur = (REAL*)malloc((size_t)(N + 1) * sizeof(REAL));
    uint8_t* choice = (uint8_t*)malloc((size_t)M * (size_t)N);
    if (!prev || !cur || !choice) { free(prev); free(cur); free(choice); return -1; }

    prev[0] = 0;
    for (int64_t j = 1; j <= N; ++j) prev[j] = (REAL)INFINITY;
    for (int64_t i = 1; i <= M; ++i) {
        cur[0] = (REAL)INFINITY;
        const REAL* bi = B + (i - 1) * d;
        for (int64_t j = 1; j <= N; ++j) {
            if (bound >= 0) {
#ifdef ORACLE_PLANT_BAND_SWAP
                const int64_t t = (i - 1) * M - (j - 1) * N;
#else
                const int64_t t = (i - 1) * N - (j - 1) * M;
#endif
                if (t > bound || -t > bound) {
                    cur[j] = (REAL)INFINITY;
                    choice[(i - 1) * N + (j - 1)] = 0;
                    continue;
                }
            }
#ifdef ORACLE_PLANT_DIAG_INDEX
            REAL dg = prev[j], up = prev[j], lf = cur[j - 1];
#else
            REAL dg = prev[j - 1], up = prev[j], lf = cur[j - 1];
#endif
            REAL m;
            uint8_t ch;
#ifdef ORACLE_PLANT_TIE_ORDER
            if (up <= dg && up <= lf) { ch = 1; m = up; }
            else if (dg <= lf) { ch = 0; m = dg; }
#else
            if (dg <= up && dg <= lf) { ch = 0; m = dg; }
            else if (up <= lf) { ch = 1; m = up; }
#endif
            else { ch = 2; m = lf; }
            cur[j] = SFX(local_cost_r)(bi, Y + (j - 1) * d, d, cost_kind) + m;
            choice[(i - 1) * N + (j - 1)] = ch;
        }
        REAL* t = prev; prev = cur; cur = t;
    }
    if (cost) *cost = prev[N];

    /* backtrack from (M,N) to (1,1) */
    int64_t i = M, j = N, len = 0;
    if (jhi) jhi[M - 1] = (int32_t)(N - 1);
    int64_t cap = M + N - 1;
    int32_t* ti = pi_i ? (int32_t*)malloc((size_t)cap * sizeof(int32_t)) : NULL;
    int32_t* tj = pi_j ? (int32_t*)malloc((size_t)cap * sizeof(int32_t)) : NULL;
    for (;;) {
        if (ti) ti[len] = (int32_t)(i - 1);
        if (tj) tj[len] = (int32_t)(j - 1);
        ++len;
        if (i == 1 && j == 1) break;
        uint8_t ch = choice[(i - 1) * N + (j - 1)];
        /* a valid choice matrix never leaves the grid: only left on row 1,
         * only up on column 1 (both predecessors elsewhere are +inf) */
        if ((i == 1 && ch != 2) || (j == 1 && ch != 1) || len >= cap) { len = -1; break; }
        if (ch == 0) {            /* diag: leave row i at column j */
            if (jlo) jlo[i - 1] = (int32_t)(j - 1);
            --i; --j;
            if (jhi) jhi[i - 1] = (int32_t)(j - 1);
        } else if (ch == 1) {     /* up */
            if (jlo) jlo[i - 1] = (int32_t)(j - 1);
            --i;
            if (jhi) jhi[i - 1] = (int32_t)(j - 1);
        } else {                  /* left */
            --j;
        }
    }
    if (len < 0) { free(ti); free(tj); free(prev); free(cur); free(choice); return -2; }
    if (jlo) jlo[0] = 0;
    if (plen) *plen = (int32_t)len;
    if (ti) { for (int64_t k = 0; k < len; ++k) pi_i[k] = ti[len - 1 - k]; free(ti); }
    if (tj) { for (int64_t k = 0; k < len; ++k) pi_j[k] = tj[len - 1 - k]; free(tj); }
    free(prev); free(cur); free(choice);
    return 0;
}

/* DTW of one pair with a float prototype (converted exactly to REAL). */
int SFX(orc_dtw)(const float* B, int64_t M, const float* Y, int64_t N, int d,
                 REAL* cost, int32_t* plen, int32_t* jlo, int32_t* jhi,
                 int32_t* pi_i, int32_t* pi_j, double band, int cost_kind)
{
    REAL* Br = (REAL*)malloc((size_t)M * d * sizeof(REAL));
    if (!Br) return -1;
    for (int64_t k = 0; k < M * d; ++k) Br[k] = (REAL)B[k];
    int rc = SFX(dtw_core)(Br, M, Y, N, d, cost, plen, jlo, jhi, pi_i, pi_j, band, cost_kind);
    free(Br);
    return rc;
}

/*
 * Similarity score (Eq. 8) for every cycle of a packed batch:
 *   d_score(B, C_k) = DTW(B, C_k) / |pi_k|, divided in the working precision.
 * Pairs are independent; they are spread over OpenMP threads.
 */
int SFX(orc_score)(const float* B, int64_t M, const float* Y, const int64_t* offsets, int T, int d,
                   REAL* score, REAL* cost, int32_t* plen, double band, int cost_kind)
{
    REAL* Br = (REAL*)malloc((size_t)M * d * sizeof(REAL));
    if (!Br) return -1;
    for (int64_t k = 0; k < M * d; ++k) Br[k] = (REAL)B[k];
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int k = 0; k < T; ++k) {
        REAL c; int32_t L;
        int64_t N = offsets[k + 1] - offsets[k];
        bad |= SFX(dtw_core)(Br, M, Y + offsets[k] * d, N, d, &c, &L, NULL, NULL, NULL, NULL, band, cost_kind) != 0;
        if (cost) cost[k] = c;
        if (plen) plen[k] = L;
        if (score) score[k] = c / (REAL)L;
    }
    free(Br);
    return bad ? -1 : 0;
}

/*
 * One DBA iteration (DTW Barycenter Averaging, the classic DBA of the
 * paper's Sec. 2 and the Table II comparison; the paper cites it without a
 * formula):
 *   1. align every cycle Y_k to B_in with DTW;
 *   2. B_out[i] = (sum over k, over (i,j) on pi_k, of y_k[j]) / counts[i],
 *      counts[i] = number of such associations (pooled over all cycles);
 *   3. cost_before = sum_k DTW(B_in, Y_k).
 * Sums are kept in double, added k ascending then j ascending, divided in
 * double and rounded once to REAL.  costs[k] (optional) = DTW(B_in, Y_k).
 */
int SFX(orc_dba)(const REAL* B_in, REAL* B_out, int64_t M, const float* Y, const int64_t* offsets,
                 int T, int d, int32_t* counts, double* cost_before, REAL* costs, double band,
                 int cost_kind)
{
    int32_t* jlo = (int32_t*)malloc((size_t)T * M * sizeof(int32_t));
    int32_t* jhi = (int32_t*)malloc((size_t)T * M * sizeof(int32_t));
    REAL* ck = (REAL*)malloc((size_t)T * sizeof(REAL));
    double* sums = (double*)calloc((size_t)M * d, sizeof(double));
    int64_t* cnt = (int64_t*)calloc((size_t)M, sizeof(int64_t));
    if (!jlo || !jhi || !ck || !sums || !cnt) { free(jlo); free(jhi); free(ck); free(sums); free(cnt); return -1; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int k = 0; k < T; ++k) {
        int64_t N = offsets[k + 1] - offsets[k];
        bad |= SFX(dtw_core)(B_in, M, Y + offsets[k] * d, N, d, &ck[k], NULL,
                             jlo + (int64_t)k * M, jhi + (int64_t)k * M, NULL, NULL, band, cost_kind) != 0;
    }
    if (!bad) {
        for (int k = 0; k < T; ++k) {
            const float* y = Y + offsets[k] * d;
            for (int64_t i = 0; i < M; ++i) {
                int32_t a = jlo[(int64_t)k * M + i], b = jhi[(int64_t)k * M + i];
                for (int32_t j = a; j <= b; ++j)
                    for (int c = 0; c < d; ++c) sums[i * d + c] += (double)y[(int64_t)j * d + c];
                cnt[i] += (int64_t)(b - a + 1);
            }
        }
        for (int64_t i = 0; i < M; ++i) {
            for (int c = 0; c < d; ++c) B_out[i * d + c] = (REAL)(sums[i * d + c] / (double)cnt[i]);
            if (counts) counts[i] = (int32_t)cnt[i];
        }
        double s = 0;
        for (int k = 0; k < T; ++k) s += (double)ck[k];
        if (cost_before) *cost_before = s;
        if (costs) for (int k = 0; k < T; ++k) costs[k] = ck[k];
    }
    free(jlo); free(jhi); free(ck); free(sums); free(cnt);
    return bad ? -1 : 0;
}

/* min^gamma of three values (Eq. 3).  gamma = 0 is the plain min.  For
 * gamma > 0 the sum is evaluated after factoring out exp(-m/gamma), m the
 * smallest argument (an exact identity that keeps the exponentials in
 * range); +inf arguments contribute exp(-inf) = 0. */
static REAL SFX(softmin3)(REAL a, REAL b, REAL c, REAL gamma)
{
    REAL m = a < b ? a : b;
    m = m < c ? m : c;
    if (gamma == 0) return m;
    REAL s = EXP(-(a - m) / gamma) + EXP(-(b - m) / gamma) + EXP(-(c - m) / gamma);
#ifdef ORACLE_PLANT_SOFTMIN_SIGN
    return m + gamma * LOG(s);
#else
    return m - gamma * LOG(s);
#endif
}

/*
 * Soft-DTW^gamma(B, Y) (Eq. 4) by the recursion Eq. 5, and its gradient with
 * respect to B (Eq. 6).  E is the matrix of the reverse recursion (Cuturi and
 * Blondel 2017, cited by the paper without restating it): with
 *   r(i,N+1) = r(M+1,j) = -inf, r(M+1,N+1) = r(M,N), delta = 0 on the extra
 *   row/column, e(M+1,N+1) = 1 and e = 0 elsewhere on the border,
 *   e(i,j) = sum over successors s in {(i+1,j), (i,j+1), (i+1,j+1)} of
 *            exp((r(s) - r(i,j) - delta(s)) / gamma) * e(s),
 * i.e. e(i,j) = d r(M,N) / d r(i,j), the expected alignment matrix.  Then
 *   grad[i][c] = sum_j e(i,j) * d delta(i,j) / d b_ic, which is
 *   sum_j e(i,j) * 2 (b_ic - y_jc) for the squared norm.
 *
 * R and E (optional, may be NULL) receive the (M+2) x (N+2) matrices in
 * 1-based layout.  grad (optional) is [M][d].  gamma must be > 0 for the
 * gradient.  Returns 0 or -1.
 */
int SFX(orc_softdtw)(const float* B, int64_t M, const float* Y, int64_t N, int d, REAL gamma,
                     REAL* value, REAL* R_out, REAL* E_out, REAL* grad, double band, int cost_kind)
{
    /* Sakoe-Chiba band as in dtw_core: 0-based cell (i, j) kept when
     * |i N - j M| <= floor(band M N); cells outside are +inf in the forward
     * and, like the border, -inf with delta = 0 (no successor weight) in the
     * reverse recursion. */
    const int64_t bound = band > 0 ? (int64_t)floor(band * (double)M * (double)N) : -1;
    if (band > 0 && bound < (M > N ? M : N)) return -3;
#define SOFT_OUT(i, j) (bound >= 0 && (((i) - 1) * N - ((j) - 1) * M > bound || ((j) - 1) * M - ((i) - 1) * N > bound))
    const int64_t W = N + 2;
    size_t cells = (size_t)(M + 2) * (size_t)W;
    REAL* R = R_out ? R_out : (REAL*)malloc(cells * sizeof(REAL));
    REAL* D = (REAL*)malloc(cells * sizeof(REAL));
    if (!R || !D) { if (!R_out) free(R); free(D); return -1; }
    for (size_t k = 0; k < cells; ++k) { R[k] = (REAL)INFINITY; D[k] = 0; }
    R[0] = 0;
    for (int64_t i = 1; i <= M; ++i)
        for (int64_t j = 1; j <= N; ++j) {
            if (SOFT_OUT(i, j)) continue;          /* stays +inf */
            REAL dl = SFX(local_cost)(B + (i - 1) * d, Y + (j - 1) * d, d, cost_kind);
            D[i * W + j] = dl;
            R[i * W + j] = dl + SFX(softmin3)(R[(i - 1) * W + j - 1], R[(i - 1) * W + j],
                                              R[i * W + j - 1], gamma);
        }
    if (value) *value = R[M * W + N];

    int rc = 0;
    if (E_out || grad) {
        if (!(gamma > 0)) { rc = -1; goto done; }
        REAL* E = E_out ? E_out : (REAL*)malloc(cells * sizeof(REAL));
        if (!E) { rc = -1; goto done; }
        for (size_t k = 0; k < cells; ++k) E[k] = 0;
        for (int64_t i = 1; i <= M; ++i) R[i * W + N + 1] = (REAL)-INFINITY;
        for (int64_t j = 1; j <= N; ++j) R[(M + 1) * W + j] = (REAL)-INFINITY;
        R[(M + 1) * W + N + 1] = R[M * W + N];
        E[(M + 1) * W + N + 1] = 1;
        for (int64_t i = 1; i <= M; ++i)
            for (int64_t j = 1; j <= N; ++j)
                if (SOFT_OUT(i, j)) R[i * W + j] = (REAL)-INFINITY;
        for (int64_t i = M; i >= 1; --i)
            for (int64_t j = N; j >= 1; --j) {
                if (SOFT_OUT(i, j)) continue;      /* e stays 0 */
                REAL r = R[i * W + j];
                REAL a = EXP((R[(i + 1) * W + j] - r - D[(i + 1) * W + j]) / gamma);
                REAL b = EXP((R[i * W + j + 1] - r - D[i * W + j + 1]) / gamma);
                REAL c = EXP((R[(i + 1) * W + j + 1] - r - D[(i + 1) * W + j + 1]) / gamma);
#ifdef ORACLE_PLANT_E_TRANSPOSE
                E[i * W + j] = a * E[i * W + j + 1] + b * E[(i + 1) * W + j] + c * E[(i + 1) * W + j + 1];
#else
                E[i * W + j] = a * E[(i + 1) * W + j] + b * E[i * W + j + 1] + c * E[(i + 1) * W + j + 1];
#endif
            }
        if (grad) {
            /* d delta / d b_ic: 2 (b_ic - y_jc) for the squared norm;
             * (b_ic - y_jc) / delta for the norm itself, 0 where delta = 0 (the
             * norm has no derivative there; 0 is the minimum-norm subgradient) */
            for (int64_t i = 1; i <= M; ++i)
                for (int c = 0; c < d; ++c) {
                    REAL g = 0;
                    for (int64_t j = 1; j <= N; ++j) {
                        const REAL t = (REAL)B[(i - 1) * d + c] - (REAL)Y[(j - 1) * d + c];
                        const REAL dl = D[i * W + j];
                        if (!cost_kind)
                            g += E[i * W + j] * 2 * t;
#ifdef ORACLE_PLANT_L2_GRAD_TWO
                        else if (dl > 0)
                            g += E[i * W + j] * 2 * t / dl;
#else
                        else if (dl > 0)
                            g += E[i * W + j] * t / dl;
#endif
                    }
                    grad[(i - 1) * d + c] = g;
                }
        }
        /* restore the forward border so R_out holds Eq. 5's matrix */
        for (int64_t i = 1; i <= M; ++i) R[i * W + N + 1] = (REAL)INFINITY;
        for (int64_t j = 1; j <= N + 1; ++j) R[(M + 1) * W + j] = (REAL)INFINITY;
        for (int64_t i = 1; i <= M; ++i)
            for (int64_t j = 1; j <= N; ++j)
                if (SOFT_OUT(i, j)) R[i * W + j] = (REAL)INFINITY;
        if (!E_out) free(E);
    }
done:
#undef SOFT_OUT
    if (!R_out) free(R);
    free(D);
    return rc;
}

/*
 * Soft-DTW barycenter objective (Eq. 7) over a packed batch and its gradient:
 *   L(B) = sum_k w_k * Soft-DTW^gamma(B, Y_k),  w_k = lambda_k / m_k
 * (weights[k] given explicitly; NULL means lambda_k = 1, w_k = 1 / N_k).
 * values[k] = Soft-DTW^gamma(B, Y_k); grad = sum_k w_k * grad_k, summed in k
 * order.  Pairs run on OpenMP threads.
 */
int SFX(orc_softdtw_batch)(const float* B, int64_t M, const float* Y, const int64_t* offsets, int T, int d,
                           REAL gamma, const REAL* weights, REAL* values, REAL* loss, REAL* grad, double band,
                           int cost_kind)
{
    REAL* g = grad ? (REAL*)calloc((size_t)T * M * d, sizeof(REAL)) : NULL;
    REAL* v = (REAL*)malloc((size_t)T * sizeof(REAL));
    if (!v || (grad && !g)) { free(g); free(v); return -1; }
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int k = 0; k < T; ++k) {
        int64_t N = offsets[k + 1] - offsets[k];
        bad |= SFX(orc_softdtw)(B, M, Y + offsets[k] * d, N, d, gamma, &v[k], NULL, NULL,
                                g ? g + (int64_t)k * M * d : NULL, band, cost_kind) != 0;
    }
    if (!bad) {
        REAL L = 0;
        for (int k = 0; k < T; ++k) {
            REAL w = weights ? weights[k] : (REAL)1 / (REAL)(offsets[k + 1] - offsets[k]);
            if (values) values[k] = v[k];
            L += w * v[k];
        }
        if (loss) *loss = L;
        if (grad) {
            for (int64_t q = 0; q < M * d; ++q) grad[q] = 0;
            for (int k = 0; k < T; ++k) {
                REAL w = weights ? weights[k] : (REAL)1 / (REAL)(offsets[k + 1] - offsets[k]);
                for (int64_t q = 0; q < M * d; ++q) grad[q] += w * g[(int64_t)k * M * d + q];
            }
        }
    }
    free(g); free(v);
    return bad ? -1 : 0;
}

/*
 * Sub-DTW (Sec. 3.2): the minimum over 0 <= a <= b < N of DTW(X, Y[a..b]),
 * the whole of X (rows, length M) against the best contiguous piece of Y
 * (columns).  Computed by the recursion of Eq. 5 (gamma = 0) with a free
 * start: the padded row 0 is r(0,j) = 0 for every j >= 0 (a path may begin in
 * any column), column 0 keeps r(i,0) = +inf for i >= 1.  Then
 *   cost = min_j r(M, j),  b* = the smallest such j (reading: the paper does
 *   not say which end wins a tie),
 * and walking the recorded choices (tie order diag > up > left, as in DTW)
 * back from (M, b*) until the walk leaves row 1 gives a*, the first column of
 * the subsequence.  Outputs are 0-based; jlo/jhi[M] are the columns of each
 * row of X on the path; plen = |pi| (cells on the path).
 * Returns 0, -1 on allocation failure, -2 if the walk leaves the grid.
 */
int SFX(orc_subdtw)(const float* X, int64_t M, const float* Y, int64_t N, int d,
                    REAL* cost, int32_t* a_star, int32_t* b_star, int32_t* plen,
                    int32_t* jlo, int32_t* jhi, int cost_kind)
{
    REAL* prev = (REAL*)malloc((size_t)(N + 1) * sizeof(REAL));
    REAL* cur = (REAL*)malloc((size_t)(N + 1) * sizeof(REAL));
    uint8_t* choice = (uint8_t*)malloc((size_t)M * (size_t)N);
    if (!prev || !cur || !choice) { free(prev); free(cur); free(choice); return -1; }

    for (int64_t j = 0; j <= N; ++j) prev[j] = 0;      /* free start */
#ifdef ORACLE_PLANT_SUB_FIXED_START
    for (int64_t j = 1; j <= N; ++j) prev[j] = (REAL)INFINITY;
#endif
    for (int64_t i = 1; i <= M; ++i) {
        cur[0] = (REAL)INFINITY;
        const float* xi = X + (i - 1) * d;
        for (int64_t j = 1; j <= N; ++j) {
            REAL dg = prev[j - 1], up = prev[j], lf = cur[j - 1];
            REAL m;
            uint8_t ch;
            if (dg <= up && dg <= lf) { ch = 0; m = dg; }
            else if (up <= lf) { ch = 1; m = up; }
            else { ch = 2; m = lf; }
            cur[j] = SFX(local_cost)(xi, Y + (j - 1) * d, d, cost_kind) + m;
            choice[(i - 1) * N + (j - 1)] = ch;
        }
        REAL* t = prev; prev = cur; cur = t;
    }
    /* prev holds row M: the cheapest end column, the first one on ties */
    int64_t jb = 1;
    for (int64_t j = 2; j <= N; ++j)
#ifdef ORACLE_PLANT_SUB_LAST_END
        if (prev[j] <= prev[jb]) jb = j;
#else
        if (prev[j] < prev[jb]) jb = j;
#endif
    if (cost) *cost = prev[jb];
    if (b_star) *b_star = (int32_t)(jb - 1);

    int64_t i = M, j = jb, len = 0;
    if (jhi) jhi[M - 1] = (int32_t)(j - 1);
    for (;;) {
        ++len;
        uint8_t ch = choice[(i - 1) * N + (j - 1)];
        if (i == 1 && ch != 2) break;           /* the path starts here (row 0 is free) */
        if ((j == 1 && ch != 1) || len > M + N) { len = -1; break; }
        if (ch == 0) {
            if (jlo) jlo[i - 1] = (int32_t)(j - 1);
            --i; --j;
            if (jhi) jhi[i - 1] = (int32_t)(j - 1);
        } else if (ch == 1) {
            if (jlo) jlo[i - 1] = (int32_t)(j - 1);
            --i;
            if (jhi) jhi[i - 1] = (int32_t)(j - 1);
        } else {
            --j;
        }
    }
    free(prev); free(cur); free(choice);
    if (len < 0) return -2;
    if (jlo) jlo[0] = (int32_t)(j - 1);
    if (a_star) *a_star = (int32_t)(j - 1);
    if (plen) *plen = (int32_t)len;
    return 0;
}
