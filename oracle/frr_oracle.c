/*
 * frr_oracle.c -- plain, slow FP64 CPU oracle for the rerandomization balance
 * check of FastRerandomize (Goldstein, Jerzak, Kamat, Zhu; arXiv 2501.07642).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path links, loads or calls
 * this file: it is used by tests/, by the smoke check and by the benchmark's
 * CPU-baseline leg. It shares no code, header or table with the CUDA path.
 *
 * Every routine is the plain definition written out step by step, in FP64,
 * compiled with -ffp-contract=off (no implicit contraction), with sums taken in
 * ascending index order. The dot products of the preparation (covariance,
 * Cholesky factor, forward substitution) add each term with one explicit fused
 * multiply-add, fma() -- a single rounding per term; every other operation is
 * rounded on its own. There is no blocking, fusion or reordering.
 *
 * Pins: each function is checked by tests/test_oracle_pins.py against values
 * fixed by the paper or by mathematics (Philox known-answer vectors, brute-force
 * enumeration, E[M] = d, affine invariance, complement symmetry, the d = 1 closed
 * form, the d = n-1 degeneracy, ranks against the enumeration order, textbook exact randomization p-values, the
 * accepted-count and minimum-p numbers printed in Sec. 2.2). No function is
 * "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11. Ten rounds of the 4x32 Philox S-box; two 32-bit   */
/* multipliers and two Weyl key increments as published there.                */
/* ------------------------------------------------------------------------- */
static const uint32_t PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t PHILOX_WEYL_A = 0x9E3779B9u; /* golden ratio */
static const uint32_t PHILOX_WEYL_B = 0xBB67AE85u; /* sqrt(3) - 1 */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { /* key schedule: bump by the Weyl constants */
            k0 += PHILOX_WEYL_A;
            k1 += PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)PHILOX_MUL_A * (uint64_t)x0;
        uint64_t pb = (uint64_t)PHILOX_MUL_B * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
        uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------- */
/* Key -> assignment (the paper keeps only a PRNG key per accepted draw and   */
/* regenerates the assignment from it, Sec. 2.1 "Key-only storage"; it fixes  */
/* no generator). Reading: key = (pool seed, 64-bit draw index b). Unit i gets */
/* the 32-bit word r_i = word (i mod 4) of Philox4x32-10 with                  */
/*   counter = (floor(i/4), 0, lo32(b), hi32(b)), key = (lo32(seed), hi32(seed)),*/
/* and the n1 units with the lexicographically smallest pairs (r_i, i) are     */
/* treated. Here: build all n pairs, sort them, mark the first n1.            */
/* ------------------------------------------------------------------------- */
typedef struct { uint32_t r; int32_t i; } key_pair;

static int cmp_key_pair(const void* a, const void* b)
{
    const key_pair* p = (const key_pair*)a;
    const key_pair* q = (const key_pair*)b;
    if (p->r != q->r) return p->r < q->r ? -1 : 1;
    return (p->i > q->i) - (p->i < q->i);
}

void oracle_unit_words(uint64_t seed, uint64_t draw, int64_t n, uint32_t* r_out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t j = 0; 4 * j < n; ++j) {
        uint32_t ctr[4] = {(uint32_t)j, 0u, (uint32_t)draw, (uint32_t)(draw >> 32)};
        uint32_t w[4];
        oracle_philox4x32_10(ctr, key, w);
        for (int c = 0; c < 4 && 4 * j + c < n; ++c) r_out[4 * j + c] = w[c];
    }
}

static void assignment_with_scratch(uint64_t seed, uint64_t draw, int64_t n, int64_t n1,
                                    uint8_t* w_out, uint32_t* r, key_pair* pairs)
{
    oracle_unit_words(seed, draw, n, r);
    for (int64_t i = 0; i < n; ++i) { pairs[i].r = r[i]; pairs[i].i = (int32_t)i; }
    qsort(pairs, (size_t)n, sizeof(key_pair), cmp_key_pair);
    memset(w_out, 0, (size_t)n);
    for (int64_t k = 0; k < n1; ++k) w_out[pairs[k].i] = 1;
}

void oracle_assignment(uint64_t seed, uint64_t draw, int64_t n, int64_t n1, uint8_t* w_out)
{
    uint32_t* r = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    key_pair* pairs = (key_pair*)malloc((size_t)n * sizeof(key_pair));
    assignment_with_scratch(seed, draw, n, n1, w_out, r, pairs);
    free(r);
    free(pairs);
}

void oracle_assignments(uint64_t seed, uint64_t first_draw, int64_t count, int64_t n, int64_t n1,
                        uint8_t* w_out /* count x n */)
{
    uint32_t* r = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    key_pair* pairs = (key_pair*)malloc((size_t)n * sizeof(key_pair));
    for (int64_t b = 0; b < count; ++b)
        assignment_with_scratch(seed, first_draw + (uint64_t)b, n, n1, w_out + b * n, r, pairs);
    free(r);
    free(pairs);
}

/* ------------------------------------------------------------------------- */
/* Exact enumeration (Sec. 2.3, randomization_type = "exact"): all C(n, n1)   */
/* assignments, visited as n-bit masks with n1 bits set in increasing integer */
/* order (Gosper's next-combination step). The rank of an assignment is its   */
/* position in that order. Requires n <= 63.                                  */
/* ------------------------------------------------------------------------- */
static uint64_t next_mask(uint64_t v)
{
    uint64_t t = v | (v - 1);
    return (t + 1) | (((~t & -(~t)) - 1) >> (__builtin_ctzll(v) + 1));
}

int64_t oracle_enum_masks(int64_t n, int64_t n1, uint64_t first_rank, int64_t count, uint64_t* masks_out)
{
    if (n < 1 || n > 63 || n1 < 1 || n1 > n) return -1;
    uint64_t v = (n1 == 64) ? ~0ull : ((1ull << n1) - 1);
    uint64_t limit = 1ull << n;
    uint64_t rank = 0;
    int64_t written = 0;
    while (v < limit && written < count) {
        if (rank >= first_rank) masks_out[written++] = v;
        ++rank;
        if (n1 == n) break;
        v = next_mask(v);
    }
    return written;
}

/* Position of a mask in that order, by the combinatorial number system (Knuth,
 * TAOCP Vol. 4A, Sec. 7.2.1.3): with the set positions c_1 < ... < c_n1, the rank
 * is sum_i C(c_i, i). Enumerating in increasing integer order is colexicographic
 * order, whose ranks are exactly these sums. */
static uint64_t binom_exact(int64_t a, int64_t b)
{
    if (b < 0 || b > a) return 0;
    if (b > a - b) b = a - b;
    unsigned __int128 r = 1;
    for (int64_t i = 1; i <= b; ++i) r = r * (unsigned __int128)(a - b + i) / (unsigned __int128)i;
    return (uint64_t)r;
}

uint64_t oracle_rank_of_mask(uint64_t mask)
{
    uint64_t rank = 0;
    int64_t i = 0;
    for (int64_t c = 0; c < 64; ++c)
        if ((mask >> c) & 1u) rank += binom_exact(c, ++i);
    return rank;
}

/* Inverse of oracle_rank_of_mask: for i = n1 down to 1 take the largest c with
 * C(c, i) <= remaining rank. */
uint64_t oracle_mask_of_rank(int64_t n, int64_t n1, uint64_t rank)
{
    uint64_t mask = 0;
    int64_t c = n - 1;
    for (int64_t i = n1; i >= 1; --i) {
        while (binom_exact(c, i) > rank) --c;
        mask |= 1ull << c;
        rank -= binom_exact(c, i);
        --c;
    }
    return mask;
}

static void mask_to_w(uint64_t mask, int64_t n, uint8_t* w)
{
    for (int64_t i = 0; i < n; ++i) w[i] = (uint8_t)((mask >> i) & 1u);
}

/* ------------------------------------------------------------------------- */
/* Covariate preparation (Sec. 2.2 and the "general Sigma_X" remark of App. A):*/
/* centre, sample covariance with the n-1 denominator, optional ridge, an      */
/* unpivoted Cholesky factor S_lambda = L L^T, and whitening Zc = Xc L^{-T} so */
/* that the Mahalanobis distance becomes a Euclidean one.                      */
/*   whiten 0 = CHOL  : S_lambda = S                                           */
/*   whiten 1 = RIDGE : S_lambda = S + lambda * (tr S / d) * I                 */
/*   whiten 2 = DIAG  : L = diag(sqrt(S_jj)) (sum of squared SMDs, Sec. 2.2)   */
/* Returns 0, or -2 when a Cholesky pivot is <= tol * max_j S_jj.              */
/* ------------------------------------------------------------------------- */
int oracle_prep(const double* X, int64_t n, int64_t d, int whiten, double ridge,
                double* Zc /* n x d */, double* L /* d x d lower, may be NULL */,
                double* xbar_out /* d, may be NULL */, double* S_out /* d x d, may be NULL */)
{
    double* xbar = (double*)calloc((size_t)d, sizeof(double));
    double* Xc = (double*)malloc((size_t)(n * d) * sizeof(double));
    double* S = (double*)calloc((size_t)(d * d), sizeof(double));
    double* Lw = (double*)calloc((size_t)(d * d), sizeof(double));
    int status = 0;

    for (int64_t j = 0; j < d; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += X[i * d + j];
        xbar[j] = s / (double)n;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < d; ++j) Xc[i * d + j] = X[i * d + j] - xbar[j];
    for (int64_t j = 0; j < d; ++j)
        for (int64_t k = 0; k < d; ++k) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) s = fma(Xc[i * d + j], Xc[i * d + k], s);
            S[j * d + k] = s / (double)(n - 1);
        }

    double maxdiag = 0.0, trace = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        trace += S[j * d + j];
        if (S[j * d + j] > maxdiag) maxdiag = S[j * d + j];
    }
    const double tol = 1e-12;

    if (whiten == 2) {
        for (int64_t j = 0; j < d; ++j) {
            if (!(S[j * d + j] > tol * maxdiag)) { status = -2; goto done; }
            Lw[j * d + j] = sqrt(S[j * d + j]);
        }
    } else {
        double* A = (double*)malloc((size_t)(d * d) * sizeof(double));
        memcpy(A, S, (size_t)(d * d) * sizeof(double));
        if (whiten == 1) {
            double add = ridge * (trace / (double)d);
            for (int64_t j = 0; j < d; ++j) A[j * d + j] += add;
        }
        /* column-oriented Cholesky, ascending k */
        for (int64_t j = 0; j < d; ++j) {
            double s = A[j * d + j];
            for (int64_t k = 0; k < j; ++k) s = fma(-Lw[j * d + k], Lw[j * d + k], s);
            if (!(s > tol * maxdiag)) { status = -2; free(A); goto done; }
            double ljj = sqrt(s);
            Lw[j * d + j] = ljj;
            for (int64_t i = j + 1; i < d; ++i) {
                double t = A[i * d + j];
                for (int64_t k = 0; k < j; ++k) t = fma(-Lw[i * d + k], Lw[j * d + k], t);
                Lw[i * d + j] = t / ljj;
            }
        }
        free(A);
    }

    /* Zc row i solves L z = Xc_i^T by forward substitution */
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < d; ++j) {
            double t = Xc[i * d + j];
            for (int64_t k = 0; k < j; ++k) t = fma(-Lw[j * d + k], Zc[i * d + k], t);
            Zc[i * d + j] = t / Lw[j * d + j];
        }
    }

done:
    if (L) memcpy(L, Lw, (size_t)(d * d) * sizeof(double));
    if (xbar_out) memcpy(xbar_out, xbar, (size_t)d * sizeof(double));
    if (S_out) memcpy(S_out, S, (size_t)(d * d) * sizeof(double));
    free(xbar); free(Xc); free(S); free(Lw);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Balance: Hotelling T^2 with whitened covariates (Sec. 2.2, Sec. 2.3):       */
/*   m1_j = mean of Zc_ij over treated i, m0_j = mean over control i          */
/*   (ascending i), Delta_j = m1_j - m0_j, M = (n1 n0 / n) * sum_j Delta_j^2. */
/* The paper's M = Delta^T Delta is this value times (1/n1 + 1/n0). Swapping   */
/* treated and control swaps m1 and m0, so when n1 = n0 an assignment and its  */
/* complement get bit-identical M.                                              */
/* ------------------------------------------------------------------------- */
double oracle_M(const double* Zc, int64_t n, int64_t d, const uint8_t* w)
{
    int64_t n1 = 0;
    for (int64_t i = 0; i < n; ++i) n1 += w[i] ? 1 : 0;
    int64_t n0 = n - n1;
    double acc = 0.0;
    for (int64_t j = 0; j < d; ++j) {
        double s1 = 0.0, s0 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (w[i]) s1 += Zc[i * d + j];
            else s0 += Zc[i * d + j];
        }
        double delta = s1 / (double)n1 - s0 / (double)n0;
        acc += delta * delta;
    }
    double scale = ((double)n1 * (double)n0) / (double)n;
    return scale * acc;
}

/* M for draws [first, first + count) of a Philox pool (seed) or, when exact != 0,
 * for enumeration ranks [first, first + count). threads <= 0: all cores. */
void oracle_balance(const double* Zc, int64_t n, int64_t d, int64_t n1, int exact, uint64_t seed,
                    uint64_t first, int64_t count, double* M_out, int threads)
{
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
    uint64_t* masks = NULL;
    if (exact) {
        masks = (uint64_t*)malloc((size_t)(count > 0 ? count : 1) * sizeof(uint64_t));
        oracle_enum_masks(n, n1, first, count, masks);
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        uint8_t* w = (uint8_t*)malloc((size_t)n);
        uint32_t* r = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
        key_pair* pairs = (key_pair*)malloc((size_t)n * sizeof(key_pair));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t b = 0; b < count; ++b) {
            if (exact) mask_to_w(masks[b], n, w);
            else assignment_with_scratch(seed, first + (uint64_t)b, n, n1, w, r, pairs);
            M_out[b] = oracle_M(Zc, n, d, w);
        }
        free(w); free(r); free(pairs);
    }
    free(masks);
}

/* M for an explicit list of draw indices (or ranks). */
void oracle_balance_list(const double* Zc, int64_t n, int64_t d, int64_t n1, int exact, uint64_t seed,
                         const uint64_t* draws, int64_t count, double* M_out, int threads)
{
#ifdef _OPENMP
    int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    (void)threads;
#endif
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        uint8_t* w = (uint8_t*)malloc((size_t)n);
        uint32_t* r = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
        key_pair* pairs = (key_pair*)malloc((size_t)n * sizeof(key_pair));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int64_t b = 0; b < count; ++b) {
            if (exact) {
                mask_to_w(oracle_mask_of_rank(n, n1, draws[b]), n, w);
            } else {
                assignment_with_scratch(seed, draws[b], n, n1, w, r, pairs);
            }
            M_out[b] = oracle_M(Zc, n, d, w);
        }
        free(w); free(r); free(pairs);
    }
}

/* ------------------------------------------------------------------------- */
/* Acceptance (Sec. 2.2: keep the best q fraction, or all M <= a). Total order */
/* (M, draw index) ascending; ties go to the lower index. q mode keeps the     */
/* first K = ceil(q B - 1e-9 q B) draws; threshold mode keeps every M <= a.    */
/* Output: accepted draw indices sorted ascending, with their M.              */
/* ------------------------------------------------------------------------- */
typedef struct { double m; uint64_t idx; } m_idx;

static int cmp_m_idx(const void* a, const void* b)
{
    const m_idx* p = (const m_idx*)a;
    const m_idx* q = (const m_idx*)b;
    if (p->m < q->m) return -1;
    if (p->m > q->m) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

int64_t oracle_k_from_q(double q, int64_t B)
{
    double qb = q * (double)B;
    double k = ceil(qb - 1e-9 * qb);
    if (k < 1.0) k = 1.0;
    if (k > (double)B) k = (double)B;
    return (int64_t)k;
}

/* Selects from the M values of draws [first, first+B) (M[b] is draw first+b).
 * Exactly one of q (0 < q <= 1) and threshold (>= 0) is used: the other is NaN.
 * Returns the number accepted; writes up to cap keys / M values. */
int64_t oracle_select_from_M(const double* M, uint64_t first, int64_t B, double q, double threshold,
                             uint64_t* keys_out, double* M_out, int64_t cap)
{
    m_idx* all = (m_idx*)malloc((size_t)(B > 0 ? B : 1) * sizeof(m_idx));
    for (int64_t b = 0; b < B; ++b) { all[b].m = M[b]; all[b].idx = first + (uint64_t)b; }
    qsort(all, (size_t)B, sizeof(m_idx), cmp_m_idx);
    int64_t K;
    if (!isnan(q)) {
        K = oracle_k_from_q(q, B);
    } else {
        K = 0;
        while (K < B && all[K].m <= threshold) ++K;
    }
    uint64_t* idx = (uint64_t*)malloc((size_t)(K > 0 ? K : 1) * sizeof(uint64_t));
    for (int64_t k = 0; k < K; ++k) idx[k] = all[k].idx;
    qsort(idx, (size_t)K, sizeof(uint64_t), cmp_u64);
    for (int64_t k = 0; k < K && k < cap; ++k) {
        keys_out[k] = idx[k];
        /* find its M (B is small enough for the oracle's purposes) */
        M_out[k] = M[idx[k] - first];
    }
    free(idx);
    free(all);
    return K;
}

/* ------------------------------------------------------------------------- */
/* Randomization test conditional on acceptance (Sec. 2.3, randomization_test;*/
/* Sec. 4 "Design-based inference"). Sharp null Y_i(1) = Y_i(0) + tau. For    */
/* each tau on the caller's grid: Yt = Y - tau * w_obs; t_k = DiM_{w_k}(Yt)   */
/* (mean over treated minus mean over control, ascending sums); count the      */
/* accepted k with |t_k| >= |t_obs| (w_obs itself included, so p >= 1/K);      */
/* p = count / K. The interval is [min, max] of the grid points with p > alpha */
/* (NaN when none). near_ties[g] counts k with ||t_k| - |t_obs|| below          */
/* 1e-12 (|t_obs| + 1): their side of the comparison is not robust to rounding.*/
/* ------------------------------------------------------------------------- */
static double dim_stat(const double* y, const uint8_t* w, int64_t n)
{
    double s1 = 0.0, s0 = 0.0;
    int64_t n1 = 0, n0 = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (w[i]) { s1 += y[i]; ++n1; }
        else { s0 += y[i]; ++n0; }
    }
    return s1 / (double)n1 - s0 / (double)n0;
}

double oracle_dim(const double* y, const uint8_t* w, int64_t n) { return dim_stat(y, w, n); }

int oracle_randtest(const uint8_t* W /* K x n accepted assignments */, int64_t K, int64_t n,
                    const uint8_t* w_obs, const double* Y, const double* tau, int64_t T, double alpha,
                    double* p_out, int64_t* count_out, int64_t* near_ties_out,
                    double* ci_lo, double* ci_hi)
{
    double* yt = (double*)malloc((size_t)n * sizeof(double));
    double lo = NAN, hi = NAN;
    for (int64_t g = 0; g < T; ++g) {
        for (int64_t i = 0; i < n; ++i) yt[i] = Y[i] - tau[g] * (double)w_obs[i];
        double t_obs = fabs(dim_stat(yt, w_obs, n));
        int64_t cnt = 0, near = 0;
        for (int64_t k = 0; k < K; ++k) {
            double t = fabs(dim_stat(yt, W + k * n, n));
            if (t >= t_obs) ++cnt;
            if (fabs(t - t_obs) < 1e-12 * (t_obs + 1.0)) ++near;
        }
        count_out[g] = cnt;
        if (near_ties_out) near_ties_out[g] = near;
        p_out[g] = (double)cnt / (double)K;
        if (p_out[g] > alpha) {
            if (isnan(lo) || tau[g] < lo) lo = tau[g];
            if (isnan(hi) || tau[g] > hi) hi = tau[g];
        }
    }
    *ci_lo = lo;
    *ci_hi = hi;
    free(yt);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Pairwise distances (Sec. 4, fast_distance): D_ij = sqrt(sum_k (x_ik - y_jk)^2) */
/* for rows x_i of X (n x d) and y_j of Y (m x d), FP32 inputs taken exactly in  */
/* FP64, differences squared and summed in ascending k. squared != 0 returns the */
/* sum itself. Y == NULL means Y = X.                                           */
/* ------------------------------------------------------------------------- */
void oracle_distance(const float* X, int64_t n, const float* Y, int64_t m, int64_t d, int squared, double* D)
{
    if (Y == NULL) { Y = X; m = n; }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < m; ++j) {
            double acc = 0.0;
            for (int64_t k = 0; k < d; ++k) {
                const double t = (double)X[i * d + k] - (double)Y[j * d + k];
                acc += t * t;
            }
            D[i * m + j] = squared ? acc : sqrt(acc);
        }
}

/* Entries (i, j) listed in pairs (count of them), same definition. */
void oracle_distance_pairs(const float* X, const float* Y, int64_t d, const int64_t* ij, int64_t count, int squared,
                           double* out)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t e = 0; e < count; ++e) {
        const float* x = X + ij[2 * e] * d;
        const float* y = Y + ij[2 * e + 1] * d;
        double acc = 0.0;
        for (int64_t k = 0; k < d; ++k) {
            const double t = (double)x[k] - (double)y[k];
            acc += t * t;
        }
        out[e] = squared ? acc : sqrt(acc);
    }
}

int oracle_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
