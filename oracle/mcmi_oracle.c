/*
 * mcmi_oracle.c -- plain, slow, FP64 CPU reference of the (MC)^2MI hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header or constant table with the CUDA path.
 *
 * What it computes (paper: Lebedev & Alexandrov, "On Advanced Monte Carlo
 * Methods for Linear Algebra on Advanced Accelerator Architectures"):
 *   - the split of Eq. 1 with the sgn(b_ii)-aware augmentation of Sec. V-C
 *     (alpha = 0 leaves B unchanged) and the Jacobi scaling of Sec. III-A /
 *     Sec. IV-A phase 2: d_i = bhat_ii, c_ij = -b_ij / d_i (j != i),
 *     s_i = ||c_i||_1 summed in CSR order;
 *   - the transition probabilities p_ij = |c_ij| / s_i (the p of Eq. 2), held
 *     as integer weights q_ij = max(1, floor(p_ij 2^31)) (0 for c_ij == 0)
 *     so that every sampled transition is an integer decision (the compact
 *     table type uses the scale 2^20 instead of 2^31, so that a row of at
 *     most six transitions fits a 32-byte record on the GPU);
 *   - the estimator of Eq. 2: N chains per row r, each starting at r with
 *     weight 1 (the empty product, j = 0 term), moving r -> s1 -> s2 ... with
 *     probability p, multiplying the weight by a/p = sign(c) s, and adding
 *     the weight to column s_j of row r at every visit; chains stop at a
 *     weight cutoff delta or a maximum length L;
 *   - phase 4 of Sec. IV (column scaling by B_1^-1) and the row filter of
 *     Sec. IV-B (keep the entries largest in magnitude).
 *
 * Readings of points the paper leaves open (each is listed with its reason in
 * the design notes): the stop rule is tested on a single-precision shadow of
 * the weight, W32 <- fl32(W32 * fl32(sign s)), before each transition, so
 * that a single-precision implementation stops at the same step; random
 * numbers are Philox4x32-10 keyed by the seed, counter (t/4, chain, row lo,
 * row hi), word t mod 4 for transition t; a row with s_i == 0 is absorbing.
 *
 * Parity pins: every exported function here is checked by the CPU test-suite
 * against something other than itself (cuRAND's host Philox, dense matrix
 * powers, path enumeration, closed forms, numpy sorting, the exact binomial
 * law).  orc_chains_from_eps follows a rule the paper does not state (that
 * of the earlier (MC)^2MI papers); it is pinned by what the rule claims: the
 * probable error of an estimate whose single-chain deviation reaches the
 * bound 1/(1 - ||C||) equals epsilon, and the walks' per-entry errors stay
 * below epsilon at least half the time.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_BAD_CSR = 2, ORC_ERR_ZERO_DIAG = 3,
       ORC_ERR_NOT_CONTRACTIVE = 4, ORC_ERR_CAPACITY = 5 };
enum { ORC_TABLE_CUMULATIVE = 0, ORC_TABLE_ALIAS = 1, ORC_TABLE_HYBRID = 2, ORC_TABLE_COMPACT = 3 };

/* Scale of the integer weights: 2^31, or 2^20 for the compact table (which */
/* samples cumulatively, like ORC_TABLE_CUMULATIVE, from the coarser q).    */
static double table_scale(int table)
{
    return table == ORC_TABLE_COMPACT ? 1048576.0 : 2147483648.0;
}

/* The hybrid table chooses per row: rows with at most ORC_HYBRID_CUM_MAX
 * transitions sample from the cumulative table, longer rows from the alias
 * table (both sample the same integer weights q, with different paths).  */
#define ORC_HYBRID_CUM_MAX 6

static int uses_alias(int table, int64_t deg)
{
    return table == ORC_TABLE_ALIAS || (table == ORC_TABLE_HYBRID && deg > ORC_HYBRID_CUM_MAX);
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of counter       */
/* words 0 and 2 with the round multipliers, outputs permuted and xored     */
/* with the key; the key is bumped by the Weyl constants between rounds.    */
/* ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ---------------------------------------------------------------------- */
/* Eq. 1 split + Jacobi scaling (Sec. III-A; Sec. IV-A phases 1-2; the      */
/* augmentation alpha*||B||_inf*sgn(b_ii) of Sec. V-C).                     */
/* ---------------------------------------------------------------------- */
int orc_split(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
              double alpha, double *d, double *s, int64_t *bad_row)
{
    double bnorm = 0.0;
    *bad_row = -1;
    if (alpha > 0.0) {
        for (int64_t i = 0; i < n; ++i) {
            double r = 0.0;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) r += fabs(val[k]);
            if (r > bnorm) bnorm = r;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        double bii = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] == i) bii = val[k];
        double di = bii;
        if (alpha > 0.0) di = bii + alpha * bnorm * (bii < 0.0 ? -1.0 : 1.0);
        if (di == 0.0) { *bad_row = i; return ORC_ERR_ZERO_DIAG; }
        double si = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            if (col[k] == i) continue;
            double c = -val[k] / di;
            si += fabs(c);
        }
        d[i] = di;
        s[i] = si;
    }
    return ORC_OK;
}

/* Integer weight of one off-diagonal entry: q = max(1, floor(|c|/s * scale)), */
/* scale = 2^31 (2^20 compact), 0 for an entry whose c is exactly zero (never */
/* sampled).                                                                */
static uint32_t weight_of(double b, double di, double si, double scale)
{
    double c = -b / di;
    if (c == 0.0) return 0u;
    double x = floor(fabs(c) / si * scale);
    uint32_t q = (uint32_t)x;
    return q < 1u ? 1u : q;
}

/* Row i's off-diagonal weights in CSR order; returns the degree.           */
static int64_t row_weights(int64_t i, const int64_t *rp, const int32_t *col, const double *val,
                           const double *d, const double *s, double scale, uint32_t *q, int32_t *cols,
                           uint8_t *neg, uint64_t *Q)
{
    int64_t m = 0;
    uint64_t tot = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (col[k] == i) continue;
        uint32_t w = s[i] > 0.0 ? weight_of(val[k], d[i], s[i], scale) : 0u;
        if (q) q[m] = w;
        if (cols) cols[m] = col[k];
        if (neg) neg[m] = (-val[k] / d[i]) < 0.0;
        tot += w;
        ++m;
    }
    *Q = tot;
    return m;
}

/* Cumulative sampler: x = floor(r Q / 2^32); the pick is the smallest m with   */
/* x < T_m, T_m = q_0 + ... + q_m.                                            */
static int64_t pick_cumulative(uint32_t r, const uint32_t *q, int64_t deg, uint64_t Q)
{
    uint64_t x = ((uint64_t)r * Q) >> 32;
    uint64_t T = 0;
    for (int64_t m = 0; m < deg; ++m) {
        T += q[m];
        if (x < T) return m;
    }
    return -1; /* unreachable when Q > 0 */
}

/* Walker/Vose alias table over the integer weights.  Bucket capacity Q,    */
/* weight of entry j is q_j * deg (so the deg buckets hold deg*Q in total).  */
/* Both work lists are stacks (last in, first out), filled in CSR order;    */
/* after each pairing the large entry is pushed back on the list its        */
/* remaining weight belongs to.                                             */
void orc_alias_build(const uint32_t *q, int64_t deg, uint64_t Q, uint32_t *prob, int32_t *alias)
{
    uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(deg > 0 ? deg : 1));
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)(deg > 0 ? deg : 1));
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)(deg > 0 ? deg : 1));
    int64_t ns = 0, nl = 0;
    for (int64_t j = 0; j < deg; ++j) {
        w[j] = (uint64_t)q[j] * (uint64_t)deg;
        if (w[j] < Q) small[ns++] = j; else large[nl++] = j;
    }
    while (ns > 0 && nl > 0) {
        int64_t a = small[--ns];
        int64_t b = large[--nl];
        prob[a] = (uint32_t)w[a];
        alias[a] = (int32_t)b;
        w[b] -= Q - w[a];
        if (w[b] < Q) small[ns++] = b; else large[nl++] = b;
    }
    while (nl > 0) { int64_t b = large[--nl]; prob[b] = (uint32_t)Q; alias[b] = (int32_t)b; }
    while (ns > 0) { int64_t a = small[--ns]; prob[a] = (uint32_t)Q; alias[a] = (int32_t)a; }
    free(w); free(small); free(large);
}

/* Alias sampler: bucket b = floor(r deg / 2^32); the low 32 bits of r*deg,   */
/* scaled to [0, Q), decide between the bucket's own entry and its alias.    */
static int64_t pick_alias(uint32_t r, int64_t deg, uint64_t Q, const uint32_t *prob, const int32_t *alias)
{
    uint64_t p = (uint64_t)r * (uint64_t)deg;
    int64_t b = (int64_t)(p >> 32);
    uint64_t y = ((p & 0xFFFFFFFFull) * Q) >> 32;
    return y < prob[b] ? b : alias[b];
}

/* Exported samplers for the CPU tests (vectorised over r).                */
void orc_pick_cumulative_many(const uint32_t *q, int64_t deg, const uint32_t *r, int64_t cnt, int64_t *out)
{
    uint64_t Q = 0;
    for (int64_t m = 0; m < deg; ++m) Q += q[m];
    for (int64_t t = 0; t < cnt; ++t) out[t] = pick_cumulative(r[t], q, deg, Q);
}

void orc_pick_alias_many(const uint32_t *prob, const int32_t *alias, int64_t deg, uint64_t Q,
                         const uint32_t *r, int64_t cnt, int64_t *out)
{
    for (int64_t t = 0; t < cnt; ++t) out[t] = pick_alias(r[t], deg, Q, prob, alias);
}

/* Per-row integer tables, for the table-parity tests.  Output per row i:    */
/* Q[i]; per off-diagonal entry (in CSR order, offsets off[i]):            */
/* q, and for the alias table prob and alias (row-local index).  table     */
/* selects the scale of q (ORC_TABLE_COMPACT: 2^20).                       */
int orc_tables_ex(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  const double *d, const double *s, int table, int64_t *off, uint64_t *Q,
                  uint32_t *q, uint32_t *prob, int32_t *alias)
{
    int64_t o = 0;
    const double scale = table_scale(table);
    for (int64_t i = 0; i < n; ++i) {
        off[i] = o;
        int64_t deg = row_weights(i, rp, col, val, d, s, scale, q + o, NULL, NULL, &Q[i]);
        if (prob && alias && deg > 0) orc_alias_build(q + o, deg, Q[i], prob + o, alias + o);
        o += deg;
    }
    off[n] = o;
    return ORC_OK;
}

int orc_tables(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
               const double *d, const double *s, int64_t *off, uint64_t *Q,
               uint32_t *q, uint32_t *prob, int32_t *alias)
{
    return orc_tables_ex(n, rp, col, val, d, s, ORC_TABLE_CUMULATIVE, off, Q, q, prob, alias);
}

/* Longest possible chain: every factor is at most fl32(max_i s_i) in        */
/* magnitude and fl32 multiplication is monotone, so no chain outlives the   */
/* product of that constant.                                               */
int64_t orc_max_walk_len(double smax, double delta, int64_t L)
{
    float f = (float)smax, w = 1.0f;
    if (!(delta > 0.0) || f >= 1.0f) return L;
    int64_t t = 0;
    while (t < L && !((double)fabsf(w) < delta)) {
        w = w * f;
        ++t;
    }
    return t;
}

/* Number of chains from the accuracy epsilon when the caller gives none.   */
/* The paper does not state the rule; this is the rule of the earlier        */
/* (MC)^2MI papers it builds on: 0.6745 is the median of |Z| for a standard  */
/* normal Z, a chain's contribution deviates by at most 1/(1 - ||C||), so    */
/* with N = (0.6745 / (eps (1 - ||C||)))^2 the probable error of the mean    */
/* of N chains is at most eps.                                               */
int64_t orc_chains_from_eps(double eps, double smax)
{
    double v = 0.6745 / (eps * (1.0 - smax));
    return (int64_t)ceil(v * v);
}

/* ---------------------------------------------------------------------- */
/* Learned proposal (an extension of the method, not in the paper): the    */
/* transition weights |c_ij| are multiplied by g_ij > 0 from a small MLP of */
/* per-edge features, and the weight update uses c_ij / p_ij with the      */
/* table's own probability p_ij = q_ij / Q_i, so the estimator of Eq. 2     */
/* stays unbiased.  The MLP is evaluated as a BF16 network: inputs, weights */
/* and hidden activations rounded to bfloat16 (nearest, ties to even),      */
/* products exact in FP32, sums in FP32 in index order, biases FP32.        */
/* Parameters (FP32), in order: W1[32][8], b1[32], W2[32][32], b2[32],      */
/* w3[32], b3.                                                              */
/* ---------------------------------------------------------------------- */
enum { MLP_IN = 8, MLP_H = 32, MLP_NPARAM = 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1 };

static float bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    u &= 0xFFFF0000u;
    memcpy(&x, &u, 4);
    return x;
}

/* g = squareplus(z) = (z + sqrt(z^2 + 4)) / 2, clamped to [1/16, 16]. */
float orc_mlp_g(const float *th, const float *feat)
{
    const float *W1 = th, *b1 = th + 256, *W2 = th + 288, *b2 = th + 1312, *w3 = th + 1344, *b3 = th + 1376;
    float x[MLP_IN], h1[MLP_H], h2[MLP_H];
    for (int k = 0; k < MLP_IN; ++k) x[k] = bf16_round(feat[k]);
    for (int o = 0; o < MLP_H; ++o) {
        float acc = b1[o];
        for (int k = 0; k < MLP_IN; ++k) acc = acc + bf16_round(W1[o * MLP_IN + k]) * x[k];
        h1[o] = bf16_round(acc > 0.0f ? acc : 0.0f);
    }
    for (int o = 0; o < MLP_H; ++o) {
        float acc = b2[o];
        for (int k = 0; k < MLP_H; ++k) acc = acc + bf16_round(W2[o * MLP_H + k]) * h1[k];
        h2[o] = bf16_round(acc > 0.0f ? acc : 0.0f);
    }
    float z = b3[0];
    for (int k = 0; k < MLP_H; ++k) z = z + bf16_round(w3[k]) * h2[k];
    float g = 0.5f * (z + sqrtf(z * z + 4.0f));
    if (g < 0.0625f) g = 0.0625f;
    if (g > 16.0f) g = 16.0f;
    return g;
}

/* Features of edge (i, j): p_ij = |c_ij|/s_i, s_i, s_j, 1/deg_i, 1/deg_j,  */
/* |d_i|/(|d_i|+|d_j|), |c_ij|/max_k|c_ik|, sign(c_ij); FP64 then FP32.     */
static void edge_features(double c, double si, double sj, int64_t degi, int64_t degj, double di, double dj,
                          double maxabs, float *f)
{
    f[0] = (float)(fabs(c) / si);
    f[1] = (float)si;
    f[2] = (float)sj;
    f[3] = (float)(1.0 / (double)degi);
    f[4] = degj > 0 ? (float)(1.0 / (double)degj) : 0.0f;
    f[5] = (float)(fabs(di) / (fabs(di) + fabs(dj)));
    f[6] = (float)(fabs(c) / maxabs);
    f[7] = c < 0.0 ? -1.0f : 1.0f;
}

static int64_t off_degree(int64_t i, const int64_t *rp, const int32_t *col)
{
    int64_t m = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) m += col[k] != i;
    return m;
}

/* Row i with a learned proposal: q_ij = max(1, floor(w_ij / sum_k w_ik 2^31))  */
/* for w_ij = |c_ij| g_ij (0 if c_ij == 0); factor f_ij = c_ij Q_i / q_ij.       */
static int64_t row_weights_learned(int64_t i, const int64_t *rp, const int32_t *col, const double *val,
                                   const double *d, const double *s, const int64_t *deg, const float *th,
                                   uint32_t *q, int32_t *cols, uint8_t *neg, double *fac, float *gout,
                                   uint64_t *Q)
{
    const double di = d[i], si = s[i];
    double maxabs = 0.0, wsum = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
        if (col[k] != i && fabs(-val[k] / di) > maxabs) maxabs = fabs(-val[k] / di);
    int64_t m = 0;
    double *w = (double *)malloc(sizeof(double) * (size_t)(rp[i + 1] - rp[i] + 1));
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (col[k] == i) continue;
        const int64_t j = col[k];
        const double c = -val[k] / di;
        float g = 0.0f;
        if (c != 0.0) {
            float f[MLP_IN];
            edge_features(c, si, s[j], deg[i], deg[j], di, d[j], maxabs, f);
            g = orc_mlp_g(th, f);
        }
        if (gout) gout[m] = g;
        w[m] = fabs(c) * (double)g;
        wsum += w[m];
        if (cols) cols[m] = (int32_t)j;
        if (neg) neg[m] = c < 0.0;
        ++m;
    }
    uint64_t tot = 0;
    for (int64_t t = 0; t < m; ++t) {
        uint32_t qq = 0;
        if (w[t] > 0.0) {
            const double x = floor(w[t] / wsum * 2147483648.0);
            qq = (uint32_t)x;
            if (qq < 1u) qq = 1u;
        }
        q[t] = qq;
        tot += qq;
    }
    m = 0;
    for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        if (col[k] == i) continue;
        const double c = -val[k] / di;
        fac[m] = q[m] > 0 ? (c * (double)tot) / (double)q[m] : 0.0;
        ++m;
    }
    free(w);
    *Q = tot;
    return m;
}

/* Learned tables of every row (for the table-parity tests): per off-diagonal */
/* entry in CSR order q, the factor f = c Q / q and g.                         */
int orc_learned_tables(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                       const double *s, const float *th, int64_t *off, uint64_t *Q, uint32_t *q, double *fac,
                       float *g)
{
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) deg[i] = off_degree(i, rp, col);
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        off[i] = o;
        o += row_weights_learned(i, rp, col, val, d, s, deg, th, q + o, NULL, NULL, fac + o, g + o, &Q[i]);
    }
    off[n] = o;
    free(deg);
    return ORC_OK;
}

/* Training edges in CSR order (diagonal slots are dummies with p = 0):      */
/* features, p_ij = |c_ij|/s_i, the target column j and the row i.           */
int orc_train_edges(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                    const double *s, float *feat, double *p, int64_t *target, int64_t *row)
{
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) deg[i] = off_degree(i, rp, col);
    for (int64_t i = 0; i < n; ++i) {
        double maxabs = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != i && fabs(-val[k] / d[i]) > maxabs) maxabs = fabs(-val[k] / d[i]);
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            row[k] = i;
            target[k] = col[k];
            const double c = col[k] == i ? 0.0 : -val[k] / d[i];
            if (c == 0.0 || !(s[i] > 0.0)) {
                for (int u = 0; u < MLP_IN; ++u) feat[8 * k + u] = 0.0f;
                p[k] = 0.0;
                continue;
            }
            edge_features(c, s[i], s[col[k]], deg[i], deg[col[k]], d[i], d[col[k]], maxabs, feat + 8 * k);
            p[k] = fabs(c) / s[i];
        }
    }
    free(deg);
    return ORC_OK;
}

/* ---------------------------------------------------------------------- */
/* Eq. 2 walks.                                                           */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const double *val;
    const double *d, *s;
    const float *theta;   /* learned proposal parameters, or NULL for p = |c|/s */
    /* derived, per row: offsets into the off-diagonal arrays */
    int64_t *off;
    uint64_t *Q;
    uint32_t *q;
    int32_t *ocol;
    uint8_t *neg;
    uint32_t *prob;
    int32_t *alias;
    double *fac;          /* learned proposal: weight factor c/p per entry */
} orc_mat;

static int mat_prepare(orc_mat *M, int table)
{
    int64_t n = M->n;
    int64_t noff = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = M->rp[i]; k < M->rp[i + 1]; ++k)
            if (M->col[k] != i) ++noff;
    size_t sz = (size_t)(noff > 0 ? noff : 1);
    M->off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    M->Q = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    M->q = (uint32_t *)malloc(sizeof(uint32_t) * sz);
    M->ocol = (int32_t *)malloc(sizeof(int32_t) * sz);
    M->neg = (uint8_t *)malloc(sz);
    M->prob = table != ORC_TABLE_CUMULATIVE ? (uint32_t *)malloc(sizeof(uint32_t) * sz) : NULL;
    M->alias = table != ORC_TABLE_CUMULATIVE ? (int32_t *)malloc(sizeof(int32_t) * sz) : NULL;
    M->fac = M->theta ? (double *)malloc(sizeof(double) * sz) : NULL;
    int64_t *degs = NULL;
    if (M->theta) {
        degs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t i = 0; i < n; ++i) degs[i] = off_degree(i, M->rp, M->col);
    }
    int64_t o = 0;
    for (int64_t i = 0; i < n; ++i) {
        M->off[i] = o;
        int64_t deg = M->theta
                          ? row_weights_learned(i, M->rp, M->col, M->val, M->d, M->s, degs, M->theta, M->q + o,
                                                M->ocol + o, M->neg + o, M->fac + o, NULL, &M->Q[i])
                          : row_weights(i, M->rp, M->col, M->val, M->d, M->s, table_scale(table), M->q + o,
                                        M->ocol + o, M->neg + o,
                                        &M->Q[i]);
        if (uses_alias(table, deg) && deg > 0)
            orc_alias_build(M->q + o, deg, M->Q[i], M->prob + o, M->alias + o);
        o += deg;
    }
    M->off[n] = o;
    free(degs);
    return ORC_OK;
}

static void mat_release(orc_mat *M)
{
    free(M->off); free(M->Q); free(M->q); free(M->ocol); free(M->neg);
    free(M->prob); free(M->alias); free(M->fac);
}

typedef struct {
    double *X, *A;
    uint32_t *V;
    int64_t *touched;
    int64_t ntouched;
} orc_acc;

static void acc_add(orc_acc *a, int64_t j, double w)
{
    if (a->V[j] == 0) a->touched[a->ntouched++] = j;
    a->X[j] += w;
    a->A[j] += fabs(w);
    a->V[j] += 1;
}

static int cmp_i64(const void *x, const void *y)
{
    int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
    return (a > b) - (a < b);
}

/* All N chains of row i (Eq. 2); fills the accumulator, returns transitions. */
static uint64_t walk_row(const orc_mat *M, int table, int64_t i, int64_t N, int64_t L,
                         double delta, uint64_t seed, orc_acc *acc)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint64_t steps = 0;
    for (int64_t k = 0; k < N; ++k) {
        int64_t state = i;
        double w = 1.0;
        float w32 = 1.0f;
        uint32_t r4[4] = {0, 0, 0, 0};
        int64_t t = 0;
        acc_add(acc, state, w);
        for (;;) {
            if (t == L) break;
            if ((double)fabsf(w32) < delta) break;
            if (M->Q[state] == 0) break;
            if (t % 4 == 0) {
                uint32_t ctr[4] = {(uint32_t)(t / 4), (uint32_t)k, (uint32_t)i, (uint32_t)((uint64_t)i >> 32)};
                orc_philox4x32_10(ctr, key, r4);
            }
            uint32_t r = r4[t % 4];
            int64_t o = M->off[state], deg = M->off[state + 1] - o;
            int64_t m = uses_alias(table, deg)
                            ? pick_alias(r, deg, M->Q[state], M->prob + o, M->alias + o)
                            : pick_cumulative(r, M->q + o, deg, M->Q[state]);
            if (M->fac) {
                /* learned proposal: W <- W c/p with the table's probability */
                const double f = M->fac[o + m];
                w = w * f;
                w32 = w32 * (float)f;
            } else {
                double sj = M->s[state];
                int negative = M->neg[o + m];
                w = w * (negative ? -sj : sj);
                float f32 = (float)sj;
                w32 = w32 * (negative ? -f32 : f32);
            }
            state = M->ocol[o + m];
            ++t;
            acc_add(acc, state, w);
        }
        steps += (uint64_t)t;
    }
    return steps;
}

static int acc_alloc(orc_acc *a, int64_t n)
{
    a->X = (double *)calloc((size_t)n, sizeof(double));
    a->A = (double *)calloc((size_t)n, sizeof(double));
    a->V = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    a->touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    a->ntouched = 0;
    return a->X && a->A && a->V && a->touched ? 0 : -1;
}

static void acc_reset(orc_acc *a)
{
    for (int64_t t = 0; t < a->ntouched; ++t) {
        int64_t j = a->touched[t];
        a->X[j] = 0.0; a->A[j] = 0.0; a->V[j] = 0;
    }
    a->ntouched = 0;
}

static void acc_free(orc_acc *a) { free(a->X); free(a->A); free(a->V); free(a->touched); }

static void set_threads(int threads)
{
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
}

/* Second moment of each listed row's chains, m_i = (1/N) sum_chains       */
/* sum_t W_t^2 (the weights of Eq. 2 along each path, t = 0 included): the  */
/* training signal of the learned proposal, whose variance-optimal one-step */
/* choice is p_ij proportional to |c_ij| sqrt(m_j).                          */
int orc_row_moments(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *d,
                    const double *s, int table, const int64_t *rows, int64_t nrows, int64_t N, int64_t L,
                    double delta, uint64_t seed, int threads, double *m_out, const float *theta)
{
    orc_mat M = {n, rp, col, val, d, s, theta};
    mat_prepare(&M, table);
    set_threads(threads);
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < nrows; ++p) {
        const int64_t i = rows[p];
        double sum = 0.0;
        for (int64_t k = 0; k < N; ++k) {
            int64_t state = i, t = 0;
            double w = 1.0;
            float w32 = 1.0f;
            uint32_t r4[4] = {0, 0, 0, 0};
            sum += w * w;
            while (t != L && !((double)fabsf(w32) < delta) && M.Q[state] != 0) {
                if (t % 4 == 0) {
                    uint32_t ctr[4] = {(uint32_t)(t / 4), (uint32_t)k, (uint32_t)i, (uint32_t)((uint64_t)i >> 32)};
                    orc_philox4x32_10(ctr, key, r4);
                }
                const int64_t o = M.off[state], deg = M.off[state + 1] - o;
                const int64_t m = uses_alias(table, deg)
                                      ? pick_alias(r4[t % 4], deg, M.Q[state], M.prob + o, M.alias + o)
                                      : pick_cumulative(r4[t % 4], M.q + o, deg, M.Q[state]);
                double f;
                if (M.fac) {
                    f = M.fac[o + m];
                } else {
                    f = M.neg[o + m] ? -M.s[state] : M.s[state];
                }
                w = w * f;
                w32 = w32 * (M.fac ? (float)f : (M.neg[o + m] ? -(float)M.s[state] : (float)M.s[state]));
                state = M.ocol[o + m];
                ++t;
                sum += w * w;
            }
        }
        m_out[p] = sum / (double)N;
    }
    mat_release(&M);
    return ORC_OK;
}

/* Raw accumulators of the listed rows: for row r (position p in rows[]),    */
/* entries p*cap .. p*cap+count[p]-1 hold (column, X/N, A/N, V) sorted by    */
/* column, where A is the sum of |W| (the scale used to judge cancellation). */
int orc_walk_rows(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  const double *d, const double *s, int table, const int64_t *rows, int64_t nrows,
                  int64_t N, int64_t L, double delta, uint64_t seed, int64_t cap, int threads,
                  int64_t *count, uint64_t *steps, int32_t *ocol, double *oX, double *oA, uint32_t *oV,
                  const float *theta)
{
    orc_mat M = {n, rp, col, val, d, s, theta};
    mat_prepare(&M, table);
    int status = ORC_OK;
    set_threads(threads);
#pragma omp parallel
    {
        orc_acc acc;
        acc_alloc(&acc, n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < nrows; ++p) {
            int64_t i = rows[p];
            steps[p] = walk_row(&M, table, i, N, L, delta, seed, &acc);
            qsort(acc.touched, (size_t)acc.ntouched, sizeof(int64_t), cmp_i64);
            if (acc.ntouched > cap) {
#pragma omp atomic write
                status = ORC_ERR_CAPACITY;
                count[p] = -1;
            } else {
                count[p] = acc.ntouched;
                for (int64_t t = 0; t < acc.ntouched; ++t) {
                    int64_t j = acc.touched[t];
                    ocol[p * cap + t] = (int32_t)j;
                    oX[p * cap + t] = acc.X[j] / (double)N;
                    oA[p * cap + t] = acc.A[j] / (double)N;
                    oV[p * cap + t] = acc.V[j];
                }
            }
            acc_reset(&acc);
        }
        acc_free(&acc);
    }
    mat_release(&M);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Phase 4 (column scaling by B_1^-1, Sec. IV-A) and the filter of Sec. IV-B. */
/* ---------------------------------------------------------------------- */
typedef struct { double mag; int64_t j; } orc_cand;

static int cmp_cand(const void *x, const void *y)
{
    const orc_cand *a = (const orc_cand *)x, *b = (const orc_cand *)y;
    if (a->mag > b->mag) return -1;
    if (a->mag < b->mag) return 1;
    return (a->j > b->j) - (a->j < b->j);
}

/* Filter one row given its column-scaled entries M_j (sorted by column).   */
/* Keeps the diagonal; off-diagonals with |M_j| >= tau * max|M| (tau > 0);  */
/* of those, the top_k largest in magnitude, ties to the smaller column.    */
int64_t orc_filter_row(int64_t i, const int32_t *cols, const double *m, int64_t cnt,
                       double tau, int64_t top_k, int32_t *out_col, double *out_val)
{
    double rowmax = 0.0;
    for (int64_t t = 0; t < cnt; ++t) if (fabs(m[t]) > rowmax) rowmax = fabs(m[t]);
    orc_cand *c = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)(cnt > 0 ? cnt : 1));
    int64_t nc = 0;
    for (int64_t t = 0; t < cnt; ++t) {
        if (cols[t] == i) continue;
        if (tau > 0.0 && !(fabs(m[t]) >= tau * rowmax)) continue;
        c[nc].mag = fabs(m[t]);
        c[nc].j = cols[t];
        ++nc;
    }
    if (top_k > 0 && nc > top_k) {
        /* rank by magnitude (descending), then column (ascending) */
        qsort(c, (size_t)nc, sizeof(orc_cand), cmp_cand);
        nc = top_k;
    }
    /* kept columns plus the diagonal, emitted in column order */
    int64_t *keep = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    int64_t nk = 0;
    for (int64_t u = 0; u < nc; ++u) keep[nk++] = c[u].j;
    for (int64_t t = 0; t < cnt; ++t) if (cols[t] == i) { keep[nk++] = i; break; }
    qsort(keep, (size_t)nk, sizeof(int64_t), cmp_i64);
    int64_t t = 0;
    for (int64_t u = 0; u < nk; ++u) {
        while (cols[t] != keep[u]) ++t;
        out_col[u] = cols[t];
        out_val[u] = m[t];
    }
    free(c); free(keep);
    return nk;
}

/* Whole preconditioner rows: walk (Eq. 2), scale column j by 1/d_j, filter. */
int orc_build_rows(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                   const double *d, const double *s, int table, const int64_t *rows, int64_t nrows,
                   int64_t N, int64_t L, double delta, uint64_t seed, double tau, int64_t top_k,
                   int64_t cap, int threads, int64_t *count, uint64_t *steps,
                   int32_t *out_col, double *out_val, const float *theta)
{
    orc_mat M = {n, rp, col, val, d, s, theta};
    mat_prepare(&M, table);
    int status = ORC_OK;
    set_threads(threads);
#pragma omp parallel
    {
        orc_acc acc;
        acc_alloc(&acc, n);
        int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        double *m = (double *)malloc(sizeof(double) * (size_t)n);
        int32_t *kc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        double *kv = (double *)malloc(sizeof(double) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (int64_t p = 0; p < nrows; ++p) {
            int64_t i = rows[p];
            steps[p] = walk_row(&M, table, i, N, L, delta, seed, &acc);
            qsort(acc.touched, (size_t)acc.ntouched, sizeof(int64_t), cmp_i64);
            for (int64_t t = 0; t < acc.ntouched; ++t) {
                int64_t j = acc.touched[t];
                cols[t] = (int32_t)j;
                m[t] = (acc.X[j] / (double)N) / d[j];
            }
            int64_t nk = orc_filter_row(i, cols, m, acc.ntouched, tau, top_k, kc, kv);
            if (nk > cap) {
#pragma omp atomic write
                status = ORC_ERR_CAPACITY;
                count[p] = -1;
            } else {
                count[p] = nk;
                memcpy(out_col + p * cap, kc, sizeof(int32_t) * (size_t)nk);
                memcpy(out_val + p * cap, kv, sizeof(double) * (size_t)nk);
            }
            acc_reset(&acc);
        }
        acc_free(&acc);
        free(cols); free(m); free(kc); free(kv);
    }
    mat_release(&M);
    return status;
}

/* y = M x for a CSR M (the preconditioner applied as in Sec. III-A's use).  */
void orc_spmv(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
              const double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) acc += val[k] * x[col[k]];
        y[i] = acc;
    }
}

/* ------------------------------------------------------------------------
 * Matrix reduction (Algorithm 1, step 2; Sec. III, "Matrix Reduction"):
 * before the split, drop a set share of the smallest (in magnitude) entries
 * of B.  Only off-diagonal entries are dropped (the split needs b_ii).
 *   mode 0, share of the entries: the k = floor(fraction * nnz_off)
 *     off-diagonal entries smallest in |b_ij|, ties broken by position in
 *     CSR order (the earlier entry is dropped first);
 *   mode 1, share of the value range (the experiments' "% of the value
 *     range of the entries removed"): the off-diagonal entries with
 *     |b_ij| < lo + fraction (hi - lo), lo and hi the smallest and largest
 *     off-diagonal |b_ij|, evaluated in FP64 in that order.
 * keep[k] is set to 1 for kept stored entries and 0 for dropped ones; the
 * return value is the number dropped (-1 on a bad argument).
 * ------------------------------------------------------------------------ */
typedef struct {
    double a;
    int64_t k;
} orc_absidx;

static int cmp_absidx(const void *x, const void *y)
{
    const orc_absidx *p = (const orc_absidx *)x, *q = (const orc_absidx *)y;
    if (p->a < q->a) return -1;
    if (p->a > q->a) return 1;
    return (p->k > q->k) - (p->k < q->k);
}

int64_t orc_reduce_mask(int64_t n, const int64_t *rp, const int32_t *col, const double *val, double fraction,
                        int mode, uint8_t *keep)
{
    if (!(fraction >= 0.0 && fraction <= 1.0) || (mode != 0 && mode != 1)) return -1;
    const int64_t nnz = rp[n];
    int64_t noff = 0;
    for (int64_t k = 0; k < nnz; ++k) keep[k] = 1;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != i) ++noff;
    if (noff == 0) return 0;
    int64_t dropped = 0;
    if (mode == 1) {
        double lo = INFINITY, hi = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
                if (col[k] != i) {
                    const double a = fabs(val[k]);
                    if (a < lo) lo = a;
                    if (a > hi) hi = a;
                }
        const double thr = lo + fraction * (hi - lo);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
                if (col[k] != i && fabs(val[k]) < thr) {
                    keep[k] = 0;
                    ++dropped;
                }
        return dropped;
    }
    const int64_t kdrop = (int64_t)floor(fraction * (double)noff);
    orc_absidx *e = (orc_absidx *)malloc((size_t)noff * sizeof(orc_absidx));
    if (!e) return -1;
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            if (col[k] != i) {
                e[m].a = fabs(val[k]);
                e[m].k = k;
                ++m;
            }
    qsort(e, (size_t)noff, sizeof(orc_absidx), cmp_absidx);
    for (int64_t t = 0; t < kdrop; ++t) keep[e[t].k] = 0;
    free(e);
    return kdrop;
}

/* ------------------------------------------------------------------------
 * Recovery of B^-1 from Bhat^-1 (Eq. 3; Algorithm 1, step 5): with
 * S = Bhat - B, which is zero except on the diagonal, s_i = alpha ||B||_inf
 * sgn(b_ii), apply for k = n-1, ..., 0 (the paper's S_{k+1}, row i = k here)
 *   X <- X + s_i X e_i e_i^T X / (1 - s_i X_ii),
 * a rank-one update by column i and row i of the current X.  X is the dense
 * n x n row-major Bhat^-1 (or an approximation of it) and is overwritten by
 * the recovered B^-1.  s: the n diagonal entries of S.  Returns 0, or -1 if
 * a denominator is zero.  O(n^3): a diagnostic for small n.
 * ------------------------------------------------------------------------ */
int orc_recover_dense(int64_t n, const double *s, double *X)
{
    double *c = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    if (!c || !r) {
        free(c);
        free(r);
        return -1;
    }
    int status = 0;
    for (int64_t i = n - 1; i >= 0 && status == 0; --i) {
        if (s[i] == 0.0) continue;
        const double den = 1.0 - s[i] * X[i * n + i];
        if (den == 0.0) {
            status = -1;
            break;
        }
        const double g = s[i] / den;
        for (int64_t a = 0; a < n; ++a) {
            c[a] = X[a * n + i];
            r[a] = X[i * n + a];
        }
        for (int64_t a = 0; a < n; ++a)
            for (int64_t b = 0; b < n; ++b) X[a * n + b] += g * c[a] * r[b];
    }
    free(c);
    free(r);
    return status;
}
