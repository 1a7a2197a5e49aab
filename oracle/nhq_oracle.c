/*
 * nhq_oracle.c -- plain, slow, serial CPU oracle of the NHQ hybrid-query path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; it is compiled with
 * -ffp-contract=off so every float operation below is one IEEE rounding.
 *
 * What it computes (paper: arXiv 2203.13601):
 *   Eq. 1        Euclidean distance delta                    or_delta64 / or_delta32
 *   Eq. 4-5      attribute distance chi (mismatch count)     or_chi
 *   Eq. 6        fusion distance Gamma = w_v*delta + w_l*chi or_gamma64 / or_gamma32
 *   Sec. 3.2     recommended weights w_v = 1, w_l = delta/m  (mode OR_W_PROPORTIONAL)
 *   Sec. 6.5     curves i/ii: w_v = chi/(delta+chi), w_l = delta/(delta+chi), i.e.
 *                the harmonic mean 2 delta chi / (delta + chi), with chi replaced by
 *                1 (chi = 0) or c * chi (chi > 0) for curve ii   (mode OR_W_HARMONIC,
 *                c = wl; wl = 0 is curve i)
 *   Def. 2, 4    exact top-k by Gamma (brute force)          or_fused_topk
 *   Sec. 6.1     hybrid ground truth (exact attribute match,
 *                k nearest by delta)                         or_filtered_topk
 *   Sec. 4.1     candidate set for edge selection: the exact
 *                K nearest by Gamma                          or_knn
 *   Sec. 4.1     landing-zone edge selection, Def. 6         or_edge_select
 *   (reading)    reverse-edge candidates for a second pass   or_reverse_candidates
 *   Alg. 2       joint pruning (ef-bounded best-first search)
 *   Sec. 4.2/5.2 two-stage "random TOGG" routing             or_search
 *   Eq. 7        graph quality Q_G                           or_graph_quality
 *
 * Precision: prec = OR_F64 computes delta in double (the truth used for error
 * statements); prec = OR_F32 is the "canonical f32" form in which the kernels
 * take their ordering decisions: squared differences summed in index order in
 * float, sqrtf, then Eq. 6 as separately rounded float operations.  Ordering is
 * always lexicographic by (Gamma, id).
 *
 * Readings where the paper is silent or ambiguous are the ones listed in the
 * design notes: ef-bounded pool for Alg. 2, splitmix64-derived seeds and S1
 * neighbour subsets, "local optimum" = an expansion that leaves the pool's
 * membership unchanged, strict inequalities in the landing-zone test.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_W_PROPORTIONAL 0
#define OR_W_CONSTANT 1
#define OR_W_HARMONIC 3
#define OR_F64 0
#define OR_F32 1

#define OR_OK 0
#define OR_ITER_LIMIT 4

/* ------------------------------------------------------------------ */
/* splitmix64 (S. Vigna's published generator): state advances by the  */
/* golden-ratio increment and each output is the mix64 finaliser.      */
/* ------------------------------------------------------------------ */
static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* j-th output (j = 0, 1, ...) of a splitmix64 stream whose state starts at s0 */
uint64_t or_splitmix64_at(uint64_t s0, uint64_t j)
{
    return or_mix64(s0 + (j + 1) * SM_GAMMA);
}

/* ------------------------------------------------------------------ */
/* Distances                                                          */
/* ------------------------------------------------------------------ */

/* Eq. 1 in double */
double or_delta64(const float *x, const float *y, int d)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = (double)x[i] - (double)y[i];
        s += t * t;
    }
    return sqrt(s);
}

/* Eq. 1 in float, summed in index order */
/* delta^2 in float, summed in index order (no square root) */
float or_dist2_32(const float *x, const float *y, int d)
{
    float s = 0.0f;
    for (int i = 0; i < d; ++i) {
        float t = x[i] - y[i];
        float t2 = t * t;
        s = s + t2;
    }
    return s;
}

float or_delta32(const float *x, const float *y, int d)
{
    float s = 0.0f;
    for (int i = 0; i < d; ++i) {
        float t = x[i] - y[i];
        float t2 = t * t;
        s = s + t2;
    }
    return sqrtf(s);
}

/* Eq. 4-5: number of attribute positions whose codes differ */
int or_chi(const uint8_t *a, const uint8_t *b, int m)
{
    int c = 0;
    for (int i = 0; i < m; ++i)
        c += (a[i] != b[i]) ? 1 : 0;
    return c;
}

/* chi of a query (codes qa) against an object (codes a) when a query code equal to
 * `wild` places no constraint on its position (a partial constraint, which the paper
 * does not define): such positions never count.  wild < 0: every position counts,
 * as or_chi. */
int or_chi_query(const uint8_t *qa, const uint8_t *a, int m, int wild)
{
    int c = 0;
    for (int i = 0; i < m; ++i)
        c += (qa[i] != a[i] && (int)qa[i] != wild) ? 1 : 0;
    return c;
}

/* whether the query leaves some position open */
static int or_query_open(const uint8_t *qa, int m, int wild)
{
    for (int i = 0; i < m; ++i)
        if ((int)qa[i] == wild)
            return 1;
    return 0;
}

/* Reduced-precision copies used for scoring (a project addition, not in the
 * paper): each object component rounded to nearest, ties to even.
 *   bf16      : 8 significant bits (the upper half of the f32 encoding)
 *   fp8 e4m3  : 4 exponent bits (bias 7), 3 mantissa bits, subnormals down to
 *               2^-9, largest finite 448; magnitudes beyond saturate to 448 */
float or_round_bf16(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

float or_round_e4m3(float x)
{
    double a = fabs((double)x);
    if (a == 0.0)
        return x;
    int e;
    frexp(a, &e);          /* a = f * 2^e with f in [0.5, 1): leading bit 2^(e-1) */
    int lead = e - 1;
    if (lead < -6)
        lead = -6;         /* subnormal range shares the quantum of 2^-6 normals */
    double quantum = ldexp(1.0, lead - 3);
    double r = nearbyint(a / quantum) * quantum;  /* default rounding: to nearest even */
    if (r > 448.0)
        r = 448.0;
    return (float)(x < 0 ? -r : r);
}

/* IEEE binary16: 11 significant bits for magnitudes from 2^-14, subnormals with the
 * quantum 2^-24 below that, largest finite 65504; rounding to nearest even, and magnitudes
 * at or above 65520 (halfway to the next binade's first value) round to infinity. */
float or_round_f16(float x)
{
    double a = fabs((double)x);
    if (a == 0.0 || isnan(x))
        return x;
    if (a >= 65520.0)
        return x < 0 ? -INFINITY : INFINITY;
    int e;
    frexp(a, &e);          /* leading bit 2^(e-1) */
    int lead = e - 1;
    if (lead < -14)
        lead = -14;        /* subnormals share the quantum of the smallest normals */
    double quantum = ldexp(1.0, lead - 10);
    double r = nearbyint(a / quantum) * quantum;
    return (float)(x < 0 ? -r : r);
}

/* Rounds n values in place: mode 1 bf16, mode 2 fp8 e4m3, mode 3 f16 (the functions above). */
void or_round_rows(float *x, int64_t n, int mode)
{
    for (int64_t i = 0; i < n; ++i)
        x[i] = mode == 1 ? or_round_bf16(x[i]) : mode == 2 ? or_round_e4m3(x[i])
                                                           : or_round_f16(x[i]);
}

/* Eq. 6 in double.  Proportional mode: w_v = 1, w_l = delta / m (Sec. 3.2). */
double or_gamma64(double delta, int chi, int m, int mode, double wv, double wl)
{
    if (mode == OR_W_HARMONIC) {
        /* the attribute term of the harmonic mean: chi itself (curve i), or the adjusted
         * value 1 for chi = 0 and c * chi otherwise (curve ii, c = wl) */
        double h = wl > 0.0 ? (chi == 0 ? 1.0 : wl * (double)chi) : (double)chi;
        double den = delta + h;
        return den == 0.0 ? 0.0 : 2.0 * delta * h / den;
    }
    if (mode == OR_W_PROPORTIONAL) {
        double w_l = delta / (double)m;
        return 1.0 * delta + w_l * (double)chi;
    }
    return wv * delta + wl * (double)chi;
}

/* Eq. 6 in float, each operation rounded once */
float or_gamma32(float delta, int chi, int m, int mode, float wv, float wl)
{
    if (mode == OR_W_HARMONIC) {
        float h = wl > 0.f ? (chi == 0 ? 1.f : wl * (float)chi) : (float)chi;
        float two_d = 2.f * delta;
        float num = two_d * h;
        float den = delta + h;
        return den == 0.f ? 0.f : num / den;
    }
    if (mode == OR_W_PROPORTIONAL) {
        float w_l = delta / (float)m;
        float t = w_l * (float)chi;
        return delta + t;
    }
    float a = wv * delta;
    float b = wl * (float)chi;
    return a + b;
}

/* Gamma between row x (attrs ax) and row y (attrs ay) in the chosen precision */
/* (wild: the query wildcard code when x is a query, else -1) */
static double pair_gamma(const float *x, const uint8_t *ax, const float *y, const uint8_t *ay,
                         int d, int m, int mode, double wv, double wl, int prec, int *chi_out,
                         int wild)
{
    int chi = or_chi_query(ax, ay, m, wild);
    if (chi_out)
        *chi_out = chi;
    if (prec == OR_F32)
        return (double)or_gamma32(or_delta32(x, y, d), chi, m, mode, (float)wv, (float)wl);
    return or_gamma64(or_delta64(x, y, d), chi, m, mode, wv, wl);
}

/* ------------------------------------------------------------------ */
/* (Gamma, id) records and their lexicographic order                  */
/* ------------------------------------------------------------------ */
typedef struct {
    double g;
    int64_t id;
    int32_t chi;
} rec_t;

static int rec_cmp(const void *pa, const void *pb)
{
    const rec_t *a = (const rec_t *)pa, *b = (const rec_t *)pb;
    if (a->g < b->g) return -1;
    if (a->g > b->g) return 1;
    if (a->id < b->id) return -1;
    if (a->id > b->id) return 1;
    return 0;
}

static int rec_less(double ga, int64_t ia, double gb, int64_t ib)
{
    return ga < gb || (ga == gb && ia < ib);
}

/* ------------------------------------------------------------------ */
/* Def. 2 with Gamma in place of delta: exact top-k by (Gamma, id).    */
/* Unfilled slots (k > N) get id -1 and Gamma +inf.                    */
/* ------------------------------------------------------------------ */
void or_fused_topk(const float *X, const uint8_t *A, int64_t N, int d, int m,
                   const float *Qv, const uint8_t *QA, int64_t nq, int k,
                   int mode, double wv, double wl, int prec,
                   int64_t *out_ids, double *out_g, int32_t *out_chi, int wild)
{
    rec_t *all = (rec_t *)malloc(sizeof(rec_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t q = 0; q < nq; ++q) {
        const float *qv = Qv + q * (int64_t)d;
        const uint8_t *qa = QA + q * (int64_t)m;
        for (int64_t v = 0; v < N; ++v) {
            int chi;
            all[v].g = pair_gamma(qv, qa, X + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                  mode, wv, wl, prec, &chi, wild);
            all[v].id = v;
            all[v].chi = chi;
        }
        qsort(all, (size_t)N, sizeof(rec_t), rec_cmp);
        for (int j = 0; j < k; ++j) {
            int64_t o = q * (int64_t)k + j;
            if (j < N) {
                out_ids[o] = all[j].id;
                out_g[o] = all[j].g;
                out_chi[o] = all[j].chi;
            } else {
                out_ids[o] = -1;
                out_g[o] = INFINITY;
                out_chi[o] = -1;
            }
        }
    }
    free(all);
}

/* Sec. 6.1: hybrid ground truth G = the k nearest by delta among the objects
 * whose attributes all equal the query's (chi = 0); out_P[q] = |P|. */
void or_filtered_topk(const float *X, const uint8_t *A, int64_t N, int d, int m,
                      const float *Qv, const uint8_t *QA, int64_t nq, int k, int prec,
                      int64_t *out_ids, double *out_delta, int64_t *out_P, int wild)
{
    rec_t *all = (rec_t *)malloc(sizeof(rec_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t q = 0; q < nq; ++q) {
        const float *qv = Qv + q * (int64_t)d;
        const uint8_t *qa = QA + q * (int64_t)m;
        int64_t n = 0;
        for (int64_t v = 0; v < N; ++v) {
            if (or_chi_query(qa, A + v * (int64_t)m, m, wild) != 0)
                continue;
            const float *x = X + v * (int64_t)d;
            all[n].g = prec == OR_F32 ? (double)or_delta32(qv, x, d) : or_delta64(qv, x, d);
            all[n].id = v;
            all[n].chi = 0;
            ++n;
        }
        qsort(all, (size_t)n, sizeof(rec_t), rec_cmp);
        out_P[q] = n;
        for (int j = 0; j < k; ++j) {
            int64_t o = q * (int64_t)k + j;
            out_ids[o] = j < n ? all[j].id : -1;
            out_delta[o] = j < n ? all[j].g : INFINITY;
        }
    }
    free(all);
}

/* Candidate set C(u) of Sec. 4.1 taken as the exact K nearest v != u by
 * (Gamma, id).  rows == NULL means every row 0..N-1 (then nrows must be N). */
void or_knn(const float *X, const uint8_t *A, int64_t N, int d, int m, int K,
            int mode, double wv, double wl, int prec,
            const int64_t *rows, int64_t nrows, int64_t *out_ids, double *out_g)
{
    rec_t *all = (rec_t *)malloc(sizeof(rec_t) * (size_t)(N > 0 ? N : 1));
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t u = rows ? rows[r] : r;
        int64_t n = 0;
        for (int64_t v = 0; v < N; ++v) {
            if (v == u)
                continue;
            all[n].g = pair_gamma(X + u * (int64_t)d, A + u * (int64_t)m, X + v * (int64_t)d,
                                  A + v * (int64_t)m, d, m, mode, wv, wl, prec, NULL, -1);
            all[n].id = v;
            ++n;
        }
        qsort(all, (size_t)n, sizeof(rec_t), rec_cmp);
        for (int j = 0; j < K; ++j) {
            out_ids[r * (int64_t)K + j] = j < n ? all[j].id : -1;
            out_g[r * (int64_t)K + j] = j < n ? all[j].g : INFINITY;
        }
    }
    free(all);
}

/* ------------------------------------------------------------------ */
/* Sec. 4.1 edge selection with the landing zone of Def. 6.           */
/*   (1) candidates C(u) (ids < 0, u itself and repeats are dropped)  */
/*   (2) sort C(u) ascending by (Gamma(p,u), id); the nearest becomes  */
/*       the first neighbour                                           */
/*   (3) each next p joins N(u) iff for every j in N(u) it lies in     */
/*       L(u, j) = H(u, j) \ B(u, Gamma(u, j)):                        */
/*         Gamma(p, u) < Gamma(p, j)   (u's side of the bisector)      */
/*         Gamma(p, u) > Gamma(u, j)   (outside the ball)              */
/*       until |N(u)| = R.  Unused slots get -1.                       */
/* Gamma plays the role of delta for the composite index (Sec. 5.1).  */
/* rows == NULL: every vertex u = 0..N-1 with cand row u (nrows = N); */
/* otherwise vertex rows[r] with cand row r, output row r.            */
/* ------------------------------------------------------------------ */
void or_edge_select(const float *X, const uint8_t *A, int64_t N, int d, int m,
                    const int64_t *cand, int K, int R, int mode, double wv, double wl, int prec,
                    const int64_t *rows, int64_t nrows, int64_t *out_nbr, int32_t *out_deg)
{
    rec_t *c = (rec_t *)malloc(sizeof(rec_t) * (size_t)(K > 0 ? K : 1));
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t u = rows ? rows[r] : r;
        const float *xu = X + u * (int64_t)d;
        const uint8_t *au = A + u * (int64_t)m;
        int n = 0;
        for (int j = 0; j < K; ++j) {
            int64_t p = cand[r * (int64_t)K + j];
            if (p < 0 || p >= N || p == u)
                continue;
            int dup = 0;
            for (int t = 0; t < n; ++t)
                if (c[t].id == p)
                    dup = 1;
            if (dup)
                continue;
            c[n].g = pair_gamma(X + p * (int64_t)d, A + p * (int64_t)m, xu, au, d, m, mode, wv,
                                wl, prec, NULL, -1);
            c[n].id = p;
            ++n;
        }
        qsort(c, (size_t)n, sizeof(rec_t), rec_cmp);
        int64_t *nb = out_nbr + r * (int64_t)R;
        double *nbg = (double *)malloc(sizeof(double) * (size_t)(R > 0 ? R : 1));
        int deg = 0;
        for (int t = 0; t < n && deg < R; ++t) {
            int64_t p = c[t].id;
            int ok = 1;
            for (int s = 0; s < deg && ok; ++s) {
                int64_t j = nb[s];
                double gpj = pair_gamma(X + p * (int64_t)d, A + p * (int64_t)m,
                                        X + j * (int64_t)d, A + j * (int64_t)m, d, m, mode,
                                        wv, wl, prec, NULL, -1);
                if (!(c[t].g < gpj && c[t].g > nbg[s]))
                    ok = 0;
            }
            if (ok) {
                nb[deg] = p;
                nbg[deg] = c[t].g;
                ++deg;
            }
        }
        for (int s = deg; s < R; ++s)
            nb[s] = -1;
        out_deg[r] = deg;
        free(nbg);
    }
    free(c);
}

/* Reverse-edge candidates (the paper is silent on reverse edges; this is the
 * stated reading used by the second selection pass): for every v,
 *   out[v] = N(v) (its selected neighbours, in slot order), followed by the
 *            sources u with v in N(u) that are not already in N(v), taking the
 *            `cap` smallest such ids in ascending order; -1 pads the row.
 * Row width is R + cap.  The second pass runs or_edge_select on these rows.
 * rows == NULL: every v = 0..N-1 (nrows = N); otherwise vertex rows[r] -> out row r. */
void or_reverse_candidates(const int64_t *nbr, int64_t N, int R, int cap,
                           const int64_t *rows, int64_t nrows, int64_t *out)
{
    int W = R + cap;
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t v = rows ? rows[r] : r;
        int64_t *row = out + r * (int64_t)W;
        int n = 0;
        for (int s = 0; s < R; ++s)
            if (nbr[v * (int64_t)R + s] >= 0)
                row[n++] = nbr[v * (int64_t)R + s];
        int taken = 0;
        /* ascending scan over u gives ascending source ids */
        for (int64_t u = 0; u < N && taken < cap; ++u) {
            int links = 0;
            for (int s = 0; s < R; ++s)
                if (nbr[u * (int64_t)R + s] == v)
                    links = 1;
            if (!links)
                continue;
            int dup = 0;
            for (int t = 0; t < n; ++t)
                if (row[t] == u)
                    dup = 1;
            if (dup)
                continue;
            row[n++] = u;
            ++taken;
        }
        for (int t = n; t < W; ++t)
            row[t] = -1;
    }
}

/* Eq. 7: Q_G = mean over u of |N(u) & M(u)| / R, M(u) = the R nearest of u */
double or_graph_quality(const int64_t *nbr, int64_t N, int R, const int64_t *knn, int K)
{
    double acc = 0.0;
    int r = R < K ? R : K;
    for (int64_t u = 0; u < N; ++u) {
        int hit = 0;
        for (int s = 0; s < R; ++s) {
            int64_t v = nbr[u * (int64_t)R + s];
            if (v < 0)
                continue;
            for (int t = 0; t < r; ++t)
                if (knn[u * (int64_t)K + t] == v) {
                    ++hit;
                    break;
                }
        }
        acc += (double)hit / (double)R;
    }
    return N > 0 ? acc / (double)N : 0.0;
}

/* ------------------------------------------------------------------ */
/* Alg. 2 (joint pruning), ef-bounded, with the two-stage routing of   */
/* Sec. 4.2 / Sec. 5.2.                                                */
/*                                                                     */
/* pool  : at most ef records sorted by (Gamma, id), each with an      */
/*         "expanded" flag; it is R of Alg. 2 and its unexpanded part  */
/*         is C.                                                       */
/* seeds : B, see or_search below (random stream, attribute entry or  */
/*         given ids).                                                 */
/* step  : take the smallest unexpanded record u (line 3), mark it     */
/*         expanded; evaluate each not-yet-evaluated neighbour v of u  */
/*         in adjacency order (lines 4-5); insert v if the pool holds  */
/*         fewer than ef records or (Gamma, v) is below the last       */
/*         record, dropping the last one (lines 6-8).                  */
/* stop  : no unexpanded record is left ("R is updated" read as "C is  */
/*         not exhausted").  Output the first k records.               */
/* S1    : while h > 1, only the ceil(R/h) valid neighbours with the    */
/*         smallest keys mix64(s_u + (slot+1)*GAMMA), s_u = mix64(s0 ^ */
/*         mix64(u+1)), are evaluated.  S1 ends at a local optimum: an */
/*         expansion after which the pool holds the same records (or   */
/*         when C is exhausted).  S2 sets C = C u R (every record       */
/*         unexpanded) and continues with all neighbours.  Neighbours  */
/*         skipped in S1 are not marked evaluated.                     */
/* max_iters caps the number of expansions; hitting it ends the query  */
/* with status OR_ITER_LIMIT and its current pool.                     */
/* ------------------------------------------------------------------ */
typedef struct {
    double g;
    int64_t id;
    int expanded;
} pool_t;

static int pool_insert(pool_t *pool, int *n, int ef, double g, int64_t id)
{
    if (*n == ef && !rec_less(g, id, pool[ef - 1].g, pool[ef - 1].id))
        return 0;
    int pos = *n < ef ? *n : ef - 1;
    while (pos > 0 && rec_less(g, id, pool[pos - 1].g, pool[pos - 1].id)) {
        pool[pos] = pool[pos - 1];
        --pos;
    }
    pool[pos].g = g;
    pool[pos].id = id;
    pool[pos].expanded = 0;
    if (*n < ef)
        ++*n;
    return 1;
}

/* Seed set B (Alg. 2 takes it as an input):
 *   seed_mode 0  random: the first min(ef, 32) distinct ids of the splitmix64
 *                stream s0 = seed ^ mix64(q), id_j = out_j mod N, j < 64
 *   seed_mode 1  attribute entry: P = the objects whose attributes all equal the
 *                query's, in ascending id; with c = |P| >= 1 and S = min(ef, 32, c),
 *                B = { P[floor(j * c / S)] : j < S }; with c = 0, as mode 0
 *   seed_mode 2  given: the valid distinct ids of seeds_in[q][0..n_seeds), in order
 *   seed_mode 3  nearest attribute entry: P as in mode 1; the M = min(256, c) members
 *                P[floor(j * c / M)], and of them the S = min(ef, 32, M) nearest to the
 *                query by (delta^2 of the f32 rows, summed in index order, id);
 *                with c = 0, as mode 0
 *   open query   (a position holding the wildcard code `wild`) under modes 1 and 3:
 *                its completions fill every open position j with a code 0..a_j (a_j the
 *                largest code of attribute j among the objects), the lowest open
 *                position varying fastest; with T <= 64 completions, P = the runs of the
 *                completions (objects equal to the completed tuple, ascending id) one
 *                after another in completion order, c = |P|, and B follows the rule of
 *                mode 1 (or 3) on that P; with T > 64 or c = 0, as mode 0 */
#define OR_MAX_COMPLETIONS 64

/* the members of an open query's completion runs, in order, into out; returns their
 * number, or -1 when the query has more than OR_MAX_COMPLETIONS completions */
static int64_t or_open_members(const uint8_t *A, int64_t N, int m, const uint8_t *qa, int wild,
                               const int *amax, uint8_t *comp, int64_t *out)
{
    int64_t T = 1;
    for (int j = 0; j < m; ++j)
        if ((int)qa[j] == wild) {
            T *= amax[j] + 1;
            if (T > OR_MAX_COMPLETIONS)
                return -1;
        }
    int64_t n = 0;
    for (int64_t t = 0; t < T; ++t) {
        int64_t rem = t;
        for (int j = 0; j < m; ++j) {
            if ((int)qa[j] == wild) {
                comp[j] = (uint8_t)(rem % (amax[j] + 1));
                rem /= amax[j] + 1;
            } else {
                comp[j] = qa[j];
            }
        }
        for (int64_t v = 0; v < N; ++v)
            if (or_chi(comp, A + v * (int64_t)m, m) == 0)
                out[n++] = v;
    }
    return n;
}

void or_search(const float *X, const uint8_t *A, int64_t N, int d, int m,
               const int64_t *nbr, int R, const float *Qv, const uint8_t *QA, int64_t nq,
               int k, int ef, int h, uint64_t seed, int64_t max_iters,
               int mode, double wv, double wl, int prec, int seed_mode,
               const int64_t *seeds_in, int n_seeds, int vec_round, int rerank,
               int64_t *out_ids, double *out_g, int32_t *out_chi,
               int64_t *out_ndc, int64_t *out_exp, int32_t *out_status, int wild)
{
    /* vec_round: 0 scores with X itself, 1 with X rounded to bf16, 2 to fp8 e4m3, 3 to f16.
     * rerank: the final pool is re-scored with X in the chosen precision prec and
     * re-sorted by (Gamma, id) before the first k are returned. */
    const float *Xs = X;
    float *Xr = NULL;
    if (vec_round != 0) {
        Xr = (float *)malloc(sizeof(float) * (size_t)(N > 0 ? N : 1) * (size_t)d);
        memcpy(Xr, X, sizeof(float) * (size_t)N * (size_t)d);
        or_round_rows(Xr, N * (int64_t)d, vec_round);
        Xs = Xr;
    }
    pool_t *pool = (pool_t *)malloc(sizeof(pool_t) * (size_t)ef);
    int64_t *before = (int64_t *)malloc(sizeof(int64_t) * (size_t)ef);
    uint8_t *evaluated = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    int *sel = (int *)malloc(sizeof(int) * (size_t)(R > 0 ? R : 1));
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(R > 0 ? R : 1));
    int *rank_buf = (int *)malloc(sizeof(int) * (size_t)(R > 0 ? R : 1));
    int s1_take = h > 1 ? (R + h - 1) / h : R;
    int *amax = (int *)calloc((size_t)(m > 0 ? m : 1), sizeof(int));
    for (int64_t v = 0; v < N; ++v)
        for (int j = 0; j < m; ++j)
            if (A[v * (int64_t)m + j] > amax[j])
                amax[j] = A[v * (int64_t)m + j];
    uint8_t *comp = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));

    for (int64_t q = 0; q < nq; ++q) {
        const float *qv = Qv + q * (int64_t)d;
        const uint8_t *qa = QA + q * (int64_t)m;
        memset(evaluated, 0, (size_t)N);
        int n = 0;
        int64_t ndc = 0, iters = 0;
        int32_t status = OR_OK;
        uint64_t s0 = seed ^ or_mix64((uint64_t)q);

        /* seed set B */
        int want = ef < 32 ? ef : 32;
        int64_t c = 0;
        const int open_q = (seed_mode == 1 || seed_mode == 3) && or_query_open(qa, m, wild);
        int64_t c_open = open_q ? or_open_members(A, N, m, qa, wild, amax, comp, members) : 0;
        if ((seed_mode == 1 || seed_mode == 3) && !open_q)
            for (int64_t v = 0; v < N; ++v)
                c += or_chi(qa, A + v * (int64_t)m, m) == 0 ? 1 : 0;
        if (open_q && c_open > 0 && seed_mode == 3) {  /* mode 3's rule on those runs */
            const int M = c_open < 256 ? (int)c_open : 256;
            rec_t *cm = (rec_t *)malloc(sizeof(rec_t) * (size_t)M);
            for (int j = 0; j < M; ++j) {
                const int64_t v = members[((int64_t)j * c_open) / M];
                cm[j].g = (double)or_dist2_32(qv, X + v * (int64_t)d, d);
                cm[j].id = v;
            }
            qsort(cm, (size_t)M, sizeof(rec_t), rec_cmp);
            const int S = want < M ? want : M;
            for (int t = 0; t < S; ++t) {
                const int64_t v = cm[t].id;
                evaluated[v] = 1;
                ++ndc;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
            free(cm);
        } else if (open_q && c_open > 0) {  /* mode 1's rule on those runs */
            const int S = (int64_t)want < c_open ? want : (int)c_open;
            for (int j = 0; j < S; ++j) {
                const int64_t v = members[((int64_t)j * c_open) / S];
                evaluated[v] = 1;
                ++ndc;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
        } else if (seed_mode == 2) {
            for (int j = 0; j < n_seeds; ++j) {
                int64_t v = seeds_in[q * (int64_t)n_seeds + j];
                if (v < 0 || v >= N || evaluated[v])
                    continue;
                evaluated[v] = 1;
                ++ndc;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
        } else if (seed_mode == 3 && c > 0) {
            const int M = c < 256 ? (int)c : 256;
            rec_t *cm = (rec_t *)malloc(sizeof(rec_t) * (size_t)M);
            int64_t rank = 0;
            int j = 0;
            for (int64_t v = 0; v < N && j < M; ++v) {
                if (or_chi(qa, A + v * (int64_t)m, m) != 0)
                    continue;
                if (rank == ((int64_t)j * c) / M) {
                    cm[j].g = (double)or_dist2_32(qv, X + v * (int64_t)d, d);
                    cm[j].id = v;
                    ++j;
                }
                ++rank;
            }
            qsort(cm, (size_t)M, sizeof(rec_t), rec_cmp);
            const int S = want < M ? want : M;
            for (int t = 0; t < S; ++t) {
                const int64_t v = cm[t].id;
                evaluated[v] = 1;
                ++ndc;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
            free(cm);
        } else if (seed_mode == 1 && c > 0) {
            int S = (int64_t)want < c ? want : (int)c;
            int64_t rank = 0;  /* position of v within P */
            int j = 0;
            for (int64_t v = 0; v < N && j < S; ++v) {
                if (or_chi(qa, A + v * (int64_t)m, m) != 0)
                    continue;
                if (rank == ((int64_t)j * c) / S) {
                    evaluated[v] = 1;
                    ++ndc;
                    double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                          mode, wv, wl, prec, NULL, wild);
                    pool_insert(pool, &n, ef, g, v);
                    ++j;
                }
                ++rank;
            }
        } else {
            int got = 0;
            for (uint64_t j = 0; j < 64 && got < want && N > 0; ++j) {
                int64_t v = (int64_t)(or_splitmix64_at(s0, j) % (uint64_t)N);
                if (evaluated[v])
                    continue;
                evaluated[v] = 1;
                ++ndc;
                ++got;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
        }

        int stage = h > 1 ? 1 : 2;
        for (;;) {
            int i = 0;
            while (i < n && pool[i].expanded)
                ++i;
            if (i == n) {
                if (stage == 1) {
                    stage = 2;
                    for (int t = 0; t < n; ++t)
                        pool[t].expanded = 0;
                    continue;
                }
                break;
            }
            if (iters >= max_iters) {
                status = OR_ITER_LIMIT;
                break;
            }
            ++iters;
            pool[i].expanded = 1;
            int64_t u = pool[i].id;
            const int64_t *nu = nbr + u * (int64_t)R;

            /* neighbour slots to evaluate, in adjacency order */
            int ns = 0;
            for (int s = 0; s < R; ++s)
                if (nu[s] >= 0)
                    sel[ns++] = s;
            if (stage == 1 && ns > s1_take) {
                uint64_t su = or_mix64(s0 ^ or_mix64((uint64_t)u + 1));
                for (int t = 0; t < ns; ++t)
                    key[t] = or_splitmix64_at(su, (uint64_t)sel[t]);
                /* keep the s1_take slots of smallest (key, slot), in slot order */
                for (int t = 0; t < ns; ++t) {
                    int rank = 0;
                    for (int o = 0; o < ns; ++o)
                        if (key[o] < key[t] || (key[o] == key[t] && sel[o] < sel[t]))
                            ++rank;
                    rank_buf[t] = rank;
                }
                int w = 0;
                for (int t = 0; t < ns; ++t)
                    if (rank_buf[t] < s1_take)
                        sel[w++] = sel[t];
                ns = w;
            }

            for (int t = 0; t < n; ++t)
                before[t] = pool[t].id;
            int n_before = n;
            for (int t = 0; t < ns; ++t) {
                int64_t v = nu[sel[t]];
                if (evaluated[v])
                    continue;
                evaluated[v] = 1;
                ++ndc;
                double g = pair_gamma(qv, qa, Xs + v * (int64_t)d, A + v * (int64_t)m, d, m,
                                      mode, wv, wl, prec, NULL, wild);
                pool_insert(pool, &n, ef, g, v);
            }
            if (stage == 1) {
                int same = (n == n_before);
                for (int t = 0; t < n && same; ++t)
                    if (before[t] != pool[t].id)
                        same = 0;
                if (same) {
                    stage = 2;
                    for (int t = 0; t < n; ++t)
                        pool[t].expanded = 0;
                }
            }
        }

        if (rerank && n > 0) {
            rec_t *rr = (rec_t *)malloc(sizeof(rec_t) * (size_t)n);
            for (int t = 0; t < n; ++t) {
                int64_t v = pool[t].id;
                rr[t].g = pair_gamma(qv, qa, X + v * (int64_t)d, A + v * (int64_t)m, d, m, mode,
                                     wv, wl, prec, NULL, wild);
                rr[t].id = v;
            }
            qsort(rr, (size_t)n, sizeof(rec_t), rec_cmp);
            for (int t = 0; t < n; ++t) {
                pool[t].g = rr[t].g;
                pool[t].id = rr[t].id;
            }
            free(rr);
        }
        for (int j = 0; j < k; ++j) {
            int64_t o = q * (int64_t)k + j;
            if (j < n) {
                int64_t v = pool[j].id;
                out_ids[o] = v;
                out_g[o] = pool[j].g;
                out_chi[o] = or_chi_query(qa, A + v * (int64_t)m, m, wild);
            } else {
                out_ids[o] = -1;
                out_g[o] = INFINITY;
                out_chi[o] = -1;
            }
        }
        out_ndc[q] = ndc;
        out_exp[q] = iters;
        out_status[q] = status;
    }
    free(amax);
    free(comp);
    free(members);
    free(pool);
    free(before);
    free(evaluated);
    free(sel);
    free(key);
    free(rank_buf);
    free(Xr);
}
