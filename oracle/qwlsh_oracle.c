/*
 * qwlsh_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, sequential FP64 restatement of the LSH index and query-workload
 * procedure that the qwLSH paper builds on (arXiv 1907.11803).  It exists so
 * that the CUDA library can be checked against something obviously correct.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the library never calls it, and it shares no code, header, table or
 * helper with the library.
 *
 * Everything is double precision, sequential, with no contraction of a*b+c into
 * a fused multiply-add (build with -ffp-contract=off).  Inputs are float32 and
 * are widened to double exactly.
 *
 * Passages followed (paper sections / equations):
 *   - Section 3, Definition 3.1 and the E2LSH family h(v) = (a.v + b) / w with
 *     a ~ N(0, I), b ~ U[0, w); the floor that makes it a bucket id is lost in
 *     the extracted text and is restored here (reading R1).
 *   - Eq. 1, the collision probability P(r) of that family.
 *   - Section 3.1, collision counting: m hash functions and a collision-count
 *     threshold l instead of l hash layers; the bound of k + v data objects
 *     read per query with v = 100 allowed false positives.
 *   - Section 2, virtual rehashing (C2LSH): the lookup range of every
 *     projection grows level by level without rehashing; range search over a
 *     sorted structure per hash function (QALSH).
 *   - Section 3 / Section 4, the c-k-ANN problem: top-k by exact distance.
 *   - Section 6, default parameters c = 2, delta = 1/e.
 * Readings of points the paper leaves open are numbered R1..R9 in the design
 * notes; the ones used here are cited at each function.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_ERR_RANGE 3

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------- */
/* Eq. 1: P(r) = int_0^w (1/r) (2/sqrt(2 pi)) exp(-t^2 / (2 r^2)) (1 - t/w) dt  */
/* evaluated in closed form:                                                   */
/*   P(r) = 1 - 2 Phi(-w/r) - (2 r / (sqrt(2 pi) w)) (1 - exp(-w^2 / (2 r^2)))  */
/* where Phi is the standard normal CDF (2 Phi(-x) = erfc(x / sqrt 2)).        */
/* ------------------------------------------------------------------------- */
double orc_collision_prob(double r, double w)
{
    if (!(r > 0.0) || !(w > 0.0)) return NAN;
    double x = w / r;
    double two_phi_neg = erfc(x / sqrt(2.0));
    double tail = (2.0 / (sqrt(2.0 * ORC_PI) * x)) * (1.0 - exp(-0.5 * x * x));
    return 1.0 - two_phi_neg - tail;
}

/* Section 3.1 names the collision threshold but not its value (reading R3).
 * It is set the way collision-counting LSH sets it: the fraction alpha of the
 * m projections is chosen between p2 = P(c) and p1 = P(1) so that the two
 * Hoeffding tail bounds are balanced,
 *     ln(1/delta) / (p1 - alpha)^2 = ln(2/beta) / (alpha - p2)^2,
 * with beta = v / n the allowed false-positive fraction (Section 3.1) and
 * delta = 1/e (Section 6).  Solving for alpha gives
 *     alpha = (z p1 + p2) / (1 + z),  z = sqrt(ln(2/beta) / ln(1/delta)).   */
double orc_alpha(double p1, double p2, double beta, double delta)
{
    double z = sqrt(log(2.0 / beta) / log(1.0 / delta));
    return (z * p1 + p2) / (1.0 + z);
}

/* l = ceil(alpha * m), at least 1, at most m. */
int32_t orc_threshold(int32_t m, double w, double c, int64_t n, int32_t v, double delta)
{
    double p1 = orc_collision_prob(1.0, w);
    double p2 = orc_collision_prob(c, w);
    double beta = (double)v / (double)n;
    if (beta >= 1.0) beta = 1.0;
    double alpha = orc_alpha(p1, p2, beta, delta);
    int32_t l = (int32_t)ceil(alpha * (double)m);
    if (l < 1) l = 1;
    if (l > m) l = m;
    return l;
}

/* ------------------------------------------------------------------------- */
/* Section 3: h_i(v) = floor((a_i . v + b_i) / w), all in double.             */
/* The dot product is summed j = 0 .. d-1 in order; then b_i is added and the  */
/* sum is divided by w; floor gives the bucket id.  H is nv x m, row-major.    */
/* ------------------------------------------------------------------------- */
int orc_hash(const float *V, int64_t nv, int32_t d, const float *A, const float *b,
             int32_t m, float w, int32_t *H)
{
    if (!V || !A || !b || !H || nv < 0 || d <= 0 || m <= 0 || !(w > 0.0f)) return ORC_ERR_ARG;
    /* A transposed so the inner loop runs over projections; each projection's
     * sum still runs over j in order. */
    double *AT = (double *)malloc(sizeof(double) * (size_t)d * (size_t)m);
    double *t = (double *)malloc(sizeof(double) * (size_t)m);
    if (!AT || !t) { free(AT); free(t); return ORC_ERR_OOM; }
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < d; ++j)
            AT[(size_t)j * m + i] = (double)A[(size_t)i * d + j];
    int status = ORC_OK;
    for (int64_t r = 0; r < nv; ++r) {
        const float *x = V + (size_t)r * d;
        for (int32_t i = 0; i < m; ++i) t[i] = 0.0;
        for (int32_t j = 0; j < d; ++j) {
            double xj = (double)x[j];
            const double *arow = AT + (size_t)j * m;
            for (int32_t i = 0; i < m; ++i) t[i] = t[i] + arow[i] * xj;
        }
        for (int32_t i = 0; i < m; ++i) {
            double u = (t[i] + (double)b[i]) / (double)w;
            double f = floor(u);
            if (!(f >= -2147483647.0 && f <= 2147483646.0)) { status = ORC_ERR_RANGE; f = 0.0; }
            H[(size_t)r * m + i] = (int32_t)f;
        }
    }
    free(AT);
    free(t);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Index (Section 2, QALSH: a sorted search structure per hash function).      */
/* o_i = min_j h_{j,i} anchors projection i so every data bucket id            */
/* bid = h - o_i is >= 0 (reading R2); span_i = max_j bid.  For every          */
/* projection the (bid, id) pairs are sorted ascending by bid, then id.        */
/* sbid, sid are m x n row-major (projection-major).                           */
/* ------------------------------------------------------------------------- */
typedef struct { int32_t bid; int32_t id; } orc_pair;

static int orc_pair_cmp(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->bid != b->bid) return a->bid < b->bid ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

int orc_build_index(const int32_t *H, int64_t n, int32_t m, int32_t *o, int32_t *span,
                    int32_t *sbid, int32_t *sid)
{
    if (!H || !o || !span || n <= 0 || m <= 0 || n > 2147483647LL) return ORC_ERR_ARG;
    for (int32_t i = 0; i < m; ++i) {
        int32_t lo = H[i], hi = H[i];
        for (int64_t j = 1; j < n; ++j) {
            int32_t h = H[(size_t)j * m + i];
            if (h < lo) lo = h;
            if (h > hi) hi = h;
        }
        if ((int64_t)hi - (int64_t)lo > 2147483646LL) return ORC_ERR_RANGE;
        o[i] = lo;
        span[i] = hi - lo;
    }
    if (!sbid || !sid) return ORC_OK;
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)n);
    if (!p) return ORC_ERR_OOM;
    for (int32_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            p[j].bid = H[(size_t)j * m + i] - o[i];
            p[j].id = (int32_t)j;
        }
        qsort(p, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
        for (int64_t j = 0; j < n; ++j) {
            sbid[(size_t)i * n + j] = p[j].bid;
            sid[(size_t)i * n + j] = p[j].id;
        }
    }
    free(p);
    return ORC_OK;
}

/* Integer floor division for a possibly negative numerator (reading R2). */
static int64_t orc_floordiv(int64_t a, int64_t R)
{
    int64_t q = a / R;
    if ((a % R != 0) && (a < 0)) q -= 1;
    return q;
}

/* Virtual rehashing (Section 2, C2LSH): at level radius R the bucket of
 * projection i is floor(bid / R); a data object collides with the query on
 * projection i when floor(bid / R) == floor(g_i / R), g_i = h_i(q) - o_i.
 * Equivalently bid lies in [beta_i R, beta_i R + R - 1].  col[o] counts the
 * projections on which o collides (Section 3.1).
 * With P probes per side (multi-probe: the neighbouring buckets of the query's
 * bucket are looked into as well, Section 2 on Lv et al.; reading R16) the
 * object collides when floor(bid / R) lies in [beta_i - P, beta_i + P], i.e.
 * bid in [(beta_i - P) R, (beta_i + P + 1) R - 1].  P = 0 is the plain rule. */
void orc_collision_counts_probes(const int32_t *H, int64_t n, int32_t m, const int32_t *o,
                                 const int32_t *hq, int64_t R, int32_t probes, int32_t *col)
{
    int64_t *lo = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    int64_t *hi = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int32_t i = 0; i < m; ++i) {
        int64_t g = (int64_t)hq[i] - (int64_t)o[i];
        int64_t beta = orc_floordiv(g, R);
        lo[i] = (beta - probes) * R;
        hi[i] = (beta + probes + 1) * R - 1;
    }
    for (int64_t j = 0; j < n; ++j) {
        int32_t cnt = 0;
        const int32_t *hrow = H + (size_t)j * m;
        for (int32_t i = 0; i < m; ++i) {
            int64_t bid = (int64_t)hrow[i] - (int64_t)o[i];
            if (bid >= lo[i] && bid <= hi[i]) cnt += 1;
        }
        col[j] = cnt;
    }
    free(lo);
    free(hi);
}

void orc_collision_counts(const int32_t *H, int64_t n, int32_t m, const int32_t *o,
                          const int32_t *hq, int64_t R, int32_t *col)
{
    orc_collision_counts_probes(H, n, m, o, hq, R, 0, col);
}

/* Number of sorted entries of projection i with bid in [lo, hi]: the range
 * search of Section 2 on the sorted arrays (binary search both ends). */
static int64_t orc_lower_bound(const int32_t *a, int64_t n, int64_t key)
{
    int64_t l = 0, r = n;
    while (l < r) {
        int64_t mid = l + (r - l) / 2;
        if ((int64_t)a[mid] < key) l = mid + 1; else r = mid;
    }
    return l;
}

int64_t orc_range_count(const int32_t *sbid_i, int64_t n, int64_t lo, int64_t hi)
{
    if (hi < lo) return 0;
    return orc_lower_bound(sbid_i, n, hi + 1) - orc_lower_bound(sbid_i, n, lo);
}

/* FP64 squared Euclidean distance, summed j = 0 .. d-1 in order. */
double orc_sqdist(const float *x, const float *q, int32_t d)
{
    double s = 0.0;
    for (int32_t j = 0; j < d; ++j) {
        double diff = (double)x[j] - (double)q[j];
        s = s + diff * diff;
    }
    return s;
}

typedef struct { int32_t prev; int32_t col; int64_t id; } orc_cand;

/* Truncation to k + v candidates (Section 3.1 bound; order is reading R5):
 * members of the previous level's candidate set first, then more collisions
 * first, then smaller id first. */
static int orc_cand_cmp(const void *pa, const void *pb)
{
    const orc_cand *a = (const orc_cand *)pa, *b = (const orc_cand *)pb;
    if (a->prev != b->prev) return a->prev > b->prev ? -1 : 1;
    if (a->col != b->col) return a->col > b->col ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

typedef struct { double dist; int64_t id; } orc_res;

static int orc_res_cmp(const void *pa, const void *pb)
{
    const orc_res *a = (const orc_res *)pa, *b = (const orc_res *)pb;
    if (a->dist != b->dist) return a->dist < b->dist ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

/* Per-query statistics, 8 int64 per query:
 *  [0] levels run (1 = stopped at R = 1)   [1] radius R of the last level
 *  [2] |C_R| at the last level            [3] candidates kept (<= k + v)
 *  [4] termination: 2 = |C_R| >= k+v, 3 = R past every bucket
 *  [5] sorted entries inside the last level's ranges (sum over projections;
 *      what an incremental scan reads)
 *  [6] sum over levels of the entries inside that level's ranges
 *  [7] |C_{R/c}|, candidates of the level before the last                   */
#define ORC_NSTAT 8

/* The query procedure for a workload (Sections 2, 3.1, 4).
 * For each query: level radii R = 1, c, c^2, ...; at each level count
 * collisions of every data object over the m projections and form
 * C_R = { o : #col(o) >= l }.  Stop at the first level with |C_R| >= k + v
 * (the k + v bound of Section 3.1), or once R exceeds every bucket id of the
 * data and of the query (after that no level can change C_R) -- readings R3,
 * R4.  Keep at most k + v candidates (order above), compute their exact
 * distances and return the k nearest by (distance, id).  Fewer than k
 * candidates are padded with id -1 and distance +inf.
 *
 * ids, dists: nq x k.  cand_ids / cand_col (optional): nq x (k + v), the kept
 * candidates in truncation order, padded with -1 / 0.  stats (optional):
 * nq x ORC_NSTAT.  sbid (optional, m x n) is used only for the scan counts. */
int orc_query_probes(const float *X, int64_t n, int32_t d, const int32_t *H, const int32_t *o,
                     const int32_t *span, int32_t m, const int32_t *sbid,
                     const float *Q, const int32_t *HQ, int64_t nq, int32_t k, int32_t v,
                     int32_t l, int32_t c, int32_t probes,
                     int64_t *ids, double *dists, int64_t *cand_ids, int32_t *cand_col,
                     int64_t *stats)
{
    if (!X || !H || !o || !span || !Q || !HQ || !ids || !dists) return ORC_ERR_ARG;
    if (n <= 0 || d <= 0 || m <= 0 || nq < 0 || k <= 0 || v < 0 || l < 1 || l > m || c < 2 ||
        probes < 0)
        return ORC_ERR_ARG;
    int64_t cap = (int64_t)k + (int64_t)v;
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *prev = (char *)malloc((size_t)n);
    orc_cand *cs = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
    orc_res *rs = (orc_res *)malloc(sizeof(orc_res) * (size_t)(cap > 0 ? cap : 1));
    if (!col || !prev || !cs || !rs) { free(col); free(prev); free(cs); free(rs); return ORC_ERR_OOM; }

    for (int64_t q = 0; q < nq; ++q) {
        const int32_t *hq = HQ + (size_t)q * m;
        /* past radius `top` no level changes C_R: every data bid lies in
         * [0, span_i]; without probes a query bid g_i < 0 never collides, with
         * probes it does once R > -g_i (reading R16) */
        int64_t top = 0;
        for (int32_t i = 0; i < m; ++i) {
            int64_t g = (int64_t)hq[i] - (int64_t)o[i];
            if (span[i] > top) top = span[i];
            if (g > top) top = g;
            if (probes > 0 && -g > top) top = -g;
        }
        memset(prev, 0, (size_t)n);
        int64_t R = 1, levels = 0, ncand = 0, nprev = 0, scanned_full = 0, scanned_last = 0;
        int term = 0;
        for (;;) {
            levels += 1;
            orc_collision_counts_probes(H, n, m, o, hq, R, probes, col);
            ncand = 0;
            for (int64_t j = 0; j < n; ++j) if (col[j] >= l) ncand += 1;
            if (sbid) {
                scanned_last = 0;
                for (int32_t i = 0; i < m; ++i) {
                    int64_t beta = orc_floordiv((int64_t)hq[i] - (int64_t)o[i], R);
                    scanned_last += orc_range_count(sbid + (size_t)i * n, n, (beta - probes) * R,
                                                    (beta + probes + 1) * R - 1);
                }
                scanned_full += scanned_last;
            }
            if (ncand >= cap) { term = 2; break; }
            if (R > top) { term = 3; break; }
            nprev = ncand;
            for (int64_t j = 0; j < n; ++j) prev[j] = (char)(col[j] >= l);
            R *= c;
        }
        /* candidates of the last level, truncated to k + v */
        int64_t nc = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (col[j] >= l) {
                cs[nc].prev = prev[j];
                cs[nc].col = col[j];
                cs[nc].id = j;
                nc += 1;
            }
        }
        qsort(cs, (size_t)nc, sizeof(orc_cand), orc_cand_cmp);
        int64_t keep = nc < cap ? nc : cap;
        if (cand_ids) {
            for (int64_t t = 0; t < cap; ++t) {
                cand_ids[(size_t)q * cap + t] = t < keep ? cs[t].id : -1;
                if (cand_col) cand_col[(size_t)q * cap + t] = t < keep ? cs[t].col : 0;
            }
        }
        /* exact distances and top-k (Section 3, c-k-ANN; ties by id, R6) */
        const float *qv = Q + (size_t)q * d;
        for (int64_t t = 0; t < keep; ++t) {
            rs[t].id = cs[t].id;
            rs[t].dist = orc_sqdist(X + (size_t)cs[t].id * d, qv, d);
        }
        qsort(rs, (size_t)keep, sizeof(orc_res), orc_res_cmp);
        for (int32_t t = 0; t < k; ++t) {
            ids[(size_t)q * k + t] = t < keep ? rs[t].id : -1;
            dists[(size_t)q * k + t] = t < keep ? sqrt(rs[t].dist) : INFINITY;
        }
        if (stats) {
            int64_t *st = stats + (size_t)q * ORC_NSTAT;
            st[0] = levels; st[1] = R; st[2] = ncand; st[3] = keep;
            st[4] = term; st[5] = scanned_last; st[6] = scanned_full; st[7] = nprev;
        }
    }
    free(col); free(prev); free(cs); free(rs);
    return ORC_OK;
}

int orc_query(const float *X, int64_t n, int32_t d, const int32_t *H, const int32_t *o,
              const int32_t *span, int32_t m, const int32_t *sbid,
              const float *Q, const int32_t *HQ, int64_t nq, int32_t k, int32_t v,
              int32_t l, int32_t c,
              int64_t *ids, double *dists, int64_t *cand_ids, int32_t *cand_col,
              int64_t *stats)
{
    return orc_query_probes(X, n, d, H, o, span, m, sbid, Q, HQ, nq, k, v, l, c, 0, ids, dists,
                            cand_ids, cand_col, stats);
}

/* ------------------------------------------------------------------------- */
/* QALSH's query-aware buckets (Section 2; the base method of the paper's      */
/* experiments, Section 6, w = 2.719): the hash function is the projection    */
/* p_i(v) = a_i . v itself (no offset, no floor), and at level radius R the   */
/* bucket of projection i is the interval of width w R centred on the query:  */
/* an object collides with the query on projection i when                     */
/*     |p_i(o) - p_i(q)| <= w R / 2        (reading R17).                     */
/* Everything else -- counts, threshold l, the k + v stop, truncation order,  */
/* top-k -- is as in orc_query.  Past the radius at which every projection's  */
/* interval holds all the data no level changes C_R (the radius rule).        */
/* ------------------------------------------------------------------------- */

/* P (nv x m, row-major) = a_i . v in double, summed j = 0 .. d-1 in order. */
int orc_project(const float *V, int64_t nv, int32_t d, const float *A, int32_t m, double *P)
{
    if (!V || !A || !P || nv < 0 || d <= 0 || m <= 0) return ORC_ERR_ARG;
    for (int64_t r = 0; r < nv; ++r) {
        const float *x = V + (size_t)r * d;
        for (int32_t i = 0; i < m; ++i) {
            const float *a = A + (size_t)i * d;
            double t = 0.0;
            for (int32_t j = 0; j < d; ++j) t = t + (double)a[j] * (double)x[j];
            P[(size_t)r * m + i] = t;
        }
    }
    return ORC_OK;
}

/* Collision counts at radius R: col[o] = #{ i : |P[o][i] - pq[i]| <= w R / 2 }. */
void orc_qalsh_counts(const double *P, int64_t n, int32_t m, const double *pq, double w,
                      int64_t R, int32_t *col)
{
    const double half = 0.5 * w * (double)R;
    for (int64_t j = 0; j < n; ++j) {
        int32_t cnt = 0;
        for (int32_t i = 0; i < m; ++i) {
            const double dlt = P[(size_t)j * m + i] - pq[i];
            if (fabs(dlt) <= half) cnt += 1;
        }
        col[j] = cnt;
    }
}

/* The query procedure with query-aware buckets.  P: n x m data projections,
 * PQ: nq x m query projections (orc_project); stats as orc_query, with [5] /
 * [6] the entries inside the last level's / every level's intervals. */
int orc_qalsh_query(const float *X, int64_t n, int32_t d, const double *P, int32_t m,
                    const float *Q, const double *PQ, int64_t nq, double w, int32_t k,
                    int32_t v, int32_t l, int32_t c, int64_t *ids, double *dists,
                    int64_t *cand_ids, int32_t *cand_col, int64_t *stats)
{
    if (!X || !P || !Q || !PQ || !ids || !dists) return ORC_ERR_ARG;
    if (n <= 0 || d <= 0 || m <= 0 || nq < 0 || k <= 0 || v < 0 || l < 1 || l > m || c < 2 ||
        !(w > 0.0))
        return ORC_ERR_ARG;
    int64_t cap = (int64_t)k + (int64_t)v;
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *prev = (char *)malloc((size_t)n);
    orc_cand *cs = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)n);
    orc_res *rs = (orc_res *)malloc(sizeof(orc_res) * (size_t)(cap > 0 ? cap : 1));
    double *pmin = (double *)malloc(sizeof(double) * (size_t)m);
    double *pmax = (double *)malloc(sizeof(double) * (size_t)m);
    if (!col || !prev || !cs || !rs || !pmin || !pmax) {
        free(col); free(prev); free(cs); free(rs); free(pmin); free(pmax);
        return ORC_ERR_OOM;
    }
    for (int32_t i = 0; i < m; ++i) {
        pmin[i] = P[i];
        pmax[i] = P[i];
        for (int64_t j = 1; j < n; ++j) {
            const double p = P[(size_t)j * m + i];
            if (p < pmin[i]) pmin[i] = p;
            if (p > pmax[i]) pmax[i] = p;
        }
    }
    for (int64_t q = 0; q < nq; ++q) {
        const double *pq = PQ + (size_t)q * m;
        memset(prev, 0, (size_t)n);
        int64_t R = 1, levels = 0, ncand = 0, nprev = 0, scanned_full = 0, scanned_last = 0;
        int term = 0;
        for (;;) {
            levels += 1;
            orc_qalsh_counts(P, n, m, pq, w, R, col);
            ncand = 0;
            scanned_last = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (col[j] >= l) ncand += 1;
                scanned_last += col[j];
            }
            scanned_full += scanned_last;
            if (ncand >= cap) { term = 2; break; }
            /* every interval holds all the data: no later level changes C_R */
            int all = 1;
            const double half = 0.5 * w * (double)R;
            for (int32_t i = 0; i < m; ++i)
                if (!(fabs(pmin[i] - pq[i]) <= half && fabs(pmax[i] - pq[i]) <= half)) all = 0;
            if (all) { term = 3; break; }
            nprev = ncand;
            for (int64_t j = 0; j < n; ++j) prev[j] = (char)(col[j] >= l);
            R *= c;
        }
        /* the stop level's candidates, truncated to k + v as in orc_query */
        int64_t nc = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (col[j] >= l) {
                cs[nc].prev = prev[j];
                cs[nc].col = col[j];
                cs[nc].id = j;
                nc += 1;
            }
        }
        qsort(cs, (size_t)nc, sizeof(orc_cand), orc_cand_cmp);
        int64_t keep = nc < cap ? nc : cap;
        if (cand_ids) {
            for (int64_t t = 0; t < cap; ++t) {
                cand_ids[(size_t)q * cap + t] = t < keep ? cs[t].id : -1;
                if (cand_col) cand_col[(size_t)q * cap + t] = t < keep ? cs[t].col : 0;
            }
        }
        const float *qv = Q + (size_t)q * d;
        for (int64_t t = 0; t < keep; ++t) {
            rs[t].id = cs[t].id;
            rs[t].dist = orc_sqdist(X + (size_t)cs[t].id * d, qv, d);
        }
        qsort(rs, (size_t)keep, sizeof(orc_res), orc_res_cmp);
        for (int32_t t = 0; t < k; ++t) {
            ids[(size_t)q * k + t] = t < keep ? rs[t].id : -1;
            dists[(size_t)q * k + t] = t < keep ? sqrt(rs[t].dist) : INFINITY;
        }
        if (stats) {
            int64_t *st = stats + (size_t)q * ORC_NSTAT;
            st[0] = levels; st[1] = R; st[2] = ncand; st[3] = keep;
            st[4] = term; st[5] = scanned_last; st[6] = scanned_full; st[7] = nprev;
        }
    }
    free(col); free(prev); free(cs); free(rs); free(pmin); free(pmax);
    return ORC_OK;
}

/* QALSH's collision probability for two points at distance r with a bucket
 * of width w centred on one of them: P(|N(0, r^2)| <= w / 2) = erf(w / (2 sqrt2 r)). */
double orc_qalsh_prob(double r, double w)
{
    if (!(r > 0.0) || !(w > 0.0)) return NAN;
    return erf(w / (2.0 * sqrt(2.0) * r));
}

/* orc_threshold with QALSH's p1 = P(1) and p2 = P(c). */
int32_t orc_qalsh_threshold(int32_t m, double w, double c, int64_t n, int32_t v, double delta)
{
    double p1 = orc_qalsh_prob(1.0, w);
    double p2 = orc_qalsh_prob(c, w);
    double beta = (double)v / (double)n;
    if (beta >= 1.0) beta = 1.0;
    double alpha = orc_alpha(p1, p2, beta, delta);
    int32_t l = (int32_t)ceil(alpha * (double)m);
    if (l < 1) l = 1;
    if (l > m) l = m;
    return l;
}

/* Exact k nearest neighbours by FP64 distance, ties by id (ground truth for
 * recall and the c-k-ANN ratio of Section 3). */
int orc_bruteforce(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq, int32_t k,
                   int64_t *ids, double *dists)
{
    if (!X || !Q || !ids || !dists || n <= 0 || d <= 0 || k <= 0) return ORC_ERR_ARG;
    orc_res *rs = (orc_res *)malloc(sizeof(orc_res) * (size_t)n);
    if (!rs) return ORC_ERR_OOM;
    for (int64_t q = 0; q < nq; ++q) {
        for (int64_t j = 0; j < n; ++j) {
            rs[j].id = j;
            rs[j].dist = orc_sqdist(X + (size_t)j * d, Q + (size_t)q * d, d);
        }
        qsort(rs, (size_t)n, sizeof(orc_res), orc_res_cmp);
        for (int32_t t = 0; t < k; ++t) {
            ids[(size_t)q * k + t] = t < n ? rs[t].id : -1;
            dists[(size_t)q * k + t] = t < n ? sqrt(rs[t].dist) : INFINITY;
        }
    }
    free(rs);
    return ORC_OK;
}
