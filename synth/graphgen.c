/*
 * Seeded synthetic bipartite-graph generators.
 *
 * This module is input infrastructure only: it draws edge lists and holds
 * none of the enumeration's arithmetic. Both the CPU oracle and the GPU
 * library consume what it produces, and neither shares code with it.
 *
 * Random numbers: xoshiro256** (Blackman & Vigna, 2018), with its 256-bit
 * state filled from the SplitMix64 sequence of the seed, as the authors
 * recommend. Build with -ffp-contract=off so that the few floating-point
 * steps (weights, log-uniform sizes) round identically on x86-64 and AArch64.
 *
 * Every generator returns an edge list (eu[k], ev[k]) in malloc'd arrays
 * that the caller releases with gg_free(); the list may hold duplicates
 * (the planted generator unions overlapping blocks). Vertex ids on both
 * sides are randomly permuted after generation so that id order carries no
 * degree information.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} gg_rng;

static uint64_t gg_splitmix(uint64_t *x)
{
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static void gg_seed(gg_rng *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = gg_splitmix(&x);
}

static inline uint64_t gg_rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t gg_next(gg_rng *r)
{
    uint64_t *s = r->s;
    const uint64_t out = gg_rotl(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = gg_rotl(s[3], 45);
    return out;
}

/* uniform double in [0,1) with 53 random bits */
static inline double gg_u53(gg_rng *r) { return (double)(gg_next(r) >> 11) * 0x1.0p-53; }

/* integer in [0,n) by the 64x64->128 multiply-high mapping */
static inline uint64_t gg_below(gg_rng *r, uint64_t n)
{
    return (uint64_t)(((unsigned __int128)gg_next(r) * n) >> 64);
}

/* ---------------------------------------------------------------- buffers */

typedef struct {
    int32_t *u, *v;
    int64_t n, cap;
} gg_edges;

static int gg_push(gg_edges *e, int32_t u, int32_t v)
{
    if (e->n == e->cap) {
        int64_t nc = e->cap ? e->cap * 2 : 1024;
        int32_t *nu = (int32_t *)realloc(e->u, (size_t)nc * sizeof(int32_t));
        if (!nu) return -1;
        e->u = nu;
        int32_t *nv = (int32_t *)realloc(e->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return -1;
        e->v = nv;
        e->cap = nc;
    }
    e->u[e->n] = u;
    e->v[e->n] = v;
    e->n++;
    return 0;
}

static int32_t *gg_permutation(gg_rng *r, int32_t n)
{
    int32_t *p = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!p) return NULL;
    for (int32_t i = 0; i < n; ++i) p[i] = i;
    for (int32_t i = n - 1; i > 0; --i) { /* Fisher-Yates */
        int32_t j = (int32_t)gg_below(r, (uint64_t)i + 1);
        int32_t t = p[i];
        p[i] = p[j];
        p[j] = t;
    }
    return p;
}

static int gg_relabel(gg_rng *r, gg_edges *e, int32_t nU, int32_t nV)
{
    int32_t *pu = gg_permutation(r, nU);
    int32_t *pv = gg_permutation(r, nV);
    if (!pu || !pv) {
        free(pu);
        free(pv);
        return -1;
    }
    for (int64_t k = 0; k < e->n; ++k) {
        e->u[k] = pu[e->u[k]];
        e->v[k] = pv[e->v[k]];
    }
    free(pu);
    free(pv);
    return 0;
}

void gg_free(void *p) { free(p); }

/* ------------------------------------------------------------ Erdos-Renyi */

static int gg_er_into(gg_rng *r, int32_t nU, int32_t nV, double p, gg_edges *e)
{
    for (int32_t u = 0; u < nU; ++u)
        for (int32_t v = 0; v < nV; ++v)
            if (gg_u53(r) < p && gg_push(e, u, v)) return -1;
    return 0;
}

/*
 * Bernoulli(p) bipartite graph: one draw per (u, v) pair, u-major, then the
 * id permutation of both sides from the same stream.
 */
int gg_erdos_renyi(int32_t nU, int32_t nV, double p, uint64_t seed, int32_t **eu, int32_t **ev,
                   int64_t *ne)
{
    gg_rng r;
    gg_seed(&r, seed);
    gg_edges e = {0};
    if (gg_er_into(&r, nU, nV, p, &e) || gg_relabel(&r, &e, nU, nV)) {
        free(e.u);
        free(e.v);
        return -1;
    }
    *eu = e.u;
    *ev = e.v;
    *ne = e.n;
    return 0;
}

/*
 * One graph of the many-small-graphs batch. Its parameters come from the
 * graph's own stream: |U| = round(exp(U(ln lo_u, ln hi_u))), likewise |V|,
 * density p ~ U(p_lo, p_hi); the edges are then drawn as in gg_erdos_renyi
 * from the same stream.
 */
int gg_batch_graph(uint64_t seed, int32_t lo_u, int32_t hi_u, int32_t lo_v, int32_t hi_v, double p_lo,
                   double p_hi, int32_t *nU_out, int32_t *nV_out, double *p_out, int32_t **eu,
                   int32_t **ev, int64_t *ne)
{
    gg_rng r;
    gg_seed(&r, seed);
    double a = log((double)lo_u), b = log((double)hi_u);
    int32_t nU = (int32_t)llround(exp(a + (b - a) * gg_u53(&r)));
    a = log((double)lo_v);
    b = log((double)hi_v);
    int32_t nV = (int32_t)llround(exp(a + (b - a) * gg_u53(&r)));
    double p = p_lo + (p_hi - p_lo) * gg_u53(&r);
    gg_edges e = {0};
    if (gg_er_into(&r, nU, nV, p, &e) || gg_relabel(&r, &e, nU, nV)) {
        free(e.u);
        free(e.v);
        return -1;
    }
    *nU_out = nU;
    *nV_out = nV;
    *p_out = p;
    *eu = e.u;
    *ev = e.v;
    *ne = e.n;
    return 0;
}

/* ---------------------------------------------------------------- planted */

/* k distinct values from [0,n), the first `keep` of them copied from src */
static void gg_pick_side(gg_rng *r, int32_t n, int32_t k, const int32_t *src, int32_t nsrc, int32_t keep,
                         int32_t *out)
{
    int32_t m = 0;
    if (keep > 0) {
        /* partial Fisher-Yates over a copy of the earlier block's side */
        int32_t *tmp = (int32_t *)malloc((size_t)nsrc * sizeof(int32_t));
        memcpy(tmp, src, (size_t)nsrc * sizeof(int32_t));
        for (int32_t i = 0; i < keep; ++i) {
            int32_t j = i + (int32_t)gg_below(r, (uint64_t)(nsrc - i));
            int32_t t = tmp[i];
            tmp[i] = tmp[j];
            tmp[j] = t;
            out[m++] = tmp[i];
        }
        free(tmp);
    }
    while (m < k) {
        int32_t x = (int32_t)gg_below(r, (uint64_t)n);
        int dup = 0;
        for (int32_t i = 0; i < m; ++i) dup |= (out[i] == x);
        if (!dup) out[m++] = x;
    }
}

/*
 * Bernoulli(p_bg) background on nU x nV plus n_blocks planted complete
 * blocks, |A| ~ U{a_lo..a_hi}, |B| ~ U{b_lo..b_hi}. Block i >= 1 picks an
 * earlier block j uniformly and reuses round(overlap*|A_i|) of j's U side
 * and round(overlap*|B_i|) of j's V side; the rest is drawn fresh. The
 * block sides are written to blk_u / blk_v (n_blocks * a_hi and
 * n_blocks * b_hi slots, -1 padded) when those are non-NULL.
 */
int gg_planted(int32_t nU, int32_t nV, double p_bg, int32_t n_blocks, int32_t a_lo, int32_t a_hi,
               int32_t b_lo, int32_t b_hi, double overlap, uint64_t seed, int32_t **eu, int32_t **ev,
               int64_t *ne)
{
    gg_rng r;
    gg_seed(&r, seed);
    gg_edges e = {0};
    int32_t *A = (int32_t *)malloc((size_t)n_blocks * a_hi * sizeof(int32_t));
    int32_t *B = (int32_t *)malloc((size_t)n_blocks * b_hi * sizeof(int32_t));
    int32_t *na = (int32_t *)malloc((size_t)n_blocks * sizeof(int32_t));
    int32_t *nb = (int32_t *)malloc((size_t)n_blocks * sizeof(int32_t));
    int rc = -1;
    if (!A || !B || !na || !nb) goto done;
    if (gg_er_into(&r, nU, nV, p_bg, &e)) goto done;
    for (int32_t i = 0; i < n_blocks; ++i) {
        na[i] = a_lo + (int32_t)gg_below(&r, (uint64_t)(a_hi - a_lo + 1));
        nb[i] = b_lo + (int32_t)gg_below(&r, (uint64_t)(b_hi - b_lo + 1));
        int32_t ka = 0, kb = 0, j = 0;
        if (i > 0) {
            j = (int32_t)gg_below(&r, (uint64_t)i);
            ka = (int32_t)llround(overlap * na[i]);
            kb = (int32_t)llround(overlap * nb[i]);
            if (ka > na[j]) ka = na[j];
            if (kb > nb[j]) kb = nb[j];
        }
        gg_pick_side(&r, nU, na[i], A + (size_t)j * a_hi, na[j], ka, A + (size_t)i * a_hi);
        gg_pick_side(&r, nV, nb[i], B + (size_t)j * b_hi, nb[j], kb, B + (size_t)i * b_hi);
        for (int32_t x = 0; x < na[i]; ++x)
            for (int32_t y = 0; y < nb[i]; ++y)
                if (gg_push(&e, A[(size_t)i * a_hi + x], B[(size_t)i * b_hi + y])) goto done;
    }
    if (gg_relabel(&r, &e, nU, nV)) goto done;
    rc = 0;
done:
    free(A);
    free(B);
    free(na);
    free(nb);
    if (rc) {
        free(e.u);
        free(e.v);
        return rc;
    }
    *eu = e.u;
    *ev = e.v;
    *ne = e.n;
    return 0;
}

/* --------------------------------------------------------------- Chung-Lu */

/*
 * Power-law weights w_i = (i+1)^(-1/(gamma-1)), scaled so that they sum to
 * m, then capped at cap: capped entries are fixed at cap and the rest are
 * rescaled to keep the sum, until no new entry crosses the cap.
 * Returns the cumulative sums (n entries) for inverse-CDF sampling.
 */
static double *gg_cl_cdf(int32_t n, double gamma, double m, double cap)
{
    double *w = (double *)malloc((size_t)n * sizeof(double));
    char *capped = (char *)calloc((size_t)n, 1);
    if (!w || !capped) {
        free(w);
        free(capped);
        return NULL;
    }
    double ex = -1.0 / (gamma - 1.0);
    for (int32_t i = 0; i < n; ++i) w[i] = pow((double)(i + 1), ex);
    for (int iter = 0; iter < 1000; ++iter) {
        double free_sum = 0.0;
        int64_t n_cap = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (capped[i]) n_cap++;
            else free_sum += w[i];
        }
        double scale = (m - (double)n_cap * cap) / free_sum;
        int changed = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (capped[i]) continue;
            w[i] *= scale;
            if (w[i] > cap) {
                capped[i] = 1;
                changed = 1;
            }
        }
        for (int32_t i = 0; i < n; ++i)
            if (capped[i]) w[i] = cap;
        if (!changed) break;
    }
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        acc += w[i];
        w[i] = acc;
    }
    free(capped);
    return w;
}

static int32_t gg_cl_draw(gg_rng *r, const double *cdf, int32_t n)
{
    double t = gg_u53(r) * cdf[n - 1];
    int32_t lo = 0, hi = n - 1; /* first index with cdf > t */
    while (lo < hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > t) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

/*
 * Chung-Lu bipartite graph with exactly m distinct edges: endpoints are
 * drawn independently, u with probability proportional to w_U and v to
 * w_V; a draw is rejected when the edge exists already or an endpoint has
 * reached degree cap.
 */
int gg_chung_lu(int32_t nU, int32_t nV, int64_t m, double gamma_u, double gamma_v, int32_t cap,
                uint64_t seed, int32_t **eu, int32_t **ev, int64_t *ne)
{
    gg_rng r;
    gg_seed(&r, seed);
    double *cu = gg_cl_cdf(nU, gamma_u, (double)m, (double)cap);
    double *cv = gg_cl_cdf(nV, gamma_v, (double)m, (double)cap);
    int32_t *du = (int32_t *)calloc((size_t)nU, sizeof(int32_t));
    int32_t *dv = (int32_t *)calloc((size_t)nV, sizeof(int32_t));
    uint64_t hcap = 1;
    while (hcap < (uint64_t)m * 2) hcap <<= 1;
    uint64_t *table = (uint64_t *)malloc(hcap * sizeof(uint64_t));
    gg_edges e = {0};
    int rc = -1;
    if (!cu || !cv || !du || !dv || !table) goto done;
    memset(table, 0xff, hcap * sizeof(uint64_t));
    while (e.n < m) {
        int32_t u = gg_cl_draw(&r, cu, nU);
        int32_t v = gg_cl_draw(&r, cv, nV);
        if (du[u] >= cap || dv[v] >= cap) continue;
        uint64_t key = (uint64_t)u * (uint64_t)nV + (uint64_t)v;
        uint64_t h = (key * 0x9e3779b97f4a7c15ULL) & (hcap - 1);
        int seen = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == key) {
                seen = 1;
                break;
            }
            h = (h + 1) & (hcap - 1);
        }
        if (seen) continue;
        table[h] = key;
        du[u]++;
        dv[v]++;
        if (gg_push(&e, u, v)) goto done;
    }
    if (gg_relabel(&r, &e, nU, nV)) goto done;
    rc = 0;
done:
    free(cu);
    free(cv);
    free(du);
    free(dv);
    free(table);
    if (rc) {
        free(e.u);
        free(e.v);
        return rc;
    }
    *eu = e.u;
    *ev = e.v;
    *ne = e.n;
    return 0;
}
