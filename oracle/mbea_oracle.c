/*
 * CPU oracle for maximal biclique enumeration.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path may call
 * this code: it exists so that tests, the smoke check and the benchmark's
 * CPU-baseline leg can check the GPU path. It shares no source with the GPU
 * path.
 *
 * What it computes (paper Section II-A, problem definition): for a bipartite
 * graph G = (U u V, E), every pair (R, L) with R a nonempty subset of U and
 * L a nonempty subset of V such that every u in R is adjacent to every v in
 * L, and no vertex outside the pair can be added on either side. With
 * Gamma(X) the common neighbours of X, these are exactly the pairs with
 * L = Gamma(R) and R = Gamma(L).
 *
 * How (paper Section II-B, Algorithm 1, MBEA): plain recursive backtracking
 * over the four sets L (subset of V), R, P, Q (subsets of U), written with
 * sorted int32 arrays and binary-search intersections, no bitsets, no
 * blocking, no pruning beyond the algorithm's own steps.
 *
 * Readings of points the paper leaves open:
 *  - Initial call: L = V, R = {}, P = U without isolated vertices, Q = {}.
 *    An isolated candidate would give L' = {} and a degenerate pair.
 *  - Candidate selection pops from P the vertex with the smallest
 *    |N(v) n L| (ascending order, Section II-C "candidate selection"),
 *    ties broken by the smaller vertex id. L is fixed for the whole while
 *    loop of one call, so these keys do not change while the loop runs and
 *    the sequence of pops is P sorted by (|N(v) n L|, id); the oracle sorts
 *    once per call instead of rescanning P before every pop.
 *  - A vertex of P that joins R' stays in P (no L - L' removal, no pivots),
 *    unless the pruned mode is asked for (see twin_reps below).
 *  - "nodes" counts the iterations of the while loop (every candidate that
 *    was popped, including those whose node fails the maximality check).
 *
 * Output digest: count = number of maximal bicliques; hash = sum over them,
 * modulo 2^64, of SM( sum_{u in R} SM(2u) + sum_{v in L} SM(2v+1) ), where
 * SM is one SplitMix64 output step (Steele, Lea & Flood, OOPSLA 2014):
 * add the golden gamma 0x9e3779b97f4a7c15, then the variant-13 mix.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ hash */

uint64_t orc_sm(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t key_u(int32_t u) { return orc_sm(2ULL * (uint64_t)u); }
static uint64_t key_v(int32_t v) { return orc_sm(2ULL * (uint64_t)v + 1ULL); }

/* ---------------------------------------------------------------- arrays */

typedef struct {
    int32_t *a;
    int64_t n, cap;
} ovec;

static int ov_push(ovec *v, int32_t x)
{
    if (v->n == v->cap) {
        int64_t nc = v->cap ? v->cap * 2 : 16;
        int32_t *na = (int32_t *)realloc(v->a, (size_t)nc * sizeof(int32_t));
        if (!na) return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->n++] = x;
    return 0;
}

static void ov_free(ovec *v)
{
    free(v->a);
    v->a = NULL;
    v->n = v->cap = 0;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* ----------------------------------------------------------------- graph */

typedef struct {
    int32_t nU, nV;
    const int32_t *u_off, *u_adj; /* N(u) for u in U, sorted V ids */
    const int32_t *v_off, *v_adj; /* N(v) for v in V, sorted U ids */
} ograph;

static const int32_t *nbr(const ograph *g, int32_t u, int64_t *deg)
{
    *deg = g->u_off[u + 1] - g->u_off[u];
    return g->u_adj + g->u_off[u];
}

static int contains(const int32_t *a, int64_t n, int32_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo < n && a[lo] == x;
}

/* |A n B| for sorted A, B: look every element of the shorter up in the longer */
static int64_t count_common(const int32_t *a, int64_t na, const int32_t *b, int64_t nb)
{
    if (na > nb) {
        const int32_t *t = a;
        a = b;
        b = t;
        int64_t tn = na;
        na = nb;
        nb = tn;
    }
    int64_t c = 0;
    for (int64_t i = 0; i < na; ++i) c += contains(b, nb, a[i]);
    return c;
}

/* A n B, sorted, for sorted A, B */
static int intersect(const int32_t *a, int64_t na, const int32_t *b, int64_t nb, ovec *out)
{
    if (na > nb) {
        const int32_t *t = a;
        a = b;
        b = t;
        int64_t tn = na;
        na = nb;
        nb = tn;
    }
    for (int64_t i = 0; i < na; ++i)
        if (contains(b, nb, a[i]) && ov_push(out, a[i])) return -1;
    return 0;
}

/* ----------------------------------------------------------- accumulator */

typedef struct {
    uint64_t count, hash, nodes;
    uint64_t bytes; /* algorithmic bytes, see bytes_node / bytes_root */
    ovec *records;  /* optional: per biclique |R|, |L|, R sorted, L sorted */
    int err;
    uint64_t bytes_b;      /* the second byte model, see bytes_node_b */
    const int32_t *rootL;  /* L of the current root's level-1 call, N(r), sorted */
    int64_t nRootL;
    int32_t min_r, min_l;  /* size filter: only bicliques with |R| >= min_r and |L| >= min_l (1, 1 = all) */
    int32_t prune;         /* iMBE's L - L' removal (Section II-C), see twin_reps */
} oacc;

/*
 * Algorithmic bytes (the roofline numerator). Below the top level every
 * candidate row is the bit pattern of N(y) n L packed in W = ceil(|L|/64)
 * 64-bit words, and the same adjacency read the other way (reverse
 * scanning, Section III-D) is one bitset over Q per vertex of L'. A node of
 * a call with level set L reads x's row (W words); for the check against Q,
 * the cheaper of all Q rows (W |Q| words) and the |L'| columns over Q
 * (|L'| ceil(|Q|/64) words), counted in full; and, when the node is
 * maximal, the rows of the rest of P (W each). A top-level node instead
 * reads the adjacency that builds the root's local universe: N(r) and N(w)
 * for every w in N(r), int32 each.
 */
static uint64_t bytes_node(int64_t nL, int64_t nLp, int64_t nQ, int64_t n_rest, int maximal)
{
    const uint64_t W = (uint64_t)((nL + 63) / 64);
    const uint64_t rows = W * (uint64_t)nQ;
    const uint64_t cols = (uint64_t)nLp * (uint64_t)((nQ + 63) / 64);
    return 8ULL * (W + (rows < cols ? rows : cols) + (maximal ? W * (uint64_t)n_rest : 0));
}

/*
 * Second algorithmic-byte model: per node below the top level, the cheaper
 * of two ways to read what the node needs.
 *  - Bitset rows: one row of ceil(|L|/32) 32-bit words for x and for every
 *    other candidate of the call (Q at this pop and P after it).
 *  - Sorted lists, scanned in reverse (Section III-D): x's adjacency inside
 *    the root's universe, |N(x) n N(r)| ids, then for every w in L' the ids
 *    of its neighbours among the other candidates, |N(w) n (Q u P_rest)|.
 * cx_sum is sum over w in L' of |N(w) n X|, X = Q u P at the call's entry;
 * at every pop X = Q u P_rest u {x}, and x is adjacent to all of L', so the
 * second sum is cx_sum - |L'|. All sizes in int32 (4 bytes).
 */
static uint64_t bytes_node_b(int64_t nL, int64_t nLp, int64_t nQ, int64_t n_rest, int64_t x_in_root,
                             uint64_t cx_sum)
{
    const uint64_t bits = 4ULL * (uint64_t)((nL + 31) / 32) * (uint64_t)(1 + nQ + n_rest);
    const uint64_t list = 4ULL * ((uint64_t)x_in_root + cx_sum - (uint64_t)nLp);
    return bits < list ? bits : list;
}

static void emit(oacc *acc, const ovec *L, const ovec *R)
{
    uint64_t s = 0;
    for (int64_t i = 0; i < R->n; ++i) s += key_u(R->a[i]);
    for (int64_t i = 0; i < L->n; ++i) s += key_v(L->a[i]);
    acc->count += 1;
    acc->hash += orc_sm(s);
    if (acc->records) {
        int32_t *rs = (int32_t *)malloc((size_t)(R->n ? R->n : 1) * sizeof(int32_t));
        if (!rs) {
            acc->err = 1;
            return;
        }
        memcpy(rs, R->a, (size_t)R->n * sizeof(int32_t));
        qsort(rs, (size_t)R->n, sizeof(int32_t), cmp_i32);
        int bad = ov_push(acc->records, (int32_t)R->n) || ov_push(acc->records, (int32_t)L->n);
        for (int64_t i = 0; i < R->n; ++i) bad |= ov_push(acc->records, rs[i]);
        for (int64_t i = 0; i < L->n; ++i) bad |= ov_push(acc->records, L->a[i]);
        free(rs);
        if (bad) acc->err = 1;
    }
}

/* ------------------------------------------------- pruned mode (iMBE) */
/*
 * Embedded pruning by L - L' removal (paper Section II-C, after Zhang et al.'s
 * iMBEA): while x's node expands, a candidate v of P that is adjacent to all
 * of L' and to nothing in L - L' leaves P. Such a v has N(v) n L = L' =
 * N(x) n L: it is a twin of x within L. Every biclique that a later sibling
 * could reach through v has its L inside N(v) n L = N(x) n L, so it also
 * fits x, which is in Q by then: the node is rejected anyway, and so is any
 * node that v would start at its own turn. Removing v therefore changes no
 * output, only the number of nodes. (Nor is v needed in Q: for every later
 * sibling and every node below it, x's test against Q gives the same answer
 * as v's.)
 *
 * Reading used here: the removal is applied whether or not x's own node is
 * maximal. If x's node fails the check, a twin of x fails the same check at
 * its turn and, in later siblings, can only lead to bicliques whose L is
 * covered by the Q vertex that rejected x; so the removal is just as safe,
 * and the removed set becomes a property of the call alone: with the pop
 * sequence seq[0..nP) fixed at the call's entry, seq[j] is removed from P
 * for every pop after rep[j], where rep[j] is the first position whose
 * vertex has the same neighbourhood in L (rep[j] = j when there is none).
 * At its own turn a removed vertex is skipped: no node, and it does not
 * join Q.
 *
 * twin_reps fills rep[0..nP): it sorts the positions by (|N(v) n L|, the
 * sorted list N(v) n L, position) and gives every run of equal lists the
 * position that starts it.
 */
typedef struct {
    const int32_t *a;
    int64_t n, pos;
} olist;

static int cmp_olist(const void *x, const void *y)
{
    const olist *p = (const olist *)x, *q = (const olist *)y;
    if (p->n != q->n) return (p->n > q->n) - (p->n < q->n);
    for (int64_t k = 0; k < p->n; ++k)
        if (p->a[k] != q->a[k]) return (p->a[k] > q->a[k]) - (p->a[k] < q->a[k]);
    return (p->pos > q->pos) - (p->pos < q->pos);
}

static int twin_reps(const ograph *g, const ovec *L, const int32_t *seq, int64_t nP, int64_t *rep)
{
    ovec all = {0};
    int64_t *start = (int64_t *)malloc((size_t)(nP + 1) * sizeof(int64_t));
    olist *lists = (olist *)malloc((size_t)(nP ? nP : 1) * sizeof(olist));
    int rc = -1;
    if (!start || !lists) goto done;
    for (int64_t i = 0; i < nP; ++i) {
        int64_t dv;
        const int32_t *Nv = nbr(g, seq[i], &dv);
        start[i] = all.n;
        if (intersect(Nv, dv, L->a, L->n, &all)) goto done;
    }
    start[nP] = all.n;
    for (int64_t i = 0; i < nP; ++i) {
        lists[i].a = all.a + start[i];
        lists[i].n = start[i + 1] - start[i];
        lists[i].pos = i;
    }
    qsort(lists, (size_t)nP, sizeof(olist), cmp_olist);
    for (int64_t k = 0, first = 0; k < nP; ++k) {
        if (k > 0) {
            const olist *p = &lists[k - 1], *q = &lists[k];
            int same = p->n == q->n;
            for (int64_t t = 0; same && t < p->n; ++t) same = p->a[t] == q->a[t];
            if (!same) first = k;
        }
        rep[lists[k].pos] = lists[first].pos;
    }
    rc = 0;
done:
    ov_free(&all);
    free(start);
    free(lists);
    return rc;
}

/* ------------------------------------------------------------ Algorithm 1 */

static void mbea(const ograph *g, const ovec *L, const ovec *R, const ovec *P, const ovec *Q, oacc *acc);

/*
 * One iteration of Algorithm 1's while loop with candidate x already popped:
 * P_rest is P after the pop, Q the current maximality-checking set. cx[k]
 * (below the top level; NULL there) is |N(L[k]) n X| for the call's
 * candidate set X (second byte model only).
 */
static void mbea_iteration(const ograph *g, const ovec *L, const ovec *R, int32_t x, const int32_t *P_rest,
                           int64_t n_rest, const int32_t *Q, int64_t nQ, const int64_t *cx, oacc *acc)
{
    ovec Rp = {0}, Lp = {0}, Pp = {0}, Qp = {0};
    int64_t dx;
    const int32_t *Nx = nbr(g, x, &dx);
    acc->nodes += 1;

    /* Step 1: R' = R u {x} */
    for (int64_t i = 0; i < R->n; ++i)
        if (ov_push(&Rp, R->a[i])) goto oom;
    if (ov_push(&Rp, x)) goto oom;

    /* Step 2: L' = { v in L : (x, v) in E } */
    if (intersect(L->a, L->n, Nx, dx, &Lp)) goto oom;

    /* Step 3: maximality check against Q */
    int is_maximal = 1;
    for (int64_t i = 0; i < nQ; ++i) {
        int64_t dq;
        const int32_t *Nq = nbr(g, Q[i], &dq);
        int64_t c = count_common(Nq, dq, Lp.a, Lp.n);
        if (c == Lp.n) {
            is_maximal = 0;
            break;
        } else if (c > 0) {
            if (ov_push(&Qp, Q[i])) goto oom;
        }
    }

    if (is_maximal) {
        /* Step 4: maximal expansion over the rest of P. With a size filter
           (min_l > 1) a candidate reaching fewer than min_l vertices of L'
           does not enter P': every node it would start has |L''| < min_l. */
        for (int64_t i = 0; i < n_rest; ++i) {
            int64_t dp;
            const int32_t *Np = nbr(g, P_rest[i], &dp);
            int64_t c = count_common(Np, dp, Lp.a, Lp.n);
            if (c == Lp.n) {
                if (ov_push(&Rp, P_rest[i])) goto oom;
            } else if (c > 0 && c >= acc->min_l) {
                if (ov_push(&Pp, P_rest[i])) goto oom;
            }
        }
        if (Rp.n >= acc->min_r && Lp.n >= acc->min_l) emit(acc, &Lp, &Rp);
        if (R->n == 0) { /* x is this root: its level-1 call works inside N(x) */
            acc->rootL = Lp.a;
            acc->nRootL = Lp.n;
        }
        /* the subtree's level sets are strictly smaller than L' and its R
           within R' u P': recurse only when some biclique there can pass */
        if (Pp.n != 0 && Lp.n - 1 >= acc->min_l && Rp.n + Pp.n >= acc->min_r) mbea(g, &Lp, &Rp, &Pp, &Qp, acc);
    }
    if (R->n == 0) { /* top level: the root's adjacency (both byte models) */
        uint64_t b = 4ULL * (uint64_t)dx;
        for (int64_t k = 0; k < dx; ++k) b += 4ULL * (uint64_t)(g->v_off[Nx[k] + 1] - g->v_off[Nx[k]]);
        acc->bytes += b;
        acc->bytes_b += b;
    } else {
        acc->bytes += bytes_node(L->n, Lp.n, nQ, n_rest, is_maximal);
        /* sum of cx over L' = L n N(x): both sorted, walk them together */
        uint64_t cx_sum = 0;
        for (int64_t i = 0, j = 0; cx && i < L->n && j < Lp.n; ++i)
            if (L->a[i] == Lp.a[j]) {
                cx_sum += (uint64_t)cx[i];
                ++j;
            }
        if (cx)
            acc->bytes_b +=
                bytes_node_b(L->n, Lp.n, nQ, n_rest, count_common(Nx, dx, acc->rootL, acc->nRootL), cx_sum);
    }
    goto done;
oom:
    acc->err = 1;
done:
    ov_free(&Rp);
    ov_free(&Lp);
    ov_free(&Pp);
    ov_free(&Qp);
}

typedef struct {
    int64_t key;
    int32_t id;
} okey;

static int cmp_key(const void *a, const void *b)
{
    const okey *x = (const okey *)a, *y = (const okey *)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->id > y->id) - (x->id < y->id);
}

/* Algorithm 1: MBEA(L, R, P, Q) */
static void mbea(const ograph *g, const ovec *L, const ovec *R, const ovec *P, const ovec *Q, oacc *acc)
{
    int64_t nP = P->n;
    okey *ord = (okey *)malloc((size_t)(nP ? nP : 1) * sizeof(okey));
    int32_t *seq = (int32_t *)malloc((size_t)(nP ? nP : 1) * sizeof(int32_t));
    int32_t *xs = NULL, *rest = NULL;
    int64_t *cx = NULL, *rep = NULL;
    ovec Qc = {0};
    if (!ord || !seq) goto oom;
    if (R->n > 0 && !acc->prune) {
        /* second byte model: cx[k] = |N(L[k]) n X| with X = Q u P, sorted copy */
        xs = (int32_t *)malloc((size_t)(Q->n + nP ? Q->n + nP : 1) * sizeof(int32_t));
        cx = (int64_t *)malloc((size_t)(L->n ? L->n : 1) * sizeof(int64_t));
        if (!xs || !cx) goto oom;
        memcpy(xs, Q->a, (size_t)Q->n * sizeof(int32_t));
        memcpy(xs + Q->n, P->a, (size_t)nP * sizeof(int32_t));
        qsort(xs, (size_t)(Q->n + nP), sizeof(int32_t), cmp_i32);
        for (int64_t k = 0; k < L->n; ++k) {
            const int32_t w = L->a[k];
            cx[k] = count_common(g->v_adj + g->v_off[w], g->v_off[w + 1] - g->v_off[w], xs, Q->n + nP);
        }
    }
    /* candidate selection key |N(v) n L|, then id */
    for (int64_t i = 0; i < nP; ++i) {
        int64_t dv;
        const int32_t *Nv = nbr(g, P->a[i], &dv);
        ord[i].key = count_common(Nv, dv, L->a, L->n);
        ord[i].id = P->a[i];
    }
    qsort(ord, (size_t)nP, sizeof(okey), cmp_key);
    for (int64_t i = 0; i < nP; ++i) seq[i] = ord[i].id;
    for (int64_t i = 0; i < Q->n; ++i)
        if (ov_push(&Qc, Q->a[i])) goto oom;

    if (acc->prune) {
        rep = (int64_t *)malloc((size_t)(nP ? nP : 1) * sizeof(int64_t));
        rest = (int32_t *)malloc((size_t)(nP ? nP : 1) * sizeof(int32_t));
        if (!rep || !rest || twin_reps(g, L, seq, nP, rep)) goto oom;
    }

    for (int64_t i = 0; i < nP && !acc->err; ++i) { /* while |P| > 0 */
        int32_t x = seq[i];                         /* x = P.pop() */
        if (!rep) {
            mbea_iteration(g, L, R, x, seq + i + 1, nP - i - 1, Qc.a, Qc.n, cx, acc);
        } else {
            if (rep[i] < i) continue; /* left P when its twin seq[rep[i]] was popped */
            int64_t nr = 0;
            for (int64_t j = i + 1; j < nP; ++j)
                if (rep[j] >= i) rest[nr++] = seq[j];
            mbea_iteration(g, L, R, x, rest, nr, Qc.a, Qc.n, NULL, acc);
        }
        if (ov_push(&Qc, x)) goto oom; /* Q = Q u {x} */
    }
    goto done;
oom:
    acc->err = 1;
done:
    free(ord);
    free(seq);
    free(xs);
    free(cx);
    free(rep);
    free(rest);
    ov_free(&Qc);
}

/* Initial sets of the top-level call: L = V, P = the U vertices of degree at
   least max(1, min_l) (an isolated vertex gives L' = {}; with a size filter
   a vertex of degree below min_l is in no biclique that passes it). */
static int top_level(const ograph *g, ovec *L, ovec *P, int32_t min_l)
{
    const int32_t dmin = min_l > 1 ? min_l : 1;
    for (int32_t v = 0; v < g->nV; ++v)
        if (ov_push(L, v)) return -1;
    for (int32_t u = 0; u < g->nU; ++u)
        if (g->u_off[u + 1] - g->u_off[u] >= dmin && ov_push(P, u)) return -1;
    return 0;
}

/*
 * Whole-graph enumeration, serial. out[0..3] = count, hash, nodes, bytes;
 * *out_b (when not NULL) = bytes under the second model (plain mode only:
 * 0 when pruning). min_r, min_l: the size filter (1, 1 = every maximal
 * biclique). prune != 0: iMBE's L - L' removal (see twin_reps). When rec != NULL, *rec receives a malloc'd int32 array of records
 * (|R|, |L|, R..., L...) and *rec_len its length (free with orc_free).
 * Returns 0, or -1 on allocation failure.
 */
int orc_enumerate(int32_t nU, int32_t nV, const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                  const int32_t *v_adj, uint64_t *out, int32_t **rec, int64_t *rec_len, uint64_t *out_b,
                  int32_t min_r, int32_t min_l, int32_t prune)
{
    ograph g = {nU, nV, u_off, u_adj, v_off, v_adj};
    ovec L = {0}, R = {0}, P = {0}, Q = {0}, records = {0};
    oacc acc = {0, 0, 0, 0, rec ? &records : NULL, 0, 0, NULL, 0, min_r, min_l, prune ? 1 : 0};
    if (top_level(&g, &L, &P, min_l)) acc.err = 1;
    else mbea(&g, &L, &R, &P, &Q, &acc);
    ov_free(&L);
    ov_free(&P);
    out[0] = acc.count;
    out[1] = acc.hash;
    out[2] = acc.nodes;
    out[3] = acc.bytes;
    if (out_b) *out_b = acc.bytes_b;
    if (rec) {
        *rec = records.a;
        *rec_len = records.n;
    } else {
        ov_free(&records);
    }
    return acc.err ? -1 : 0;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------ per-root driver */
/*
 * The i-th iteration of the top-level while loop depends only on the
 * top-level pop sequence: x = seq[i], P after the pop = seq[i+1..],
 * Q = seq[0..i). So each top-level iteration ("root") can be run on its
 * own, and the per-root results of all roots add up to the whole run.
 */

typedef struct {
    const ograph *g;
    const int32_t *seq;
    const int64_t *pos;
    int64_t nseq;
    const int64_t *rep;    /* pruned mode: twin_reps of the top-level sequence, else NULL */
    const int32_t *kept;   /* pruned mode: the vertices of seq with rep[i] = i, in order */
    const int64_t *nkept;  /* pruned mode: nkept[i] = how many of them sit before position i */
    const ovec *L;
    const int32_t *roots;
    int64_t nroots;
    uint64_t *out;
    uint64_t *out_b;
    int32_t min_r, min_l;
    int64_t next;
    pthread_mutex_t mu;
    int err;
} root_job;

static void run_root(root_job *j, int64_t k)
{
    int32_t r = j->roots[k];
    uint64_t *o = j->out + 4 * k;
    o[0] = o[1] = o[2] = o[3] = 0;
    if (j->out_b) j->out_b[k] = 0;
    if (r < 0 || r >= j->g->nU || j->pos[r] < 0) return; /* isolated: never popped */
    int64_t i = j->pos[r];
    ovec R = {0};
    oacc acc = {0, 0, 0, 0, NULL, 0, 0, NULL, 0, j->min_r, j->min_l, j->rep != NULL};
    if (!j->rep) {
        mbea_iteration(j->g, j->L, &R, r, j->seq + i + 1, j->nseq - i - 1, j->seq, i, NULL, &acc);
    } else if (j->rep[i] == i) { /* a removed root is never popped */
        int32_t *rest = (int32_t *)malloc((size_t)(j->nseq - i > 0 ? j->nseq - i : 1) * sizeof(int32_t));
        if (!rest) {
            j->err = 1;
            return;
        }
        int64_t nr = 0;
        for (int64_t t = i + 1; t < j->nseq; ++t)
            if (j->rep[t] >= i) rest[nr++] = j->seq[t];
        /* Q at this pop: the earlier roots that were popped */
        mbea_iteration(j->g, j->L, &R, r, rest, nr, j->kept, j->nkept[i], NULL, &acc);
        free(rest);
    }
    o[0] = acc.count;
    o[1] = acc.hash;
    o[2] = acc.nodes;
    o[3] = acc.bytes;
    if (j->out_b) j->out_b[k] = acc.bytes_b;
    if (acc.err) j->err = 1;
}

static void *root_worker(void *arg)
{
    root_job *j = (root_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t k = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (k >= j->nroots) break;
        run_root(j, k);
    }
    return NULL;
}

/*
 * Per-root results: out[4k..4k+3] = (count, hash, nodes, bytes) of the top-level
 * iteration whose candidate is roots[k] (zeros for a vertex that is never
 * popped), and out_b[k] (when out_b is not NULL) its bytes under the second
 * model; min_r, min_l, prune: as in orc_enumerate (a root removed by the
 * pruning gives zeros). Runs on nthreads POSIX threads. Returns 0 or -1.
 */
int orc_per_root(int32_t nU, int32_t nV, const int32_t *u_off, const int32_t *u_adj, const int32_t *v_off,
                 const int32_t *v_adj, const int32_t *roots, int64_t nroots, uint64_t *out, int32_t nthreads,
                 uint64_t *out_b, int32_t min_r, int32_t min_l, int32_t prune)
{
    ograph g = {nU, nV, u_off, u_adj, v_off, v_adj};
    ovec L = {0}, P = {0};
    int rc = -1;
    okey *ord = NULL;
    int32_t *seq = NULL, *kept = NULL;
    int64_t *pos = NULL, *rep = NULL, *nkept = NULL;
    if (top_level(&g, &L, &P, min_l)) goto done;
    ord = (okey *)malloc((size_t)(P.n ? P.n : 1) * sizeof(okey));
    seq = (int32_t *)malloc((size_t)(P.n ? P.n : 1) * sizeof(int32_t));
    pos = (int64_t *)malloc((size_t)(nU ? nU : 1) * sizeof(int64_t));
    if (!ord || !seq || !pos) goto done;
    /* the same top-level pop sequence as mbea(): (|N(u) n V|, id) */
    for (int64_t i = 0; i < P.n; ++i) {
        int64_t du;
        const int32_t *Nu = nbr(&g, P.a[i], &du);
        ord[i].key = count_common(Nu, du, L.a, L.n);
        ord[i].id = P.a[i];
    }
    qsort(ord, (size_t)P.n, sizeof(okey), cmp_key);
    for (int32_t u = 0; u < nU; ++u) pos[u] = -1;
    for (int64_t i = 0; i < P.n; ++i) {
        seq[i] = ord[i].id;
        pos[seq[i]] = i;
    }
    if (prune) {
        rep = (int64_t *)malloc((size_t)(P.n ? P.n : 1) * sizeof(int64_t));
        kept = (int32_t *)malloc((size_t)(P.n ? P.n : 1) * sizeof(int32_t));
        nkept = (int64_t *)malloc((size_t)(P.n + 1) * sizeof(int64_t));
        if (!rep || !kept || !nkept || twin_reps(&g, &L, seq, P.n, rep)) goto done;
        int64_t nk = 0;
        for (int64_t i = 0; i < P.n; ++i) {
            nkept[i] = nk;
            if (rep[i] == i) kept[nk++] = seq[i];
        }
        nkept[P.n] = nk;
    }
    root_job job;
    job.g = &g;
    job.seq = seq;
    job.pos = pos;
    job.nseq = P.n;
    job.rep = rep;
    job.kept = kept;
    job.nkept = nkept;
    job.L = &L;
    job.roots = roots;
    job.nroots = nroots;
    job.out = out;
    job.out_b = out_b;
    job.min_r = min_r;
    job.min_l = min_l;
    job.next = 0;
    job.err = 0;
    pthread_mutex_init(&job.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads == 1) {
        root_worker(&job);
    } else {
        pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
        int started = 0;
        for (int t = 0; t < nthreads && th; ++t)
            if (pthread_create(&th[t], NULL, root_worker, &job) == 0) started++;
        if (started == 0) root_worker(&job);
        for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
        free(th);
    }
    pthread_mutex_destroy(&job.mu);
    rc = job.err ? -1 : 0;
done:
    ov_free(&L);
    ov_free(&P);
    free(ord);
    free(seq);
    free(pos);
    free(rep);
    free(kept);
    free(nkept);
    return rc;
}

/* The top-level pop sequence (non-isolated U sorted by (degree, id)). */
int orc_root_order(int32_t nU, const int32_t *u_off, int32_t *seq_out, int64_t *n_out)
{
    okey *ord = (okey *)malloc((size_t)(nU ? nU : 1) * sizeof(okey));
    if (!ord) return -1;
    int64_t n = 0;
    for (int32_t u = 0; u < nU; ++u) {
        int64_t d = u_off[u + 1] - u_off[u];
        if (d > 0) {
            ord[n].key = d;
            ord[n].id = u;
            n++;
        }
    }
    qsort(ord, (size_t)n, sizeof(okey), cmp_key);
    for (int64_t i = 0; i < n; ++i) seq_out[i] = ord[i].id;
    *n_out = n;
    free(ord);
    return 0;
}

/* ------------------------------------------------------ many-graph driver */

typedef struct {
    int32_t n_graphs;
    const int32_t *nU, *nV;
    const int64_t *edge_off, *u_off_start, *v_off_start;
    const int32_t *u_off, *u_adj, *v_off, *v_adj;
    const int32_t *order;
    uint64_t *out;
    int64_t next;
    pthread_mutex_t mu;
    int err;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *j = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        int64_t k = j->next++;
        pthread_mutex_unlock(&j->mu);
        if (k >= j->n_graphs) break;
        int32_t gi = j->order ? j->order[k] : (int32_t)k;
        int64_t e0 = j->edge_off[gi];
        const int32_t *uo = j->u_off + j->u_off_start[gi];
        const int32_t *vo = j->v_off + j->v_off_start[gi];
        if (orc_enumerate(j->nU[gi], j->nV[gi], uo, j->u_adj + e0, vo, j->v_adj + e0, j->out + 4 * (int64_t)gi,
                          NULL, NULL, NULL, 1, 1, 0))
            j->err = 1;
    }
    return NULL;
}

/*
 * Many independent graphs (concatenated CSR/CSC, per-graph local offsets).
 * out[4g..4g+3] = (count, hash, nodes, bytes) of graph g. order (optional) is the
 * sequence in which threads pick graphs up. Returns 0 or -1.
 */
int orc_batch(int32_t n_graphs, const int32_t *nU, const int32_t *nV, const int64_t *edge_off,
              const int64_t *u_off_start, const int64_t *v_off_start, const int32_t *u_off,
              const int32_t *u_adj, const int32_t *v_off, const int32_t *v_adj, const int32_t *order,
              uint64_t *out, int32_t nthreads)
{
    batch_job job = {n_graphs, nU, nV, edge_off, u_off_start, v_off_start, u_off, u_adj, v_off, v_adj,
                     order, out, 0};
    job.err = 0;
    pthread_mutex_init(&job.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
    int started = 0;
    for (int t = 0; t < nthreads && th; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &job) == 0) started++;
    if (started == 0) batch_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    pthread_mutex_destroy(&job.mu);
    return job.err ? -1 : 0;
}

/* ---------------------------------------------------------- brute force */
/*
 * Independent second oracle straight from the definition: for every
 * nonempty A subset of U (|U| <= 24), B = Gamma(A); keep (A, B) when B is
 * nonempty and Gamma(B) = A. Sets are 64-bit word bitsets over V.
 * out[0..1] = count, hash; records as in orc_enumerate.
 */
int orc_bruteforce(int32_t nU, int32_t nV, const int32_t *u_off, const int32_t *u_adj, uint64_t *out,
                   int32_t **rec, int64_t *rec_len)
{
    if (nU > 24 || nU < 0) return -1;
    int64_t W = (nV + 63) / 64;
    uint64_t *rows = (uint64_t *)calloc((size_t)(nU ? nU : 1) * (size_t)(W ? W : 1), sizeof(uint64_t));
    uint64_t *B = (uint64_t *)malloc((size_t)(W ? W : 1) * sizeof(uint64_t));
    ovec records = {0};
    int err = 0;
    if (!rows || !B) {
        free(rows);
        free(B);
        return -1;
    }
    for (int32_t u = 0; u < nU; ++u)
        for (int32_t k = u_off[u]; k < u_off[u + 1]; ++k) rows[(int64_t)u * W + u_adj[k] / 64] |= 1ULL << (u_adj[k] % 64);
    uint64_t count = 0, hash = 0;
    for (uint64_t mask = 1; mask < (1ULL << nU); ++mask) {
        for (int64_t w = 0; w < W; ++w) B[w] = ~0ULL;
        if (nV % 64 && W) B[W - 1] = (1ULL << (nV % 64)) - 1;
        for (int32_t u = 0; u < nU; ++u)
            if (mask >> u & 1)
                for (int64_t w = 0; w < W; ++w) B[w] &= rows[(int64_t)u * W + w];
        int nonempty = 0;
        for (int64_t w = 0; w < W; ++w) nonempty |= (B[w] != 0);
        if (!nonempty) continue;
        uint64_t closure = 0; /* Gamma(B) as a mask over U */
        for (int32_t u = 0; u < nU; ++u) {
            int sup = 1;
            for (int64_t w = 0; w < W; ++w) sup &= ((rows[(int64_t)u * W + w] & B[w]) == B[w]);
            if (sup) closure |= 1ULL << u;
        }
        if (closure != mask) continue;
        uint64_t s = 0;
        int32_t na = 0, nb = 0;
        for (int32_t u = 0; u < nU; ++u)
            if (mask >> u & 1) {
                s += key_u(u);
                na++;
            }
        for (int32_t v = 0; v < nV; ++v)
            if (B[v / 64] >> (v % 64) & 1) {
                s += key_v(v);
                nb++;
            }
        count++;
        hash += orc_sm(s);
        if (rec) {
            err |= ov_push(&records, na) | ov_push(&records, nb);
            for (int32_t u = 0; u < nU; ++u)
                if (mask >> u & 1) err |= ov_push(&records, u);
            for (int32_t v = 0; v < nV; ++v)
                if (B[v / 64] >> (v % 64) & 1) err |= ov_push(&records, v);
        }
    }
    free(rows);
    free(B);
    out[0] = count;
    out[1] = hash;
    if (rec) {
        *rec = records.a;
        *rec_len = records.n;
    } else {
        ov_free(&records);
    }
    return err ? -1 : 0;
}
