/*
 * rnsm_oracle.c -- plain, slow FP64 CPU oracle of the RNSM merge path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path and must never be used as a fallback.
 *
 * What it follows (arxiv 2602.17099):
 *   - distance delta(x,y): Section 2.1 / notation table (squared L2 is used as
 *     the native distance; it orders exactly like delta).  Inner product
 *     (1 - <x,y>) is the unit-norm embedding extension.
 *   - beam search: Algorithm 1 (Section 2.2).
 *   - two-stage PG build (search, RNG-style prune, reverse edges): Section 2.2.
 *   - RNSM: Algorithm 2 (Section 4.2): neighbour expansion, reverse kNN
 *     inversion, lazy-greedy pivot selection, pivot naive search, follower
 *     local sliding, UpdateGraph (concatenate with the existing list and prune;
 *     target vertices gain cross edges only via reverse edges).
 *   - MOS: Algorithm 3 (Section 5) and the execution order of its edges.
 *
 * Readings where the paper is silent:
 *   - candidate order is lexicographic on (distance, id); ties go to the
 *     lower id everywhere;
 *   - "each unexpanded neighbour" of Algorithm 1 is read as "each neighbour
 *     not evaluated before" (equivalent results: an evaluated node that left
 *     C can never re-enter it);
 *   - the prune is the alpha occlusion rule: walk W in (d, id) order, drop a
 *     candidate c if some already kept s has alpha*d(s,c) <= d(v,c), stop at R;
 *   - every search during a merge reads the original (frozen) target graph.
 *
 * Every function is deterministic and independent of the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_L2 0
#define ORC_IP 1

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2

/* ------------------------------------------------------------------------ */
/* Distances (notation table, Section 2.1)                                    */
/* ------------------------------------------------------------------------ */

static double dist64(const float *a, const float *b, int64_t d, int metric) {
    double s = 0.0;
    if (metric == ORC_L2) {
        for (int64_t i = 0; i < d; ++i) {
            double t = (double)a[i] - (double)b[i];
            s += t * t;
        }
        return s;
    }
    for (int64_t i = 0; i < d; ++i) s += (double)a[i] * (double)b[i];
    return 1.0 - s;
}

double orc_distance(const float *a, const float *b, int64_t d, int32_t metric) {
    return dist64(a, b, d, metric);
}

static int lex_less(double da, int32_t ia, double db, int32_t ib) {
    return da < db || (da == db && ia < ib);
}

/* Relative gap of a comparison; used for the per-query decision margin. */
static double rel_gap(double a, double b) {
    double m = fabs(a) > fabs(b) ? fabs(a) : fabs(b);
    if (m == 0.0) return 0.0;
    return fabs(a - b) / m;
}

static void set_threads(int32_t nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int32_t orc_max_threads(void) {
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Beam search (Algorithm 1)                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    double d;
    int32_t id;
    int32_t expanded;
} cand_t;

typedef struct {
    int32_t *stamp; /* per-vertex "evaluated" stamp */
    int32_t epoch;
    int64_t n;
} visit_t;

static int visit_init(visit_t *v, int64_t n) {
    v->stamp = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    v->epoch = 0;
    v->n = n;
    return v->stamp ? 0 : -1;
}

static void visit_free(visit_t *v) { free(v->stamp); v->stamp = NULL; }

static void visit_reset(visit_t *v) {
    if (++v->epoch == INT32_MAX) {
        memset(v->stamp, 0, (size_t)v->n * sizeof(int32_t));
        v->epoch = 1;
    }
}

/* Insert (d,id) into the sorted set C of capacity ef; Algorithm 1's
 * "C <- C u {(v, d)}; resize C to ef" done one candidate at a time, which
 * leaves the same set as inserting the whole neighbourhood and resizing. */
static void c_insert(cand_t *C, int *size, int ef, double d, int32_t id, double *margin) {
    if (*size == ef) {
        cand_t *w = &C[ef - 1];
        double g = rel_gap(d, w->d);
        if (g < *margin) *margin = g;
        if (!lex_less(d, id, w->d, w->id)) return;
        --*size;
    }
    int pos = *size;
    while (pos > 0 && lex_less(d, id, C[pos - 1].d, C[pos - 1].id)) {
        C[pos] = C[pos - 1];
        --pos;
    }
    C[pos].d = d;
    C[pos].id = id;
    C[pos].expanded = 0;
    ++*size;
    if (pos > 0) {
        double g = rel_gap(d, C[pos - 1].d);
        if (g < *margin) *margin = g;
    }
    if (pos + 1 < *size) {
        double g = rel_gap(d, C[pos + 1].d);
        if (g < *margin) *margin = g;
    }
}

/* One query.  Returns |C| (<= ef); C sorted by (d, id). */
static int beam_search_one(const float *X, int64_t n, int64_t d, const int32_t *adj, int32_t r_in,
                           int metric, const float *q, const int32_t *seeds, int32_t n_seeds,
                           int32_t ef, cand_t *C, visit_t *vis, int64_t *ndc, int64_t *nexp,
                           double *margin) {
    int size = 0;
    visit_reset(vis);
    for (int32_t s = 0; s < n_seeds; ++s) {
        int32_t e = seeds[s];
        if (e < 0 || e >= n) continue;
        if (vis->stamp[e] == vis->epoch) continue;
        vis->stamp[e] = vis->epoch;
        double de = dist64(X + (int64_t)e * d, q, d, metric);
        ++*ndc;
        c_insert(C, &size, ef, de, e, margin);
    }
    for (;;) {
        int i = 0;
        while (i < size && C[i].expanded) ++i;
        if (i == size) break; /* no unexpanded node left */
        C[i].expanded = 1;
        ++*nexp;
        int32_t u = C[i].id;
        const int32_t *nb = adj + (int64_t)u * r_in;
        for (int32_t j = 0; j < r_in; ++j) {
            int32_t v = nb[j];
            if (v < 0 || v >= n) continue;
            if (vis->stamp[v] == vis->epoch) continue;
            vis->stamp[v] = vis->epoch;
            double dv = dist64(X + (int64_t)v * d, q, d, metric);
            ++*ndc;
            c_insert(C, &size, ef, dv, v, margin);
        }
    }
    return size;
}

/*
 * Batched beam search.  seeds: [nq * n_seeds] vertex ids (-1 = none).
 * Outputs the first k entries of each final C: out_ids [nq*k] (-1 padded),
 * out_d [nq*k] (INFINITY padded).  Optional per-query NDC, expansions and
 * minimum relative decision margin.
 */
int32_t orc_beam_search_batch(const float *X, int64_t n, int64_t d, const int32_t *adj,
                              int32_t r_in, int32_t metric, const float *Q, int64_t nq,
                              const int32_t *seeds, int32_t n_seeds, int32_t ef, int32_t k,
                              int32_t *out_ids, double *out_d, int64_t *out_ndc,
                              int64_t *out_nexp, double *out_margin, int32_t nthreads) {
    if (ef < 1 || k < 1 || k > ef || n < 1 || d < 1 || r_in < 0) return ORC_EINVAL;
    set_threads(nthreads);
    int32_t err = 0;
#pragma omp parallel
    {
        visit_t vis;
        cand_t *C = (cand_t *)malloc(sizeof(cand_t) * (size_t)ef);
        int ok = (visit_init(&vis, n) == 0) && C;
        if (!ok) {
#pragma omp atomic write
            err = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!ok) continue;
            int64_t ndc = 0, nexp = 0;
            double margin = INFINITY;
            int sz = beam_search_one(X, n, d, adj, r_in, metric, Q + qi * d,
                                     seeds + qi * n_seeds, n_seeds, ef, C, &vis, &ndc, &nexp,
                                     &margin);
            for (int32_t j = 0; j < k; ++j) {
                out_ids[qi * k + j] = j < sz ? C[j].id : -1;
                if (out_d) out_d[qi * k + j] = j < sz ? C[j].d : INFINITY;
            }
            if (out_ndc) out_ndc[qi] = ndc;
            if (out_nexp) out_nexp[qi] = nexp;
            if (out_margin) out_margin[qi] = margin;
        }
        if (C) free(C);
        visit_free(&vis);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* Medoid: default entry point of a segment graph                             */
/* ------------------------------------------------------------------------ */

/* Vertex nearest (native metric) to the FP64 centroid; ties to the lower id. */
int32_t orc_medoid(const float *X, int64_t n, int64_t d, int32_t metric) {
    if (n < 1) return -1;
    double *c = (double *)calloc((size_t)d, sizeof(double));
    if (!c) return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < d; ++j) c[j] += (double)X[i * d + j];
    for (int64_t j = 0; j < d; ++j) c[j] /= (double)n;
    int32_t best = -1;
    double bd = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        const float *x = X + i * d;
        if (metric == ORC_L2) {
            for (int64_t j = 0; j < d; ++j) {
                double t = (double)x[j] - c[j];
                s += t * t;
            }
        } else {
            for (int64_t j = 0; j < d; ++j) s += (double)x[j] * c[j];
            s = 1.0 - s;
        }
        if (s < bd) {
            bd = s;
            best = (int32_t)i;
        }
    }
    free(c);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Occlusion prune (heuristic edge selection, Section 2.2 / Section 4.2)      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double d;
    int32_t id;
} pair_t;

static int pair_cmp(const void *a, const void *b) {
    const pair_t *x = (const pair_t *)a, *y = (const pair_t *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/*
 * Prune the candidate pool W of owner v (all ids index the same vector table
 * X).  Steps: drop v, negatives and duplicates; sort by (d(v,c), id); walk in
 * order, keeping c unless some kept s satisfies alpha * d(s,c) <= d(v,c);
 * stop once R are kept.  If keep_all_if_fit and the deduplicated pool has at
 * most R entries, all are kept (in sorted order) without the occlusion test.
 * Returns the number kept; out/out_d receive them in order.
 */
static int prune_one(const float *X, int64_t d, int metric, int64_t v, const int32_t *W, int nw,
                     int R, float alpha, int keep_all_if_fit, pair_t *buf, int32_t *out,
                     double *out_d, double *margin) {
    int m = 0;
    for (int i = 0; i < nw; ++i) {
        int32_t c = W[i];
        if (c < 0 || (int64_t)c == v) continue;
        int dup = 0;
        for (int j = 0; j < m; ++j)
            if (buf[j].id == c) { dup = 1; break; }
        if (dup) continue;
        buf[m].id = c;
        buf[m].d = dist64(X + v * d, X + (int64_t)c * d, d, metric);
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(pair_t), pair_cmp);
    if (margin)
        for (int i = 1; i < m; ++i) {
            double g = rel_gap(buf[i].d, buf[i - 1].d);
            if (g < *margin) *margin = g;
        }
    int kept = 0;
    if (keep_all_if_fit && m <= R) {
        for (int i = 0; i < m; ++i) {
            out[i] = buf[i].id;
            if (out_d) out_d[i] = buf[i].d;
        }
        return m;
    }
    const double a = (double)alpha;
    for (int i = 0; i < m && kept < R; ++i) {
        int32_t c = buf[i].id;
        int occluded = 0;
        for (int s = 0; s < kept; ++s) {
            double dsc = dist64(X + (int64_t)out[s] * d, X + (int64_t)c * d, d, metric);
            double lhs = a * dsc;
            if (margin) {
                double g = rel_gap(lhs, buf[i].d);
                if (g < *margin) *margin = g;
            }
            if (lhs <= buf[i].d) { occluded = 1; break; }
        }
        if (!occluded) {
            out[kept] = c;
            if (out_d) out_d[kept] = buf[i].d;
            ++kept;
        }
    }
    return kept;
}

/*
 * Batched prune (UpdateGraph's edge selection).  owners[nv] index X;
 * W [nv * w_len] candidate ids into X (-1 = none).  out [nv * R] (-1 padded).
 */
int32_t orc_prune_batch(const float *X, int64_t d, int32_t metric, const int64_t *owners,
                        int64_t nv, const int32_t *W, int32_t w_len, int32_t R, float alpha,
                        int32_t keep_all_if_fit, int32_t *out, double *out_margin,
                        int32_t nthreads) {
    if (R < 1 || w_len < 0) return ORC_EINVAL;
    set_threads(nthreads);
    int32_t err = 0;
#pragma omp parallel
    {
        pair_t *buf = (pair_t *)malloc(sizeof(pair_t) * (size_t)(w_len > 0 ? w_len : 1));
        int32_t *o = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
        int ok = buf && o;
        if (!ok) {
#pragma omp atomic write
            err = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < nv; ++i) {
            if (!ok) continue;
            double margin = INFINITY;
            int kept = prune_one(X, d, metric, owners[i], W + i * w_len, w_len, R, alpha,
                                 keep_all_if_fit, buf, o, NULL, out_margin ? &margin : NULL);
            for (int j = 0; j < R; ++j) out[i * R + j] = j < kept ? o[j] : -1;
            if (out_margin) out_margin[i] = margin;
        }
        free(buf);
        free(o);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* Reverse edges (UpdateGraph, target side)                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t u, v;
} edge_t;

static int edge_cmp(const void *a, const void *b) {
    const edge_t *x = (const edge_t *)a, *y = (const edge_t *)b;
    if (x->u != y->u) return (x->u > y->u) - (x->u < y->u);
    return (x->v > y->v) - (x->v < y->v);
}

/*
 * Insert the reverse edges u <- v of the kept cross edges v -> u.
 * lists: [N * R] current out-lists over X's ids (-1 padded), updated in place.
 * For each target u: pool = list(u) u {v : (u, v) in edges}; if the pool has
 * at most R distinct entries all are kept sorted by (d, id), otherwise the
 * pool is pruned with the occlusion rule.
 */
int32_t orc_reverse_edges(const float *X, int64_t d, int32_t metric, int32_t *lists, int32_t R,
                          const int32_t *eu, const int32_t *ev, int64_t ne, float alpha,
                          int32_t nthreads) {
    if (R < 1) return ORC_EINVAL;
    set_threads(nthreads);
    edge_t *E = (edge_t *)malloc(sizeof(edge_t) * (size_t)(ne > 0 ? ne : 1));
    if (!E) return ORC_ENOMEM;
    for (int64_t i = 0; i < ne; ++i) {
        E[i].u = eu[i];
        E[i].v = ev[i];
    }
    qsort(E, (size_t)ne, sizeof(edge_t), edge_cmp);
    /* segment starts */
    int64_t nseg = 0;
    int64_t *starts = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ne + 1));
    if (!starts) { free(E); return ORC_ENOMEM; }
    for (int64_t i = 0; i < ne; ++i)
        if (i == 0 || E[i].u != E[i - 1].u) starts[nseg++] = i;
    starts[nseg] = ne;
    int32_t err = 0;
#pragma omp parallel
    {
        int cap = 0;
        int32_t *W = NULL;
        pair_t *buf = NULL;
        int32_t *o = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
        if (!o) {
#pragma omp atomic write
            err = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t s = 0; s < nseg; ++s) {
            if (!o) continue;
            int64_t b = starts[s], e = starts[s + 1];
            int32_t u = E[b].u;
            int need = R + (int)(e - b);
            if (need > cap) {
                free(W);
                free(buf);
                cap = need;
                W = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
                buf = (pair_t *)malloc(sizeof(pair_t) * (size_t)cap);
                if (!W || !buf) {
#pragma omp atomic write
                    err = ORC_ENOMEM;
                    cap = 0;
                    continue;
                }
            }
            int nw = 0;
            for (int j = 0; j < R; ++j)
                if (lists[(int64_t)u * R + j] >= 0) W[nw++] = lists[(int64_t)u * R + j];
            for (int64_t i = b; i < e; ++i) W[nw++] = E[i].v;
            int kept = prune_one(X, d, metric, u, W, nw, R, alpha, 1, buf, o, NULL, NULL);
            for (int j = 0; j < R; ++j) lists[(int64_t)u * R + j] = j < kept ? o[j] : -1;
        }
        free(W);
        free(buf);
        free(o);
    }
    free(E);
    free(starts);
    return err;
}

/* ------------------------------------------------------------------------ */
/* RNSM Phase 1: neighbour expansion and reverse kNN inversion               */
/* ------------------------------------------------------------------------ */

/*
 * ExpandNeighbors (Algorithm 2, Phase 1): for every v, a beam search in its
 * own graph for x_v seeded at v with ef = k_plus + 1; v itself is dropped and
 * the next k_plus results form N+(v).  out [n * k_plus] (-1 padded).
 */
int32_t orc_expand(const float *X, int64_t n, int64_t d, const int32_t *adj, int32_t r_in,
                   int32_t metric, int32_t k_plus, int32_t *out, int64_t *out_ndc,
                   int64_t *out_nexp, double *out_margin, int32_t nthreads) {
    if (k_plus < 1 || n < 1) return ORC_EINVAL;
    set_threads(nthreads);
    const int32_t ef = k_plus + 1;
    int32_t err = 0;
#pragma omp parallel
    {
        visit_t vis;
        cand_t *C = (cand_t *)malloc(sizeof(cand_t) * (size_t)ef);
        int ok = (visit_init(&vis, n) == 0) && C;
        if (!ok) {
#pragma omp atomic write
            err = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t v = 0; v < n; ++v) {
            if (!ok) continue;
            int64_t ndc = 0, nexp = 0;
            double margin = INFINITY;
            int32_t seed = (int32_t)v;
            int sz = beam_search_one(X, n, d, adj, r_in, metric, X + v * d, &seed, 1, ef, C, &vis,
                                     &ndc, &nexp, &margin);
            int j = 0;
            for (int i = 0; i < sz && j < k_plus; ++i)
                if (C[i].id != (int32_t)v) out[v * k_plus + j++] = C[i].id;
            for (; j < k_plus; ++j) out[v * k_plus + j] = -1;
            if (out_ndc) out_ndc[v] = ndc;
            if (out_nexp) out_nexp[v] = nexp;
            if (out_margin) out_margin[v] = margin;
        }
        free(C);
        visit_free(&vis);
    }
    return err;
}

/*
 * BuildReverseIndex (Algorithm 2, Phase 1): R_k(x) = { y : x in the first k
 * entries of N+(y) }.  CSR output: offs [n+1], ids [offs[n]] with each
 * R_k(x) listed in ascending y.  ids must hold n*k entries.
 */
int32_t orc_reverse_knn(const int32_t *nplus, int64_t n, int32_t k_plus, int32_t k, int64_t *offs,
                        int32_t *ids) {
    if (k < 1 || k > k_plus) return ORC_EINVAL;
    memset(offs, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t y = 0; y < n; ++y)
        for (int32_t j = 0; j < k; ++j) {
            int32_t x = nplus[y * k_plus + j];
            if (x >= 0 && x < n) offs[x + 1]++;
        }
    for (int64_t x = 0; x < n; ++x) offs[x + 1] += offs[x];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return ORC_ENOMEM;
    memcpy(fill, offs, sizeof(int64_t) * (size_t)n);
    for (int64_t y = 0; y < n; ++y) /* ascending y => each R_k(x) sorted */
        for (int32_t j = 0; j < k; ++j) {
            int32_t x = nplus[y * k_plus + j];
            if (x >= 0 && x < n) ids[fill[x]++] = (int32_t)y;
        }
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* RNSM Phase 2: lazy-greedy pivot selection                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t g;
    int32_t x;
} heap_t;

/* max-heap on (gain desc, id asc) */
static int heap_above(heap_t a, heap_t b) { return a.g > b.g || (a.g == b.g && a.x < b.x); }

static void heap_push(heap_t *h, int64_t *n, heap_t e) {
    int64_t i = (*n)++;
    h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!heap_above(h[i], h[p])) break;
        heap_t t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static heap_t heap_pop(heap_t *h, int64_t *n) {
    heap_t top = h[0];
    h[0] = h[--*n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, b = i;
        if (l < *n && heap_above(h[l], h[b])) b = l;
        if (r < *n && heap_above(h[r], h[b])) b = r;
        if (b == i) break;
        heap_t t = h[i]; h[i] = h[b]; h[b] = t;
        i = b;
    }
    return top;
}

/*
 * Phase 2 of Algorithm 2.  H holds (|R_k(x)|, x) for all x.  Pop the top;
 * skip it if covered; if its current gain |R_k(x) \ Covered| is below the
 * stored one, reinsert with the current gain; otherwise x becomes a pivot,
 * F_x = R_k(x) \ Covered, Covered u= {x} u R_k(x).
 * pivot_of[y] = pivot of follower y, -1 for pivots.  pivots[] in selection
 * order, *n_pivots its length.  Also returns the number of pivots that have
 * an earlier pivot in their R_k (independence is not enforced by Algorithm 2).
 */
int32_t orc_select_pivots(int64_t n, const int64_t *offs, const int32_t *ids, int32_t *pivot_of,
                          int32_t *pivots, int64_t *n_pivots, int64_t *n_dependent) {
    heap_t *h = (heap_t *)malloc(sizeof(heap_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *covered = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    uint8_t *is_pivot = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!h || !covered || !is_pivot) {
        free(h); free(covered); free(is_pivot);
        return ORC_ENOMEM;
    }
    int64_t hn = 0, np = 0, dep = 0;
    for (int64_t x = 0; x < n; ++x) {
        heap_t e = {offs[x + 1] - offs[x], (int32_t)x};
        heap_push(h, &hn, e);
        pivot_of[x] = -2;
    }
    while (hn > 0) {
        heap_t top = heap_pop(h, &hn);
        int32_t x = top.x;
        if (covered[x]) continue;
        int64_t g = 0;
        for (int64_t i = offs[x]; i < offs[x + 1]; ++i) g += !covered[ids[i]];
        if (g < top.g) {
            heap_t e = {g, x};
            heap_push(h, &hn, e);
            continue;
        }
        for (int64_t i = offs[x]; i < offs[x + 1]; ++i) {
            int32_t y = ids[i];
            if (is_pivot[y]) ++dep; /* an earlier pivot is a reverse neighbour of x */
            if (!covered[y]) {
                covered[y] = 1;
                pivot_of[y] = x;
            }
        }
        covered[x] = 1;
        is_pivot[x] = 1;
        pivot_of[x] = -1;
        pivots[np++] = x;
    }
    *n_pivots = np;
    if (n_dependent) *n_dependent = dep;
    free(h);
    free(covered);
    free(is_pivot);
    return ORC_OK;
}

/* IDPS cost of Definition "IDPS" (Section 4.1): gamma*|P| + sum over
 * non-pivots v of min over adjacent pivots of beta*delta(x_v, x_p).  The
 * distance is given as a dense n x n matrix D (tests use tiny n); adjacency
 * as a dense n x n 0/1 matrix A.  Returns INFINITY if P does not dominate. */
double orc_idps_cost(int64_t n, const double *D, const uint8_t *A, const uint8_t *in_P,
                     double gamma, double beta) {
    double cost = 0.0;
    for (int64_t v = 0; v < n; ++v) {
        if (in_P[v]) {
            cost += gamma;
            continue;
        }
        double best = INFINITY;
        for (int64_t p = 0; p < n; ++p)
            if (in_P[p] && A[v * n + p] && beta * D[v * n + p] < best) best = beta * D[v * n + p];
        cost += best;
    }
    return cost;
}

/* ------------------------------------------------------------------------ */
/* Two-stage PG build (Section 2.2), batch-synchronous                        */
/* ------------------------------------------------------------------------ */

/*
 * Builds a degree-R graph over X.  The entry point is the medoid.  Vertices
 * are inserted in id order (the entry first) in rounds; a round inserts the
 * next min(|inserted|, batch_max) vertices: each searches the graph as it
 * stood at the start of the round (seed = entry, ef = L, all L results are
 * candidates), prunes its candidates to R, and then every kept edge v -> u
 * adds the reverse edge u -> v (pool <= R: keep all, else prune).
 * out_adj [n * R] local ids, -1 padded.  *entry receives the medoid.
 */
int32_t orc_build(const float *X, int64_t n, int64_t d, int32_t metric, int32_t R, int32_t L,
                  float alpha, int64_t batch_max, int32_t *out_adj, int32_t *entry,
                  int32_t nthreads) {
    if (n < 1 || R < 1 || L < 1 || batch_max < 1) return ORC_EINVAL;
    set_threads(nthreads);
    int32_t ep = orc_medoid(X, n, d, metric);
    if (ep < 0) return ORC_ENOMEM;
    *entry = ep;
    for (int64_t i = 0; i < n * R; ++i) out_adj[i] = -1;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *snap = (int32_t *)malloc(sizeof(int32_t) * (size_t)n * (size_t)R);
    int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(batch_max * L));
    int32_t *newl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(batch_max * R));
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(batch_max * R));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(batch_max * R));
    int64_t *own = (int64_t *)malloc(sizeof(int64_t) * (size_t)batch_max);
    int32_t *seeds = (int32_t *)malloc(sizeof(int32_t) * (size_t)batch_max);
    float *Qb = (float *)malloc(sizeof(float) * (size_t)(batch_max * d));
    int32_t rc = ORC_OK;
    if (!order || !snap || !cand || !newl || !eu || !ev || !own || !seeds || !Qb) {
        rc = ORC_ENOMEM;
        goto done;
    }
    {
        int64_t k = 0;
        order[k++] = ep;
        for (int64_t i = 0; i < n; ++i)
            if (i != ep) order[k++] = (int32_t)i;
    }
    int64_t inserted = 1;
    while (inserted < n) {
        int64_t b = inserted < batch_max ? inserted : batch_max;
        if (b > n - inserted) b = n - inserted;
        memcpy(snap, out_adj, sizeof(int32_t) * (size_t)n * (size_t)R);
        for (int64_t i = 0; i < b; ++i) {
            int32_t v = order[inserted + i];
            own[i] = v;
            seeds[i] = ep;
            memcpy(Qb + i * d, X + (int64_t)v * d, sizeof(float) * (size_t)d);
        }
        rc = orc_beam_search_batch(X, n, d, snap, R, metric, Qb, b, seeds, 1, L, L, cand, NULL,
                                   NULL, NULL, NULL, nthreads);
        if (rc) goto done;
        rc = orc_prune_batch(X, d, metric, own, b, cand, L, R, alpha, 0, newl, NULL, nthreads);
        if (rc) goto done;
        int64_t ne = 0;
        for (int64_t i = 0; i < b; ++i) {
            int32_t v = (int32_t)own[i];
            for (int32_t j = 0; j < R; ++j) {
                int32_t u = newl[i * R + j];
                out_adj[(int64_t)v * R + j] = u;
                if (u >= 0) {
                    eu[ne] = u;
                    ev[ne] = v;
                    ++ne;
                }
            }
        }
        rc = orc_reverse_edges(X, d, metric, out_adj, R, eu, ev, ne, alpha, nthreads);
        if (rc) goto done;
        inserted += b;
    }
done:
    free(order); free(snap); free(cand); free(newl); free(eu); free(ev); free(own); free(seeds);
    free(Qb);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Brute-force kNN (ground truth for Recall@K, Section 2.1)                   */
/* ------------------------------------------------------------------------ */

int32_t orc_bruteforce_knn(const float *X, int64_t n, int64_t d, int32_t metric, const float *Q,
                           int64_t nq, int32_t k, int32_t *out_ids, double *out_d,
                           int32_t nthreads) {
    if (k < 1) return ORC_EINVAL;
    set_threads(nthreads);
    int32_t err = 0;
#pragma omp parallel
    {
        pair_t *best = (pair_t *)malloc(sizeof(pair_t) * (size_t)(k + 1));
        if (!best) {
#pragma omp atomic write
            err = ORC_ENOMEM;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t qi = 0; qi < nq; ++qi) {
            if (!best) continue;
            int m = 0;
            for (int64_t i = 0; i < n; ++i) {
                double di = dist64(X + i * d, Q + qi * d, d, metric);
                if (m == k && !lex_less(di, (int32_t)i, best[k - 1].d, best[k - 1].id)) continue;
                int pos = m < k ? m++ : k - 1;
                while (pos > 0 && lex_less(di, (int32_t)i, best[pos - 1].d, best[pos - 1].id)) {
                    best[pos] = best[pos - 1];
                    --pos;
                }
                best[pos].d = di;
                best[pos].id = (int32_t)i;
            }
            for (int j = 0; j < k; ++j) {
                out_ids[qi * k + j] = j < m ? best[j].id : -1;
                if (out_d) out_d[qi * k + j] = j < m ? best[j].d : INFINITY;
            }
        }
        free(best);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* RNSM merge (Algorithm 2) over a sequence of segment pairs                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t computed;
    int32_t *nplus;    /* [n_s * k_plus] local ids */
    int64_t *offs;     /* R_k CSR */
    int32_t *rk;
    int32_t *pivot_of; /* -1 for pivots */
    int32_t *pivots;
    int64_t n_pivots;
} src_cache_t;

/*
 * X: all vectors [N * d] in segment-concatenation order (global ids).
 * seg_off [m+1]; adj: each segment's graph in its local ids, concatenated
 * [N * r_in]; entries[m]: local entry vertex of each segment.
 * plan: n_plan ordered pairs (plan_src[i] merged into plan_dst[i]).
 * Per pair (s -> t):
 *   S1-S3 on segment s (once per segment), S4 naive search of every pivot in
 *   the frozen G_t from entry_t with ef = L, S5 local sliding of every
 *   follower seeded with the first min(ef_slide, L) results of its pivot,
 *   ef = ef_slide, S6 prune of list(v) u first c_cross results for every v in
 *   s, S7 reverse edges into t for the kept cross edges.
 * out_adj [N * R] global ids, initialised from the input graphs.
 * stats (nullable) [8]: ndc_expand, ndc_search, nexp_expand, nexp_search,
 * n_pivots_total, n_followers_total, n_dependent_pivots, reverse_edges.
 * cm != 0: the Cross-query Merge comparator of Section 3.1 instead (the
 * paper's CM baseline of Section 6: one-way naive search of every source
 * vertex in the target, no expansion, pivots or sliding): S1-S3 are skipped,
 * every source vertex is a pivot and S4 runs for all of them; S6 and S7 as
 * for RNSM.
 * union_prune != 0: the multi-pair union variant (not in the paper; the
 * merge of several pairs at once, e.g. several new partitions of an
 * incremental merge): S1-S5 of every plan edge as above, then ONE prune per
 * source vertex of W = list(v) u the first c_cross results of each of its
 * plan edges (blocks in plan order), then ONE reverse-edge pass over the kept
 * cross edges of every source, a cross edge being one into a target segment
 * of a plan edge of that source.  Every prune of the plan sees the lists as
 * they were before the plan's reverse edges.
 */
int32_t orc_rnsm_merge(const float *X, int64_t d, const int64_t *seg_off, int32_t m,
                       const int32_t *adj, int32_t r_in, const int32_t *entries, int32_t metric,
                       int32_t R, int32_t L, float alpha, int32_t k_rev, int32_t k_plus,
                       int32_t ef_slide, int32_t c_cross, const int32_t *plan_src,
                       const int32_t *plan_dst, int32_t n_plan, int32_t *out_adj, int64_t *stats,
                       int32_t nthreads, int32_t cm, int32_t union_prune) {
    if (m < 1 || R < 1 || L < 1 || r_in < 0 || r_in > R || k_rev < 1 || k_plus < k_rev ||
        ef_slide < 1 || ef_slide > L || c_cross < 1 || c_cross > ef_slide)
        return ORC_EINVAL;
    set_threads(nthreads);
    int64_t st[8] = {0};
    /* initial merged lists: input lists in global ids */
    for (int32_t s = 0; s < m; ++s)
        for (int64_t v = seg_off[s]; v < seg_off[s + 1]; ++v)
            for (int32_t j = 0; j < R; ++j) {
                int32_t u = j < r_in ? adj[v * r_in + j] : -1;
                out_adj[v * R + j] = u >= 0 ? (int32_t)(u + seg_off[s]) : -1;
            }
    src_cache_t *cache = (src_cache_t *)calloc((size_t)m, sizeof(src_cache_t));
    if (!cache) return ORC_ENOMEM;
    int32_t rc = ORC_OK;
    int64_t nmax = 0;
    for (int32_t s = 0; s < m; ++s)
        if (seg_off[s + 1] - seg_off[s] > nmax) nmax = seg_off[s + 1] - seg_off[s];
    int32_t ks = ef_slide < L ? ef_slide : L;
    float *Qb = (float *)malloc(sizeof(float) * (size_t)(nmax * d));
    int32_t *seedb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * ks));
    int32_t *resP = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * L));  /* by local v */
    int32_t *resB = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * L));
    int32_t *W = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * (R + c_cross)));
    int32_t *newl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * R));
    int64_t *own = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * R));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmax * R));
    int64_t *qidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
    int64_t *ndcb = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
    int64_t *nexb = (int64_t *)malloc(sizeof(int64_t) * (size_t)nmax);
    /* union mode: plan edges of each source (E_s), the block of each edge in its
     * source's union pool, and the pools themselves [n_s * E_s * c_cross] */
    int32_t *n_edges = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    int32_t *blk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_plan > 0 ? n_plan : 1));
    int32_t **upool = (int32_t **)calloc((size_t)m, sizeof(int32_t *));
    if (!Qb || !seedb || !resP || !resB || !W || !newl || !own || !eu || !ev || !qidx || !ndcb ||
        !nexb || !n_edges || !blk || !upool) {
        rc = ORC_ENOMEM;
        goto done;
    }
    if (union_prune)
        for (int32_t pi = 0; pi < n_plan; ++pi) {
            int32_t s = plan_src[pi];
            if (s < 0 || s >= m) { rc = ORC_EINVAL; goto done; }
            blk[pi] = n_edges[s]++;
        }
    for (int32_t pi = 0; pi < n_plan; ++pi) {
        int32_t s = plan_src[pi], t = plan_dst[pi];
        if (s < 0 || s >= m || t < 0 || t >= m || s == t) { rc = ORC_EINVAL; goto done; }
        int64_t s0 = seg_off[s], ns = seg_off[s + 1] - s0;
        int64_t t0 = seg_off[t], nt = seg_off[t + 1] - t0;
        const float *Xs = X + s0 * d, *Xt = X + t0 * d;
        const int32_t *Gs = adj + s0 * r_in, *Gt = adj + t0 * r_in;
        src_cache_t *c = &cache[s];
        if (!c->computed) {
            /* S1: expansion; S2: inversion; S3: pivots */
            c->nplus = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns * k_plus));
            c->offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ns + 1));
            c->rk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns * k_rev));
            c->pivot_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)ns);
            c->pivots = (int32_t *)malloc(sizeof(int32_t) * (size_t)ns);
            if (!c->nplus || !c->offs || !c->rk || !c->pivot_of || !c->pivots) {
                rc = ORC_ENOMEM;
                goto done;
            }
            if (cm) {
                /* CM: every vertex is a pivot, in id order */
                for (int64_t v = 0; v < ns; ++v) {
                    c->pivots[v] = (int32_t)v;
                    c->pivot_of[v] = -1;
                }
                c->n_pivots = ns;
            } else {
                rc = orc_expand(Xs, ns, d, Gs, r_in, metric, k_plus, c->nplus, ndcb, nexb, NULL,
                                nthreads);
                if (rc) goto done;
                for (int64_t i = 0; i < ns; ++i) { st[0] += ndcb[i]; st[2] += nexb[i]; }
                rc = orc_reverse_knn(c->nplus, ns, k_plus, k_rev, c->offs, c->rk);
                if (rc) goto done;
                int64_t dep = 0;
                rc = orc_select_pivots(ns, c->offs, c->rk, c->pivot_of, c->pivots, &c->n_pivots,
                                       &dep);
                if (rc) goto done;
                st[6] += dep;
            }
            c->computed = 1;
        }
        st[4] += c->n_pivots;
        st[5] += ns - c->n_pivots;
        /* S4: pivot naive search in frozen G_t from its default entry */
        int64_t np = c->n_pivots;
        for (int64_t i = 0; i < np; ++i) {
            memcpy(Qb + i * d, Xs + (int64_t)c->pivots[i] * d, sizeof(float) * (size_t)d);
            seedb[i] = entries[t];
        }
        rc = orc_beam_search_batch(Xt, nt, d, Gt, r_in, metric, Qb, np, seedb, 1, L, L, resB, NULL,
                                   ndcb, nexb, NULL, nthreads);
        if (rc) goto done;
        for (int64_t i = 0; i < np; ++i) {
            st[1] += ndcb[i];
            st[3] += nexb[i];
            memcpy(resP + (int64_t)c->pivots[i] * L, resB + i * L, sizeof(int32_t) * (size_t)L);
        }
        /* S5: follower local sliding seeded with its pivot's results */
        int64_t nf = 0;
        for (int64_t y = 0; y < ns; ++y) {
            int32_t p = c->pivot_of[y];
            if (p < 0) continue;
            qidx[nf] = y;
            memcpy(Qb + nf * d, Xs + y * d, sizeof(float) * (size_t)d);
            memcpy(seedb + nf * ks, resP + (int64_t)p * L, sizeof(int32_t) * (size_t)ks);
            ++nf;
        }
        rc = orc_beam_search_batch(Xt, nt, d, Gt, r_in, metric, Qb, nf, seedb, ks, ef_slide,
                                   ef_slide, resB, NULL, ndcb, nexb, NULL, nthreads);
        if (rc) goto done;
        for (int64_t i = 0; i < nf; ++i) {
            st[1] += ndcb[i];
            st[3] += nexb[i];
            memcpy(resP + qidx[i] * L, resB + i * ef_slide, sizeof(int32_t) * (size_t)ef_slide);
        }
        if (union_prune) {
            /* keep the first c_cross results (global ids) in this edge's block */
            if (!upool[s]) {
                upool[s] = (int32_t *)malloc(sizeof(int32_t) * (size_t)ns * (size_t)n_edges[s] *
                                             (size_t)c_cross);
                if (!upool[s]) { rc = ORC_ENOMEM; goto done; }
            }
            const int64_t w = (int64_t)n_edges[s] * c_cross;
            for (int64_t v = 0; v < ns; ++v)
                for (int32_t j = 0; j < c_cross; ++j) {
                    int32_t u = resP[v * L + j];
                    upool[s][v * w + (int64_t)blk[pi] * c_cross + j] = u >= 0 ? (int32_t)(u + t0) : -1;
                }
            continue;
        }
        /* S6: source-side UpdateGraph: list(v) u first c_cross results, prune */
        int32_t wl = R + c_cross;
        for (int64_t v = 0; v < ns; ++v) {
            own[v] = s0 + v;
            memcpy(W + v * wl, out_adj + (s0 + v) * R, sizeof(int32_t) * (size_t)R);
            for (int32_t j = 0; j < c_cross; ++j) {
                int32_t u = resP[v * L + j];
                W[v * wl + R + j] = u >= 0 ? (int32_t)(u + t0) : -1;
            }
        }
        rc = orc_prune_batch(X, d, metric, own, ns, W, wl, R, alpha, 0, newl, NULL, nthreads);
        if (rc) goto done;
        int64_t ne = 0;
        for (int64_t v = 0; v < ns; ++v)
            for (int32_t j = 0; j < R; ++j) {
                int32_t u = newl[v * R + j];
                out_adj[(s0 + v) * R + j] = u;
                if (u >= t0 && u < t0 + nt) { /* kept cross edge into t */
                    eu[ne] = u;
                    ev[ne] = (int32_t)(s0 + v);
                    ++ne;
                }
            }
        st[7] += ne;
        /* S7: reverse edges into the target segment */
        rc = orc_reverse_edges(X, d, metric, out_adj, R, eu, ev, ne, alpha, nthreads);
        if (rc) goto done;
    }
    if (union_prune && n_plan > 0) {
        /* one prune per source vertex over its union pool, sources in order of
         * their first plan edge; then one reverse-edge pass */
        int64_t cap = 0;
        for (int32_t s = 0; s < m; ++s)
            if (n_edges[s]) cap += (seg_off[s + 1] - seg_off[s]) * R;
        int32_t *Eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
        int32_t *Ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));
        uint8_t *is_tgt = (uint8_t *)malloc((size_t)m);
        int64_t ne = 0;
        if (!Eu || !Ev || !is_tgt) rc = ORC_ENOMEM;
        for (int32_t pi = 0; pi < n_plan && rc == ORC_OK; ++pi) {
            int32_t s = plan_src[pi];
            if (blk[pi] != 0) continue;   /* not the source's first edge */
            int64_t s0 = seg_off[s], ns = seg_off[s + 1] - s0;
            int64_t w = (int64_t)n_edges[s] * c_cross, wl = R + w;
            int32_t *Wu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns * wl));
            int64_t *ow = (int64_t *)malloc(sizeof(int64_t) * (size_t)ns);
            int32_t *nl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ns * R));
            if (!Wu || !ow || !nl) {
                rc = ORC_ENOMEM;
            } else {
                for (int64_t v = 0; v < ns; ++v) {
                    ow[v] = s0 + v;
                    memcpy(Wu + v * wl, out_adj + (s0 + v) * R, sizeof(int32_t) * (size_t)R);
                    memcpy(Wu + v * wl + R, upool[s] + v * w, sizeof(int32_t) * (size_t)w);
                }
                rc = orc_prune_batch(X, d, metric, ow, ns, Wu, (int32_t)wl, R, alpha, 0, nl, NULL,
                                     nthreads);
            }
            if (rc == ORC_OK) {
                memset(is_tgt, 0, (size_t)m);
                for (int32_t pj = 0; pj < n_plan; ++pj)
                    if (plan_src[pj] == s) is_tgt[plan_dst[pj]] = 1;
                for (int64_t v = 0; v < ns; ++v)
                    for (int32_t j = 0; j < R; ++j) {
                        int32_t u = nl[v * R + j];
                        out_adj[(s0 + v) * R + j] = u;
                        if (u < 0) continue;
                        int32_t su = 0;   /* segment of u */
                        while (seg_off[su + 1] <= u) ++su;
                        if (is_tgt[su]) {
                            Eu[ne] = u;
                            Ev[ne] = (int32_t)(s0 + v);
                            ++ne;
                        }
                    }
            }
            free(Wu); free(ow); free(nl);
        }
        if (rc == ORC_OK) {
            st[7] += ne;
            rc = orc_reverse_edges(X, d, metric, out_adj, R, Eu, Ev, ne, alpha, nthreads);
        }
        free(Eu); free(Ev); free(is_tgt);
    }
done:
    if (stats) memcpy(stats, st, sizeof(st));
    for (int32_t s = 0; s < m; ++s) {
        free(cache[s].nplus); free(cache[s].offs); free(cache[s].rk);
        free(cache[s].pivot_of); free(cache[s].pivots);
    }
    free(cache);
    free(Qb); free(seedb); free(resP); free(resB); free(W); free(newl); free(own); free(eu);
    free(ev); free(qidx); free(ndcb); free(nexb);
    if (upool)
        for (int32_t s = 0; s < m; ++s) free(upool[s]);
    free(upool); free(n_edges); free(blk);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* MOS (Algorithm 3) and the execution order of its edges (Section 5)         */
/* ------------------------------------------------------------------------ */

#define HOP_INF 0x3fffffff

static void mos_hops(int32_t m, const uint8_t *A, int32_t *H, int32_t *queue) {
    for (int32_t s = 0; s < m; ++s) {
        for (int32_t j = 0; j < m; ++j) H[s * m + j] = HOP_INF;
        H[s * m + s] = 0;
        int32_t qh = 0, qt = 0;
        queue[qt++] = s;
        while (qh < qt) {
            int32_t a = queue[qh++];
            for (int32_t b = 0; b < m; ++b)
                if (A[a * m + b] && H[s * m + b] == HOP_INF) {
                    H[s * m + b] = H[s * m + a] + 1;
                    queue[qt++] = b;
                }
        }
    }
}

/*
 * Algorithm 3 on a symmetric cost matrix C [m*m].  Vertices are visited in
 * ascending order of their mean cost to their Rm cheapest others (ties: lower
 * index).  For v, while some x has hop(v,x) > Delta, take the cheapest such x
 * (ties: lower index): both below the degree bound -> edge (v,x); x saturated
 * -> relay to the cheapest neighbour x' of x that is below the bound, edge
 * (v,x'); v saturated -> symmetric relay (v',x); no feasible relay or both
 * saturated -> edge (v,x) anyway (connectivity is kept, the bound is not).
 * Hops are recomputed by BFS after every edge.
 * Output: edges in insertion order (ea[i] < eb[i] not guaranteed), flags[i]
 * = 1 if that edge broke the degree bound.  Returns the edge count via *ne.
 */
int32_t orc_mos(int32_t m, const double *C, int32_t Rm, int32_t Delta, int32_t *ea, int32_t *eb,
                int32_t *flags, int32_t *ne, int32_t cap) {
    if (m < 1 || Rm < 1 || Delta < 1) return ORC_EINVAL;
    uint8_t *A = (uint8_t *)calloc((size_t)m * (size_t)m, 1);
    int32_t *H = (int32_t *)malloc(sizeof(int32_t) * (size_t)m * (size_t)m);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int32_t *deg = (int32_t *)calloc((size_t)m, sizeof(int32_t));
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    double *avg = (double *)malloc(sizeof(double) * (size_t)m);
    double *row = (double *)malloc(sizeof(double) * (size_t)m);
    int32_t rc = ORC_OK, k = 0;
    if (!A || !H || !queue || !deg || !order || !avg || !row) { rc = ORC_ENOMEM; goto done; }
    /* mean cost to the Rm cheapest other vertices */
    for (int32_t i = 0; i < m; ++i) {
        int32_t c = 0;
        for (int32_t j = 0; j < m; ++j)
            if (j != i) row[c++] = C[i * m + j];
        /* insertion sort: m is tiny */
        for (int32_t a = 1; a < c; ++a) {
            double t = row[a];
            int32_t b = a;
            while (b > 0 && row[b - 1] > t) { row[b] = row[b - 1]; --b; }
            row[b] = t;
        }
        int32_t take = c < Rm ? c : Rm;
        double s = 0.0;
        for (int32_t a = 0; a < take; ++a) s += row[a];
        avg[i] = take > 0 ? s / take : 0.0;
        order[i] = i;
    }
    for (int32_t a = 1; a < m; ++a) {
        int32_t t = order[a], b = a;
        while (b > 0 && (avg[order[b - 1]] > avg[t] ||
                         (avg[order[b - 1]] == avg[t] && order[b - 1] > t))) {
            order[b] = order[b - 1];
            --b;
        }
        order[b] = t;
    }
    mos_hops(m, A, H, queue);
    for (int32_t oi = 0; oi < m; ++oi) {
        int32_t v = order[oi];
        for (;;) {
            int32_t x = -1;
            for (int32_t j = 0; j < m; ++j) {
                if (j == v || H[v * m + j] <= Delta) continue;
                if (x < 0 || C[v * m + j] < C[v * m + x]) x = j;
            }
            if (x < 0) break;
            int32_t a = v, b = x, flag = 0;
            if (deg[v] < Rm && deg[x] < Rm) {
                /* direct edge */
            } else if (deg[v] < Rm && deg[x] >= Rm && Delta >= 2) {
                int32_t best = -1;
                for (int32_t y = 0; y < m; ++y)
                    if (A[x * m + y] && y != v && !A[v * m + y] && deg[y] < Rm &&
                        (best < 0 || C[y * m + v] < C[best * m + v]))
                        best = y;
                if (best >= 0) b = best; else flag = 1;
            } else if (deg[v] >= Rm && deg[x] < Rm && Delta >= 2) {
                int32_t best = -1;
                for (int32_t y = 0; y < m; ++y)
                    if (A[v * m + y] && y != x && !A[x * m + y] && deg[y] < Rm &&
                        (best < 0 || C[y * m + x] < C[best * m + x]))
                        best = y;
                if (best >= 0) a = best; else flag = 1;
            } else {
                flag = 1; /* feasibility fallback: keep connectivity */
            }
            if (k >= cap) { rc = ORC_EINVAL; goto done; }
            A[a * m + b] = A[b * m + a] = 1;
            ++deg[a];
            ++deg[b];
            ea[k] = a;
            eb[k] = b;
            if (flags) flags[k] = flag || deg[a] > Rm || deg[b] > Rm;
            ++k;
            mos_hops(m, A, H, queue);
        }
    }
done:
    *ne = k;
    free(A); free(H); free(queue); free(deg); free(order); free(avg); free(row);
    return rc;
}

/*
 * Merge plan from segment sizes and (optionally) centroids.  Cost: Euclidean
 * distance between centroids, or 1 for every pair when centroids is NULL
 * (random partitions).  Edges of Algorithm 3 are executed closer pairs first
 * (ascending cost; ties by (min index, max index)) and each is oriented
 * smaller segment -> larger one (equal sizes: the larger index is the source).
 * Rm <= 0 selects ceil(sqrt(m-1)) + 1; Delta <= 0 selects 2.
 */
int32_t orc_mos_plan(int32_t m, const int64_t *sizes, const float *centroids, int32_t D,
                     int32_t Rm, int32_t Delta, int32_t *out_src, int32_t *out_dst,
                     double *out_cost, int32_t *n_out, int32_t cap) {
    if (m < 1) return ORC_EINVAL;
    if (Rm <= 0) {
        int32_t r = 0;
        while ((int64_t)r * r < (int64_t)(m - 1)) ++r;
        Rm = r + 1;
    }
    if (Delta <= 0) Delta = 2;
    double *C = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    int32_t *ea = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m * m));
    int32_t *eb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m * m));
    if (!C || !ea || !eb) { free(C); free(ea); free(eb); return ORC_ENOMEM; }
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j) {
            double c = 0.0;
            if (i != j) {
                if (centroids) {
                    for (int32_t t = 0; t < D; ++t) {
                        double z = (double)centroids[i * D + t] - (double)centroids[j * D + t];
                        c += z * z;
                    }
                    c = sqrt(c);
                } else {
                    c = 1.0;
                }
            }
            C[i * m + j] = c;
        }
    int32_t ne = 0;
    int32_t rc = orc_mos(m, C, Rm, Delta, ea, eb, NULL, &ne, m * m);
    if (rc == ORC_OK && ne > cap) rc = ORC_EINVAL;
    if (rc == ORC_OK) {
        /* sort edges by (cost, min idx, max idx) */
        for (int32_t i = 0; i < ne; ++i)
            if (ea[i] > eb[i]) { int32_t t = ea[i]; ea[i] = eb[i]; eb[i] = t; }
        for (int32_t a = 1; a < ne; ++a) {
            int32_t xa = ea[a], xb = eb[a], b = a;
            while (b > 0) {
                double cp = C[ea[b - 1] * m + eb[b - 1]], cc = C[xa * m + xb];
                int before = cp > cc || (cp == cc && (ea[b - 1] > xa ||
                                                      (ea[b - 1] == xa && eb[b - 1] > xb)));
                if (!before) break;
                ea[b] = ea[b - 1];
                eb[b] = eb[b - 1];
                --b;
            }
            ea[b] = xa;
            eb[b] = xb;
        }
        for (int32_t i = 0; i < ne; ++i) {
            int32_t a = ea[i], b = eb[i]; /* a < b */
            int src, dst;
            if (sizes[a] < sizes[b]) { src = a; dst = b; }
            else if (sizes[b] < sizes[a]) { src = b; dst = a; }
            else { src = b; dst = a; } /* equal: larger index merges into smaller */
            out_src[i] = src;
            out_dst[i] = dst;
            if (out_cost) out_cost[i] = C[a * m + b];
        }
        *n_out = ne;
    }
    free(C); free(ea); free(eb);
    return rc;
}
