/*
 * CPU ORACLE for radix-factorised biased sampling on dynamic graphs
 * (Bingo, arXiv 2504.10233).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg load this library.  It shares no code with the CUDA path.
 *
 * What it computes, as plain definitions:
 *   - a dynamic multigraph as explicit per-vertex adjacency lists of
 *     (dst, bias, edge id), kept in ascending edge-id order;
 *   - batched updates with the paper's per-batch order: all insertions, then
 *     all deletions, where deleting a duplicated edge removes the earliest
 *     copy (Section 5.2, parallel batched updates);
 *   - the radix factorisation recomputed from scratch from the adjacency:
 *     D(w) (Eq. dwi), group sizes |G_k| and totals W(p_k) = 2^k |G_k| (Eq. wpk),
 *     and the group kinds of Eq. group (alpha, beta in percent);
 *   - next-hop sampling by inverse transform sampling over exact u64
 *     cumulative biases (Section 2.3, ITS), which draws neighbour i with
 *     probability w_i / sum w (Eq. transition probability);
 *   - DeepWalk, PPR (geometric stop) and node2vec (Eq. node2vec, sampled
 *     directly from the normalised w * f, no rejection) walks;
 *   - the factorised sampler's exact per-neighbour probability
 *     sum_k P(p_k) P(v_i | p_k) (Eqs. group_prob and pvp, Theorem 1), as a
 *     reduced fraction, for pinning Theorem 1 on small inputs;
 *   - radix base 4 (Appendix, Fig. base4): one group per base-4 digit position i,
 *     split into value sub-groups v = 1, 2, 3 (the edges whose digit i equals
 *     v, each carrying v * 4^i); as a graph mode (o_set_base4), sub-group
 *     (i, v) occupies group slot 3 i + v - 1;
 *   - floating-point biases with an amortisation factor lambda: integer part
 *     radix-decomposed, decimal parts in one extra group (Section 4.3), both
 *     for a single vertex (o_float_factor, real arithmetic) and as a graph
 *     mode (o_set_lambda) whose edge weight is lambda*b kept to 2^-8:
 *     256*floor(lambda b) + floor(frac(lambda b) * 256), in integers.
 *
 * Randomness: the oracle's own counter hash; its stream is unrelated to the
 * GPU path's, so walks are compared statistically, never path by path.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

enum { O_EMPTY = 0, O_DENSE = 1, O_ONE = 2, O_SPARSE = 3, O_REGULAR = 4 };
enum { O_OK = 0, O_INVALID = 1, O_NOMEM = 2 };
enum { O_DEEPWALK = 0, O_PPR = 1, O_NODE2VEC = 2 };
#define O_PAD 0xFFFFFFFFu

typedef struct { uint32_t dst, w; uint64_t eid; } o_edge;
typedef struct { o_edge* e; uint64_t len, cap; } o_adj;
typedef struct { uint32_t n; o_adj* a; uint64_t next_eid; double lam; int base4; } o_graph;

/* ------------------------------------------------------------------------------ real biases */

/*
 * Real-valued bias of an edge (Section 4.3, steps (i)-(ii)): the stored 32-bit
 * word is the IEEE-754 binary32 encoding of b.  x = lam * b is rounded once to
 * binary64; its integer part I = floor(x) is radix-decomposed like an integer
 * bias and its decimal part x - I is kept to 8 fractional bits,
 * q = floor((x - I) * 256).  Invalid: b not finite or b < 0, x >= 2^31, or a
 * zero weight (I = q = 0).  Returns 0 when valid.
 */
#define O_FRAC_BITS 8
static int o_real_parts(uint32_t bits, double lam, uint32_t* I, uint32_t* q) {
    float b;
    memcpy(&b, &bits, sizeof b);
    if (!isfinite(b) || b < 0.0f) return 1;
    const double x = lam * (double)b;
    if (!(x < 2147483648.0)) return 1;
    const double ip = floor(x);
    const double fr = x - ip;
    *I = (uint32_t)ip;
    *q = (uint32_t)floor(fr * (double)(1u << O_FRAC_BITS));
    return (*I == 0 && *q == 0) ? 1 : 0;
}

/* ------------------------------------------------------------------------------ radix base 4 */

/* Base-4 digit i of w: floor(w / 4^i) mod 4. */
static inline uint32_t o_digit4(uint32_t w, int i) {
    uint64_t p = 1;
    for (int t = 0; t < i; t++) p *= 4;
    return (uint32_t)((w / p) % 4);
}
#define O_B4_POSITIONS 10 /* base-4 mode: biases below 4^10, sub-groups 3 i + v - 1 < 30 */

/* Integer part, the part of an edge that is radix-decomposed. */
static inline uint32_t o_int_part(const o_graph* g, uint32_t w) {
    if (g->lam == 0.0) return w;
    uint32_t I, q;
    o_real_parts(w, g->lam, &I, &q);
    return I;
}

/* Sampling weight of an edge: the integer bias, or 2^8 * I + q for real biases. */
static inline uint64_t o_weight(const o_graph* g, uint32_t w) {
    if (g->lam == 0.0) return w;
    uint32_t I, q;
    o_real_parts(w, g->lam, &I, &q);
    return ((uint64_t)I << O_FRAC_BITS) + q;
}

/* 1 iff an edge with stored word w belongs to group slot k: bit k of the (integer part of the)
 * bias, or in base 4 the sub-group of digit position k / 3 with value k % 3 + 1. */
static inline int o_in_slot(const o_graph* g, uint32_t w, int k) {
    if (g->base4) return k < 3 * O_B4_POSITIONS && o_digit4(w, k / 3) == (uint32_t)(k % 3 + 1);
    return (o_int_part(g, w) >> k) & 1u;
}

/* Weight one member of slot k carries: 2^k, 2^(k+8) for real biases (units of 2^-8), or
 * v * 4^i for base-4 sub-group (i, v). */
static inline uint64_t o_slot_unit(const o_graph* g, int k) {
    if (g->base4) {
        uint64_t p = 1;
        for (int t = 0; t < k / 3; t++) p *= 4;
        return (uint64_t)(k % 3 + 1) * p;
    }
    return (uint64_t)1 << (k + (g->lam != 0.0 ? O_FRAC_BITS : 0));
}

static inline uint32_t o_dec_part(const o_graph* g, uint32_t w) {
    if (g->lam == 0.0) return 0;
    uint32_t I, q;
    o_real_parts(w, g->lam, &I, &q);
    return q;
}

/* ------------------------------------------------------------------------------ graph */

static int adj_push(o_adj* a, o_edge x) {
    if (a->len == a->cap) {
        uint64_t nc = a->cap ? a->cap * 2 : 4;
        o_edge* ne = (o_edge*)realloc(a->e, sizeof(o_edge) * nc);
        if (!ne) return O_NOMEM;
        a->e = ne;
        a->cap = nc;
    }
    a->e[a->len++] = x;
    return O_OK;
}

/* Edge ids are assigned 0..m-1 in CSR order. */
o_graph* o_create(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w) {
    o_graph* g = (o_graph*)calloc(1, sizeof(o_graph));
    if (!g) return NULL;
    g->n = n;
    g->a = (o_adj*)calloc(n ? n : 1, sizeof(o_adj));
    if (!g->a) { free(g); return NULL; }
    for (uint32_t v = 0; v < n; v++) {
        uint64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d) {
            g->a[v].e = (o_edge*)malloc(sizeof(o_edge) * d);
            g->a[v].cap = d;
        }
        for (uint64_t j = row_ptr[v]; j < row_ptr[v + 1]; j++) {
            o_edge x = {col[j], w[j], j};
            g->a[v].e[g->a[v].len++] = x;
        }
    }
    g->next_eid = row_ptr[n];
    return g;
}

/* The same with explicit edge ids: edge j of the CSR has id eid[j] (ascending within each row), and
 * later insertions continue from next_eid.  A graph holding only some sources' rows keeps the ids
 * those edges have in the whole graph (sampled-vertex parity: Section 5.2's batch semantics are per
 * source, so a source's edges depend only on its own rows and records). */
o_graph* o_create_ids(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                      const uint64_t* eid, uint64_t next_eid) {
    o_graph* g = o_create(n, row_ptr, col, w);
    if (!g) return NULL;
    for (uint32_t v = 0; v < n; v++)
        for (uint64_t j = 0; j < g->a[v].len; j++) g->a[v].e[j].eid = eid[row_ptr[v] + j];
    g->next_eid = next_eid;
    return g;
}

void o_destroy(o_graph* g) {
    if (!g) return;
    for (uint32_t v = 0; v < g->n; v++) free(g->a[v].e);
    free(g->a);
    free(g);
}

uint64_t o_num_edges(const o_graph* g) {
    uint64_t m = 0;
    for (uint32_t v = 0; v < g->n; v++) m += g->a[v].len;
    return m;
}

uint32_t o_degree(const o_graph* g, uint32_t v) { return (uint32_t)g->a[v].len; }

/* Export the live edges of every vertex in ascending edge-id order. offs has n+1 entries. */
void o_export_edges(const o_graph* g, uint64_t* offs, uint32_t* dst, uint32_t* w, uint64_t* eid) {
    uint64_t p = 0;
    for (uint32_t v = 0; v < g->n; v++) {
        offs[v] = p;
        for (uint64_t j = 0; j < g->a[v].len; j++, p++) {
            dst[p] = g->a[v].e[j].dst;
            w[p] = g->a[v].e[j].w;
            eid[p] = g->a[v].e[j].eid;
        }
    }
    offs[g->n] = p;
}

/* Switch the graph to real-valued biases with amortisation factor lam > 0
 * (stored words are binary32 encodings).  O_INVALID if any edge is invalid. */
int o_set_lambda(o_graph* g, double lam) {
    if (!(lam > 0.0)) return O_INVALID;
    for (uint32_t v = 0; v < g->n; v++)
        for (uint64_t j = 0; j < g->a[v].len; j++) {
            uint32_t I, q;
            if (o_real_parts(g->a[v].e[j].w, lam, &I, &q)) return O_INVALID;
        }
    g->lam = lam;
    return O_OK;
}

/* Switch the graph to radix base 4 (integer biases below 4^10).  O_INVALID if an edge's bias is
 * too wide or the graph holds real biases. */
int o_set_base4(o_graph* g) {
    if (g->lam != 0.0) return O_INVALID;
    for (uint32_t v = 0; v < g->n; v++)
        for (uint64_t j = 0; j < g->a[v].len; j++)
            if (g->a[v].e[j].w >= (1u << (2 * O_B4_POSITIONS))) return O_INVALID;
    g->base4 = 1;
    return O_OK;
}

/* Integer and decimal parts of every live edge, in the order of o_export_edges,
 * and the decimal total Q_D = sum of q per vertex. */
void o_export_real(const o_graph* g, uint32_t* I, uint32_t* q, uint64_t* qsum) {
    uint64_t p = 0;
    for (uint32_t v = 0; v < g->n; v++) {
        uint64_t s = 0;
        for (uint64_t j = 0; j < g->a[v].len; j++, p++) {
            uint32_t ii = 0, qq = 0;
            if (g->lam != 0.0) o_real_parts(g->a[v].e[j].w, g->lam, &ii, &qq);
            else ii = g->a[v].e[j].w;
            I[p] = ii;
            q[p] = qq;
            s += qq;
        }
        qsum[v] = s;
    }
}

/* 1 iff a live edge u -> x exists (linear scan). */
int o_has_edge(const o_graph* g, uint32_t u, uint32_t x) {
    const o_adj* a = &g->a[u];
    for (uint64_t j = 0; j < a->len; j++)
        if (a->e[j].dst == x) return 1;
    return 0;
}

/* ------------------------------------------------------------------------------ updates */

/*
 * Apply one batch.  rec is [count][4] = {src, dst, bias, op}; op 0 = insert,
 * 1 = delete (bias ignored), 2 = change bias, which is an insertion of
 * (src, dst, bias) plus a deletion of (src, dst) (Section 4.2: other updates
 * are built from insertions and deletions).
 * Order: all insertions in batch order (new edge ids continue after the
 * largest id ever assigned), then all deletions in batch order, each removing
 * the live copy of (src, dst) with the smallest edge id (Section 5.2).
 * A deletion that finds no copy changes nothing and is counted in not_found.
 * Validation (src, dst < n; 1 <= bias < 2^max_bits for insertions; op <= 2)
 * runs over the whole batch first; any failure returns O_INVALID and leaves
 * the graph unchanged.
 * stats (nullable) = {inserted, deleted, not_found}.
 */
typedef struct { uint32_t src; uint64_t idx; } o_del;
static int o_del_cmp(const void* a, const void* b) {
    const o_del* x = (const o_del*)a;
    const o_del* y = (const o_del*)b;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int o_u32_cmp(const void* a, const void* b) {
    const uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return x < y ? -1 : (x > y);
}

/* As o_apply, with the id of every insertion given: record i, if it inserts (op 0 or 2), adds edge
 * id ins_eid[i].  Ids must exceed every id of the record's source and increase in batch order per
 * source (o_apply passes next_eid, next_eid + 1, ... in batch order).
 * Deletions (Section 5.2): each removes the live copy of (src, dst) with the smallest edge id, in
 * batch order.  Deletions of different sources touch different lists and deletions of different
 * destinations of one source touch different copies, so a source whose batch deletes destination x
 * r times loses the r earliest live copies of x (all of them if it has fewer; the rest are not
 * found).  Each source is therefore applied in one pass over its list in edge-id order, dropping
 * an edge while its destination still has deletions left (sources in parallel). */
int o_apply_ids(o_graph* g, const uint32_t* rec, uint64_t count, uint32_t max_bits, const uint64_t* ins_eid,
                uint64_t* stats) {
    for (uint64_t i = 0; i < count; i++) {
        const uint32_t* r = rec + 4 * i;
        if (r[0] >= g->n || r[1] >= g->n || r[3] > 2) return O_INVALID;
        if (r[3] != 1) {
            if (g->lam != 0.0) {
                uint32_t I, q;
                if (o_real_parts(r[2], g->lam, &I, &q)) return O_INVALID;
                continue;
            }
            if (r[2] == 0) return O_INVALID;
            if (max_bits < 32 && (r[2] >> max_bits) != 0) return O_INVALID;
            if (g->base4 && r[2] >= (1u << (2 * O_B4_POSITIONS))) return O_INVALID;
        }
    }
    uint64_t ins = 0, del = 0, nf = 0, ndel = 0;
    for (uint64_t i = 0; i < count; i++) {
        const uint32_t* r = rec + 4 * i;
        if (r[3] == 0 || r[3] == 2) {
            o_edge x = {r[1], r[2], ins_eid[i]};
            if (adj_push(&g->a[r[0]], x) != O_OK) return O_NOMEM;
            if (ins_eid[i] >= g->next_eid) g->next_eid = ins_eid[i] + 1;
            ins++;
        }
        if (r[3] == 1 || r[3] == 2) ndel++;
    }
    o_del* dl = (o_del*)malloc(sizeof(o_del) * (ndel ? ndel : 1));
    uint32_t* dd = (uint32_t*)malloc(sizeof(uint32_t) * (ndel ? ndel : 1));
    uint64_t* run = (uint64_t*)malloc(sizeof(uint64_t) * (ndel + 1));
    if (!dl || !dd || !run) { free(dl); free(dd); free(run); return O_NOMEM; }
    uint64_t t = 0;
    for (uint64_t i = 0; i < count; i++)
        if (rec[4 * i + 3] == 1 || rec[4 * i + 3] == 2) { dl[t].src = rec[4 * i]; dl[t].idx = i; t++; }
    qsort(dl, ndel, sizeof(o_del), o_del_cmp); /* by source */
    uint64_t nrun = 0;
    for (uint64_t i = 0; i < ndel; i++) {
        if (i == 0 || dl[i].src != dl[i - 1].src) run[nrun++] = i;
        dd[i] = rec[4 * dl[i].idx + 1];
    }
    run[nrun] = ndel;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : del, nf)
    for (int64_t q = 0; q < (int64_t)nrun; q++) {
        /* this source's deleted destinations, sorted; left[k] deletions of dd[a + k] remain */
        const uint64_t a = run[q], k = run[q + 1] - run[q];
        uint32_t* xs = dd + a;
        qsort(xs, k, sizeof(uint32_t), o_u32_cmp);
        uint32_t* left = (uint32_t*)calloc(k, sizeof(uint32_t));
        uint64_t nu = 0;
        for (uint64_t j = 0; j < k; j++) {
            if (nu && xs[nu - 1] == xs[j]) { left[nu - 1]++; continue; }
            xs[nu] = xs[j];
            left[nu++] = 1;
        }
        o_adj* A = &g->a[dl[a].src];
        uint64_t w = 0;
        for (uint64_t j = 0; j < A->len; j++) {  /* ascending edge id */
            uint64_t lo = 0, hi = nu;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) / 2;
                if (xs[mid] < A->e[j].dst) lo = mid + 1; else hi = mid;
            }
            if (lo < nu && xs[lo] == A->e[j].dst && left[lo]) { left[lo]--; del++; continue; }
            A->e[w++] = A->e[j];
        }
        A->len = w;
        for (uint64_t j = 0; j < nu; j++) nf += left[j];
        free(left);
    }
    free(run);
    free(dd);
    free(dl);
    if (stats) { stats[0] = ins; stats[1] = del; stats[2] = nf; }
    return O_OK;
}

int o_apply(o_graph* g, const uint32_t* rec, uint64_t count, uint32_t max_bits, uint64_t* stats) {
    uint64_t* ids = (uint64_t*)malloc(sizeof(uint64_t) * (count ? count : 1));
    if (!ids) return O_NOMEM;
    uint64_t next = g->next_eid;
    for (uint64_t i = 0; i < count; i++) ids[i] = (rec[4 * i + 3] == 0 || rec[4 * i + 3] == 2) ? next++ : 0;
    const int rc = o_apply_ids(g, rec, count, max_bits, ids, stats);
    free(ids);
    return rc;
}

/* Export the live edges of the listed vertices (row i = ids[i]) in ascending edge-id order;
 * offs has count+1 entries. */
void o_edges_of(const o_graph* g, const uint32_t* ids, uint64_t count, uint64_t* offs, uint32_t* dst, uint32_t* w,
                uint64_t* eid) {
    uint64_t p = 0;
    for (uint64_t i = 0; i < count; i++) {
        const o_adj* a = &g->a[ids[i]];
        offs[i] = p;
        for (uint64_t j = 0; j < a->len; j++, p++) {
            dst[p] = a->e[j].dst;
            w[p] = a->e[j].w;
            eid[p] = a->e[j].eid;
        }
    }
    offs[count] = p;
}

/* Live copies of (us[i], xs[i]) for i < count: each source's list is sorted once by destination
 * (a copy) and searched for its queries (sources in parallel). */
typedef struct { uint32_t u; uint64_t i; } o_query;
static int o_query_cmp(const void* a, const void* b) {
    const o_query* x = (const o_query*)a;
    const o_query* y = (const o_query*)b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    return x->i < y->i ? -1 : (x->i > y->i);
}
void o_count_edges(const o_graph* g, const uint32_t* us, const uint32_t* xs, uint64_t count, uint32_t* out) {
    o_query* q = (o_query*)malloc(sizeof(o_query) * (count ? count : 1));
    uint64_t* run = (uint64_t*)malloc(sizeof(uint64_t) * (count + 1));
    for (uint64_t i = 0; i < count; i++) { q[i].u = us[i]; q[i].i = i; }
    qsort(q, count, sizeof(o_query), o_query_cmp);
    uint64_t nrun = 0;
    for (uint64_t i = 0; i < count; i++)
        if (i == 0 || q[i].u != q[i - 1].u) run[nrun++] = i;
    run[nrun] = count;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < (int64_t)nrun; r++) {
        const uint32_t u = q[run[r]].u;
        const o_adj* A = u < g->n ? &g->a[u] : NULL;
        const uint64_t d = A ? A->len : 0;
        uint32_t* row = (uint32_t*)malloc(sizeof(uint32_t) * (d ? d : 1));
        for (uint64_t j = 0; j < d; j++) row[j] = A->e[j].dst;
        qsort(row, d, sizeof(uint32_t), o_u32_cmp);
        for (uint64_t t = run[r]; t < run[r + 1]; t++) {
            const uint32_t x = xs[q[t].i];
            uint64_t lo = 0, hi = d;
            while (lo < hi) { const uint64_t mid = (lo + hi) / 2; if (row[mid] < x) lo = mid + 1; else hi = mid; }
            uint64_t b = lo;
            hi = d;
            while (b < hi) { const uint64_t mid = (b + hi) / 2; if (row[mid] <= x) b = mid + 1; else hi = mid; }
            out[q[t].i] = (uint32_t)(b - lo);
        }
        free(row);
    }
    free(run);
    free(q);
}

uint64_t o_degree_sum(const o_graph* g, const uint32_t* ids, uint64_t count) {
    uint64_t s = 0;
    for (uint64_t i = 0; i < count; i++) s += g->a[ids[i]].len;
    return s;
}

/* ------------------------------------------------------------------------------ factorisation */

/* Eq. group, evaluated in its printed order (first match wins), with percent
 * thresholds compared in integers: dense iff |G|/d > alpha%, one-element iff
 * |G| = 1, sparse iff |G|/d < beta% (and |G| != 1), regular otherwise.
 * alpha = O_ALL_REGULAR turns group adaption off (every nonempty group regular). */
#define O_ALL_REGULAR 0xFFFFFFFFu /* alpha value selecting the paper's BS baseline (Section 6.2,
                                     Fig. Moptimization): every nonempty group in regular format */
int o_kind(uint64_t cnt, uint64_t d, uint32_t alpha, uint32_t beta) {
    if (cnt == 0) return O_EMPTY;
    if (alpha == O_ALL_REGULAR) return O_REGULAR;
    if (100 * cnt > (uint64_t)alpha * d) return O_DENSE;
    if (cnt == 1) return O_ONE;
    if (100 * cnt < (uint64_t)beta * d) return O_SPARSE;
    return O_REGULAR;
}

/* For vertex v: |G_k| for k < 32 (Eq. dwi: edge i is in group k iff w_i AND 2^k != 0,
 * w_i the integer part for real biases), the kinds of Eq. group, and the sum of the
 * sampling weights. */
void o_factor(const o_graph* g, uint32_t v, uint32_t alpha, uint32_t beta, uint32_t* cnt, uint8_t* kind,
              uint64_t* sumw) {
    const o_adj* a = &g->a[v];
    uint64_t s = 0;
    for (int k = 0; k < 32; k++) cnt[k] = 0;
    for (uint64_t j = 0; j < a->len; j++) {
        s += o_weight(g, a->e[j].w);
        for (int k = 0; k < 32; k++)
            if (o_in_slot(g, a->e[j].w, k)) cnt[k]++;
    }
    for (int k = 0; k < 32; k++) kind[k] = (uint8_t)o_kind(cnt[k], a->len, alpha, beta);
    *sumw = s;
}

void o_factor_all(const o_graph* g, uint32_t alpha, uint32_t beta, uint32_t* cnt, uint8_t* kind, uint64_t* sumw) {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < (int64_t)g->n; v++)
        o_factor(g, (uint32_t)v, alpha, beta, cnt + 32 * v, kind + 32 * v, sumw + v);
}

/* Group totals W(p_k) = sum_i (w_i AND 2^k) (Eq. wpk), summed directly.  For real
 * biases, in units of 2^-8 (each integer part counts 2^8 times) and W[31] is the
 * decimal group's total Q_D. */
void o_group_totals(const o_graph* g, uint32_t v, uint64_t* W) {
    const o_adj* a = &g->a[v];
    const int sh = g->lam != 0.0 ? O_FRAC_BITS : 0;
    for (int k = 0; k < 32; k++) {
        uint64_t s = 0;
        if (g->base4) {  /* sum of the digit values v * 4^i the members contribute */
            for (uint64_t j = 0; j < a->len; j++)
                if (o_in_slot(g, a->e[j].w, k)) s += o_slot_unit(g, k);
        } else {
            for (uint64_t j = 0; j < a->len; j++) s += (uint64_t)(o_int_part(g, a->e[j].w) & (1u << k)) << sh;
        }
        W[k] = s;
    }
    if (sh) {
        uint64_t s = 0;
        for (uint64_t j = 0; j < a->len; j++) s += o_dec_part(g, a->e[j].w);
        W[31] = s;
    }
}

/* Group membership for every (v, k) as ascending edge ids.  offs has 32n+1
 * entries; entries of (v, k) are eids[offs[32v+k] .. offs[32v+k+1]). */
uint64_t o_members_count(const o_graph* g) {
    uint64_t t = 0;
    for (uint32_t v = 0; v < g->n; v++)
        for (uint64_t j = 0; j < g->a[v].len; j++)
            for (int k = 0; k < 32; k++) t += (uint64_t)o_in_slot(g, g->a[v].e[j].w, k);
    return t;
}

void o_members_all(const o_graph* g, uint64_t* offs, uint64_t* eids) {
    uint64_t p = 0;
    for (uint32_t v = 0; v < g->n; v++) {
        const o_adj* a = &g->a[v];
        for (int k = 0; k < 32; k++) {
            offs[32 * (uint64_t)v + k] = p;
            for (uint64_t j = 0; j < a->len; j++)
                if (o_in_slot(g, a->e[j].w, k)) eids[p++] = a->e[j].eid;
        }
    }
    offs[32 * (uint64_t)g->n] = p;
}

/* ------------------------------------------------------------------------------ exact probabilities */

static unsigned __int128 gcd128(unsigned __int128 a, unsigned __int128 b) {
    while (b) { unsigned __int128 t = a % b; a = b; b = t; }
    return a;
}

/*
 * Probability that the factorised sampler returns neighbour index i of v, as
 * a reduced fraction num/den: sum over the groups k containing i of
 * P(p_k) * P(v_i | p_k), with P(p_k) = W(p_k) / sum_j W(p_j) (Eq. group_prob)
 * and P(v_i | p_k) uniform over G_k (Eq. pvp).  A dense group reaches its
 * members by rejection on the whole neighbour list (Section 5.1): one trial
 * picks i with probability 1/d and succeeds with probability |G_k|/d, so the
 * conditional probability is (1/d) / (|G_k|/d), summed here as that ratio.
 * Base 4 (Appendix): slot 3 i + v - 1 carries v * 4^i |S_iv|, so choosing it is choosing group
 * 4^i and then its value sub-group v; the member is uniform within the sub-group.
 * Real biases (Section 4.3): the integer groups carry W(p_k) = 2^8 * 2^k |G_k|
 * (units of 2^-8) and the decimal group D carries Q_D = sum of the decimal parts
 * q_j; within D, neighbour i is drawn with probability q_i / Q_D (step (iii):
 * ITS or rejection over the decimal parts), so its term is Q_D/tot * q_i/Q_D.
 * Returns 0 on success, 1 if the vertex has no edges.
 */
int o_factored_prob(const o_graph* g, uint32_t v, uint64_t i, uint32_t alpha, uint32_t beta, uint64_t* num,
                    uint64_t* den) {
    uint32_t cnt[32];
    uint8_t kind[32];
    uint64_t sw;
    o_factor(g, v, alpha, beta, cnt, kind, &sw);
    const o_adj* a = &g->a[v];
    if (a->len == 0) return 1;
    const int sh = g->lam != 0.0 ? O_FRAC_BITS : 0;
    uint64_t W[32], tot = 0, QD = 0;
    for (int k = 0; k < 32; k++) { W[k] = (uint64_t)cnt[k] * o_slot_unit(g, k); tot += W[k]; }
    if (sh) {
        for (uint64_t j = 0; j < a->len; j++) QD += o_dec_part(g, a->e[j].w);
        tot += QD;
    }
    unsigned __int128 pn = 0, pd = 1;
    for (int k = 0; k < 32; k++) {
        if (!o_in_slot(g, a->e[i].w, k)) continue;
        /* term = (W_k / tot) * q_k where q_k is the within-group probability */
        unsigned __int128 qn, qd;
        if (kind[k] == O_DENSE) { /* (1/d) / (cnt/d) */
            qn = (unsigned __int128)1 * a->len;
            qd = (unsigned __int128)a->len * cnt[k];
        } else {
            qn = 1;
            qd = cnt[k];
        }
        unsigned __int128 tn = (unsigned __int128)W[k] * qn, td = (unsigned __int128)tot * qd;
        unsigned __int128 t = gcd128(tn, td);
        tn /= t; td /= t;
        pn = pn * td + tn * pd;
        pd = pd * td;
        t = gcd128(pn, pd);
        pn /= t; pd /= t;
    }
    const uint32_t qi = o_dec_part(g, a->e[i].w);
    if (qi) { /* decimal group: (Q_D / tot) * (q_i / Q_D) */
        unsigned __int128 tn = (unsigned __int128)QD * qi, td = (unsigned __int128)tot * QD;
        unsigned __int128 t = gcd128(tn, td);
        tn /= t; td /= t;
        pn = pn * td + tn * pd;
        pd = pd * td;
        t = gcd128(pn, pd);
        pn /= t; pd /= t;
    }
    *num = (uint64_t)pn;
    *den = (uint64_t)pd;
    return 0;
}

/* ------------------------------------------------------------------------------ sampling */

/* Oracle randomness: a counter hash (splitmix64 finaliser chain). */
static inline uint64_t o_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
typedef struct { uint64_t seed, walker, ctr; } o_rng;
static inline uint64_t o_next(o_rng* r) {
    return o_mix(o_mix(o_mix(r->seed) ^ r->walker) + r->ctr++);
}
/* Uniform in [0, range), range >= 1: reject the top partial block, then reduce. */
static inline uint64_t o_below(o_rng* r, uint64_t range) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % range + 1) % range; /* largest multiple of range, minus 1 */
    uint64_t x;
    do { x = o_next(r); } while (x > lim);
    return x % range;
}

/* ITS: smallest index j with r < c[j], where c is the inclusive prefix sum of
 * the weights (c[d-1] = total), found by binary search. */
static uint64_t its_search(const uint64_t* c, uint64_t d, uint64_t r) {
    uint64_t lo = 0, hi = d - 1;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (r < c[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

/* Neighbour index picked by ITS for a given r in [0, sum w) at vertex v. */
uint64_t o_its_pick(const o_graph* g, uint32_t v, uint64_t r) {
    const o_adj* a = &g->a[v];
    uint64_t* c = (uint64_t*)malloc(sizeof(uint64_t) * (a->len ? a->len : 1));
    uint64_t s = 0;
    for (uint64_t j = 0; j < a->len; j++) { s += o_weight(g, a->e[j].w); c[j] = s; }
    uint64_t j = its_search(c, a->len, r);
    free(c);
    return j;
}

/* node2vec distance (Eq. node2vec): 0 if x is prev, 1 if an edge prev -> x is live, 2 otherwise. */
static int n2v_dist(const o_graph* g, uint32_t prev, uint32_t x) {
    if (x == prev) return 0;
    return o_has_edge(g, prev, x) ? 1 : 2;
}

/* Unnormalised second-order weights at u after prev: w_ux * a[dist(prev, x)],
 * where a[] are the acceptance thresholds f/max f scaled by 2^32. */
void o_n2v_weights(const o_graph* g, uint32_t prev, uint32_t u, const uint64_t* a, uint64_t* out) {
    const o_adj* A = &g->a[u];
    for (uint64_t j = 0; j < A->len; j++) out[j] = o_weight(g, A->e[j].w) * a[n2v_dist(g, prev, A->e[j].dst)];
}

typedef struct {
    uint32_t kind;          /* O_DEEPWALK, O_PPR, O_NODE2VEC */
    uint32_t max_len;       /* steps */
    uint32_t ppr_stop_u32;  /* stop iff a uniform u32 < this, checked before every step */
    uint32_t pad;
    uint64_t n2v_accept[3]; /* f(dist)/max f scaled to [0, 2^32], dist 0/1/2 */
} o_policy;

/*
 * Walks.  paths is [nwalkers][stride] (stride >= longest length + 1), padded
 * with 0xFFFFFFFF; path_len[i] counts vertices including the start.
 * A walk of length L takes L sampled steps; a vertex without out-edges ends it.
 * PPR: before every step, stop with probability ppr_stop_u32 / 2^32.
 * node2vec: the first step is first-order; later steps sample x with
 * probability proportional to w_ux * f(prev, x) (Eq. node2vec), normalised.
 */
void o_walk(const o_graph* g, uint64_t nwalkers, const uint32_t* starts, const uint32_t* lengths,
            const uint8_t* policy_ids, const o_policy* pol, uint64_t seed, uint64_t stride, uint32_t* paths,
            uint32_t* path_len) {
    /* prefix sums of the biases, per vertex, for first-order ITS */
    uint64_t* off = (uint64_t*)malloc(sizeof(uint64_t) * ((uint64_t)g->n + 1));
    off[0] = 0;
    for (uint32_t v = 0; v < g->n; v++) off[v + 1] = off[v] + g->a[v].len;
    uint64_t* c = (uint64_t*)malloc(sizeof(uint64_t) * (off[g->n] ? off[g->n] : 1));
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < (int64_t)g->n; v++) {
        uint64_t s = 0;
        for (uint64_t j = 0; j < g->a[v].len; j++) { s += o_weight(g, g->a[v].e[j].w); c[off[v] + j] = s; }
    }
#pragma omp parallel
    {
        uint64_t wcap = 0;
        uint64_t* wbuf = NULL;
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < (int64_t)nwalkers; i++) {
            const o_policy* P = &pol[policy_ids ? policy_ids[i] : 0];
            uint32_t L = lengths ? lengths[i] : P->max_len;
            uint32_t* row = paths + (uint64_t)i * stride;
            o_rng rng = {seed, (uint64_t)i, 0};
            uint32_t u = starts[i], prev = O_PAD;
            uint32_t len = 0;
            row[len++] = u;
            for (uint32_t s = 0; s < L; s++) {
                if (P->kind == O_PPR && (uint32_t)(o_next(&rng) >> 32) < P->ppr_stop_u32) break;
                const o_adj* A = &g->a[u];
                if (A->len == 0) break;
                uint64_t j;
                if (P->kind == O_NODE2VEC && prev != O_PAD) {
                    if (A->len > wcap) {
                        wcap = A->len;
                        wbuf = (uint64_t*)realloc(wbuf, sizeof(uint64_t) * wcap);
                    }
                    o_n2v_weights(g, prev, u, P->n2v_accept, wbuf);
                    uint64_t tot = 0;
                    for (uint64_t t = 0; t < A->len; t++) { tot += wbuf[t]; wbuf[t] = tot; }
                    if (tot == 0) break;
                    j = its_search(wbuf, A->len, o_below(&rng, tot));
                } else {
                    const uint64_t* cv = c + off[u];
                    j = its_search(cv, A->len, o_below(&rng, cv[A->len - 1]));
                }
                prev = u;
                u = A->e[j].dst;
                row[len++] = u;
            }
            path_len[i] = len;
            for (uint64_t t = len; t < stride; t++) row[t] = O_PAD;
        }
        free(wbuf);
    }
    free(c);
    free(off);
}

/* One-step samples from a single vertex: out[t] = neighbour index drawn by ITS. */
void o_sample_many(const o_graph* g, uint32_t v, uint64_t count, uint64_t seed, uint64_t* out) {
    const o_adj* a = &g->a[v];
    uint64_t* c = (uint64_t*)malloc(sizeof(uint64_t) * (a->len ? a->len : 1));
    uint64_t s = 0;
    for (uint64_t j = 0; j < a->len; j++) { s += o_weight(g, a->e[j].w); c[j] = s; }
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < (int64_t)count; t++) {
        o_rng r = {seed, (uint64_t)t, 0};
        out[t] = its_search(c, a->len, o_below(&r, s));
    }
    free(c);
}

/* Threads for the OpenMP loops (walkers, per-source deletions); the bench times the oracle at one
 * thread and at all host cores. */
void o_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int o_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------ float biases */

/*
 * Floating-point biases with amortisation factor lambda (Section 4.3): each
 * bias b is scaled to lambda*b, split into an integer part I = floor(lambda*b)
 * and a decimal part lambda*b - I.  The integer parts are radix-decomposed
 * (group k holds edges with bit k of I set); the decimal parts form one extra
 * group.  Outputs: cnt[32] of the integer groups, the decimal-group size, and
 * W_I = sum I, W_D = sum of decimal parts (as doubles).
 */
void o_float_factor(uint64_t d, const double* b, double lambda, uint32_t* cnt, uint64_t* n_dec, double* WI,
                    double* WD) {
    double wi = 0, wd = 0;
    uint64_t nd = 0;
    for (int k = 0; k < 32; k++) cnt[k] = 0;
    for (uint64_t j = 0; j < d; j++) {
        double x = lambda * b[j];
        double ip = floor(x);
        uint32_t I = (uint32_t)ip;
        double dp = x - ip;
        for (int k = 0; k < 32; k++)
            if (I & (1u << k)) cnt[k]++;
        wi += ip;
        wd += dp;
        if (dp > 0) nd++;
    }
    *n_dec = nd;
    *WI = wi;
    *WD = wd;
}
