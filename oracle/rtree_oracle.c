/*
 * rtree_oracle.c -- scalar CPU oracle for R-tree range select and R-tree join.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  The CUDA path never calls
 * it, and this file shares no code, header or constant with the CUDA path.
 *
 * What it computes (arXiv 2309.16913, "SIMD-ified R-tree Query Processing
 * and Optimization"):
 *
 *   select(q) = { id_i : R_i intersects q }      (Section 3, spatial select)
 *   join(R,S) = { (r_id, s_id) : R_r intersects S_s }  (Section 4, R-tree join)
 *
 * with the closed-interval intersection predicate
 *
 *   a.lx <= b.hx  &&  b.lx <= a.hx  &&  a.ly <= b.hy  &&  b.ly <= a.hy
 *
 * (Section 4.1 step 3 states the disjointness tests; touching rectangles
 * count as intersecting here, and the four tests are combined with logical
 * '&&' as in the scalar select variant of Section 3).  Results are returned
 * sorted: ids ascending per query, pairs lexicographically.
 *
 * Structure, in the paper's order:
 *   - node = up to F entries (MBR, ptr) plus depth and count (Section 2.3);
 *   - select: recursive depth-first descent from the root following every
 *     entry whose MBR meets the query (the scalar algorithm of Section 3);
 *   - join: synchronized top-down traversal of both trees from the roots,
 *     following entry pairs that intersect (Section 4, after Brinkhoff,
 *     Kriegel and Seeger 1993); where heights differ only the deeper tree
 *     descends, its entries tested against the other node's MBR;
 *   - brute force: nested loops over all rectangles (the plain definition).
 *
 * The paper does not say how the tree is built.  This oracle bulk-loads it
 * with Sort-Tile-Recursive (Leutenegger, Lopez and Edgington 1997):
 *   m items, P = ceil(m/F) nodes, S = ceil(sqrt(P)) slabs of S*F items;
 *   order A: sort by (kx, item index), kx = lx + hx in float32;
 *   slab(item) = rank in A / (S*F);
 *   order B: sort by (slab, ky, item index), ky = ly + hy in float32;
 *   node k takes items B[kF .. kF+F-1] (the last node may be partial);
 *   repeat on the node MBRs until one node remains (the root).
 * A centre key that is NaN (only -inf + inf) counts as 0, and -0 counts as
 * +0.  Query results do not depend on the tree at all; the build is fixed
 * only so that a tree built elsewhere can be compared node by node.
 *
 * For timing on all host cores, orc_select_mt and orc_join_mt run the same
 * scalar routines on contiguous chunks of the queries (or of the join's
 * top-level node pairs) in POSIX threads, each into its own output, and
 * concatenate the outputs; threads share nothing but the read-only trees.
 *
 * Compile with -O2 -fno-fast-math -ffp-contract=off: float32 sums and
 * comparisons must follow IEEE 754 exactly.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float lx, ly, hx, hy;
} box;

/* Closed-interval intersection, logical form. */
static int intersects(box a, box b)
{
    return a.lx <= b.hx && b.lx <= a.hx && a.ly <= b.hy && b.ly <= a.hy;
}

/* ---------------------------------------------------------------- buffers */

typedef struct {
    int32_t *v;
    int64_t n, cap;
} ivec;

static int ivec_push(ivec *a, int32_t x)
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? a->cap * 2 : 64;
        int32_t *p = (int32_t *)realloc(a->v, (size_t)nc * sizeof(int32_t));
        if (!p)
            return -1;
        a->v = p;
        a->cap = nc;
    }
    a->v[a->n++] = x;
    return 0;
}

static int cmp_i32(const void *p, const void *q)
{
    int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
    return (a > b) - (a < b);
}

static int cmp_pair(const void *p, const void *q)
{
    const int32_t *a = (const int32_t *)p, *b = (const int32_t *)q;
    if (a[0] != b[0])
        return (a[0] > b[0]) - (a[0] < b[0]);
    return (a[1] > b[1]) - (a[1] < b[1]);
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------- tree */

typedef struct onode {
    int height;           /* 0 = leaf */
    int count;            /* entries in use, 1..F */
    box *mbr;             /* entry MBRs */
    struct onode **child; /* height > 0 */
    int32_t *id;          /* height == 0 */
} onode;

typedef struct {
    int fanout;
    int sorted; /* entries of every node ascending by lx (Section 4.2 pruning) */
    int levels; /* 0 for an empty tree */
    int64_t n;
    onode *root;
    box root_mbr;
    onode **all;
    int64_t n_nodes;
} otree;

static float centre_key(float lo, float hi)
{
    float k = lo + hi;
    if (k != k)
        k = 0.0f;
    if (k == 0.0f)
        k = 0.0f; /* -0 -> +0 */
    return k;
}

static int64_t ceil_sqrt(int64_t p)
{
    int64_t s = (int64_t)sqrt((double)p);
    while (s * s < p)
        s++;
    while (s > 1 && (s - 1) * (s - 1) >= p)
        s--;
    return s;
}

typedef struct {
    float k;
    int64_t slab;
    int64_t idx;
} skey;

static int cmp_key_idx(const void *p, const void *q)
{
    const skey *a = (const skey *)p, *b = (const skey *)q;
    if (a->k < b->k)
        return -1;
    if (a->k > b->k)
        return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int cmp_slab_key_idx(const void *p, const void *q)
{
    const skey *a = (const skey *)p, *b = (const skey *)q;
    if (a->slab != b->slab)
        return (a->slab > b->slab) - (a->slab < b->slab);
    return cmp_key_idx(p, q);
}

/* STR packing order of m items: order[r] = item placed at position r. */
static int str_order(const box *b, int64_t m, int F, int64_t *order)
{
    int64_t P = (m + F - 1) / F;
    int64_t S = ceil_sqrt(P);
    int64_t cap = S * (int64_t)F;
    skey *t = (skey *)malloc((size_t)m * sizeof(skey));
    int64_t *slab = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    if (!t || !slab) {
        free(t);
        free(slab);
        return -1;
    }
    for (int64_t i = 0; i < m; i++) {
        t[i].k = centre_key(b[i].lx, b[i].hx);
        t[i].slab = 0;
        t[i].idx = i;
    }
    qsort(t, (size_t)m, sizeof(skey), cmp_key_idx);
    for (int64_t r = 0; r < m; r++)
        slab[t[r].idx] = r / cap;
    for (int64_t i = 0; i < m; i++) {
        t[i].k = centre_key(b[i].ly, b[i].hy);
        t[i].slab = slab[i];
        t[i].idx = i;
    }
    qsort(t, (size_t)m, sizeof(skey), cmp_slab_key_idx);
    for (int64_t r = 0; r < m; r++)
        order[r] = t[r].idx;
    free(t);
    free(slab);
    return 0;
}

static box node_mbr(const onode *nd)
{
    box r = nd->mbr[0];
    for (int e = 1; e < nd->count; e++) {
        box c = nd->mbr[e];
        if (c.lx < r.lx) r.lx = c.lx;
        if (c.ly < r.ly) r.ly = c.ly;
        if (c.hx > r.hx) r.hx = c.hx;
        if (c.hy > r.hy) r.hy = c.hy;
    }
    return r;
}

static void free_nodes(onode **all, int64_t n)
{
    for (int64_t i = 0; i < n; i++) {
        if (!all[i])
            continue;
        free(all[i]->mbr);
        free(all[i]->child);
        free(all[i]->id);
        free(all[i]);
    }
    free(all);
}

void orc_tree_free(otree *t)
{
    if (!t)
        return;
    free_nodes(t->all, t->n_nodes);
    free(t);
}

/*
 * Section 4.2 assumes the entries of every node are ordered by one MBR key,
 * lx.  With sort_children set, each node's entries are put in ascending lx
 * order once the node is packed (equal lx, including -0 against +0, keep
 * their packing order): an insertion sort, so it is stable.  Which items
 * share a node, and so every node MBR, is unchanged.
 */
static void sort_entries_by_lx(onode *nd)
{
    for (int e = 1; e < nd->count; e++) {
        box b = nd->mbr[e];
        int32_t id = nd->height == 0 ? nd->id[e] : 0;
        onode *ch = nd->height == 0 ? NULL : nd->child[e];
        int k = e - 1;
        while (k >= 0 && nd->mbr[k].lx > b.lx) {
            nd->mbr[k + 1] = nd->mbr[k];
            if (nd->height == 0)
                nd->id[k + 1] = nd->id[k];
            else
                nd->child[k + 1] = nd->child[k];
            k--;
        }
        nd->mbr[k + 1] = b;
        if (nd->height == 0)
            nd->id[k + 1] = id;
        else
            nd->child[k + 1] = ch;
    }
}

/* Bulk-load with STR.  rects: n x [xmin, ymin, xmax, ymax]; ids: n. */
otree *orc_tree_build2(const float *rects, const int32_t *ids, int64_t n, int fanout,
                       int sort_children)
{
    if (fanout < 2 || n < 0)
        return NULL;
    otree *t = (otree *)calloc(1, sizeof(otree));
    if (!t)
        return NULL;
    t->fanout = fanout;
    t->sorted = sort_children != 0;
    t->n = n;
    if (n == 0)
        return t;

    /* total node count is bounded by n (each level at most halves) */
    int64_t cap_nodes = 0, m = n;
    do {
        m = (m + fanout - 1) / fanout;
        cap_nodes += m;
    } while (m > 1);
    t->all = (onode **)calloc((size_t)cap_nodes, sizeof(onode *));
    if (!t->all) {
        free(t);
        return NULL;
    }

    /* level 0 items: the data rectangles */
    m = n;
    box *b = (box *)malloc((size_t)m * sizeof(box));
    onode **items = NULL; /* payload of higher levels */
    if (!b)
        goto fail;
    for (int64_t i = 0; i < n; i++) {
        b[i].lx = rects[4 * i + 0];
        b[i].ly = rects[4 * i + 1];
        b[i].hx = rects[4 * i + 2];
        b[i].hy = rects[4 * i + 3];
    }
    int height = 0;
    for (;;) {
        int64_t P = (m + fanout - 1) / fanout;
        int64_t *order = (int64_t *)malloc((size_t)m * sizeof(int64_t));
        onode **nodes = (onode **)calloc((size_t)P, sizeof(onode *));
        box *nb = (box *)malloc((size_t)P * sizeof(box));
        if (!order || !nodes || !nb || str_order(b, m, fanout, order)) {
            free(order);
            free(nodes);
            free(nb);
            goto fail;
        }
        for (int64_t k = 0; k < P; k++) {
            int64_t lo = k * fanout, hi = lo + fanout < m ? lo + fanout : m;
            onode *nd = (onode *)calloc(1, sizeof(onode));
            if (!nd)
                goto fail_level;
            t->all[t->n_nodes++] = nd;
            nodes[k] = nd;
            nd->height = height;
            nd->count = (int)(hi - lo);
            nd->mbr = (box *)malloc((size_t)nd->count * sizeof(box));
            if (height == 0)
                nd->id = (int32_t *)malloc((size_t)nd->count * sizeof(int32_t));
            else
                nd->child = (onode **)malloc((size_t)nd->count * sizeof(onode *));
            if (!nd->mbr || (height == 0 ? !nd->id : !nd->child))
                goto fail_level;
            for (int64_t r = lo; r < hi; r++) {
                int64_t it = order[r];
                nd->mbr[r - lo] = b[it];
                if (height == 0)
                    nd->id[r - lo] = ids[it];
                else
                    nd->child[r - lo] = items[it];
            }
            if (t->sorted)
                sort_entries_by_lx(nd);
            nb[k] = node_mbr(nd);
        }
        free(order);
        free(b);
        free(items);
        b = nb;
        items = nodes;
        m = P;
        height++;
        if (P == 1)
            break;
        continue;
    fail_level:
        free(order);
        free(nodes);
        free(nb);
        goto fail;
    }
    t->root = items[0];
    t->root_mbr = b[0];
    t->levels = height;
    free(b);
    free(items);
    return t;
fail:
    free(b);
    free(items);
    orc_tree_free(t);
    return NULL;
}

otree *orc_tree_build(const float *rects, const int32_t *ids, int64_t n, int fanout)
{
    return orc_tree_build2(rects, ids, n, fanout, 0);
}

int orc_tree_levels(const otree *t) { return t ? t->levels : 0; }
int64_t orc_tree_nodes(const otree *t) { return t ? t->n_nodes : 0; }

/*
 * Export the tree level by level from the root.  Within a level, nodes come
 * in the order their parents list them; a node's entries keep their packing
 * order.  Outputs (caller-allocated):
 *   level_nodes[levels]  nodes per level, root level first;
 *   counts[M]            entries per node;
 *   mbrs[M * F * 4]      entry MBRs, unused slots = (+inf, +inf, -inf, -inf);
 *   leaf_ids[n]          ids of leaf entries, leaves in export order.
 */
int orc_tree_export(const otree *t, int64_t *level_nodes, int32_t *counts, float *mbrs,
                    int32_t *leaf_ids)
{
    if (!t || t->levels == 0)
        return 0;
    int F = t->fanout;
    const onode **cur = (const onode **)malloc((size_t)t->n_nodes * sizeof(onode *));
    const onode **nxt = (const onode **)malloc((size_t)t->n_nodes * sizeof(onode *));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return -1;
    }
    int64_t nc = 1, g = 0, li = 0;
    cur[0] = t->root;
    for (int lv = 0; lv < t->levels; lv++) {
        level_nodes[lv] = nc;
        int64_t nn = 0;
        for (int64_t k = 0; k < nc; k++, g++) {
            const onode *nd = cur[k];
            counts[g] = nd->count;
            for (int e = 0; e < F; e++) {
                float *o = mbrs + ((size_t)g * F + e) * 4;
                if (e < nd->count) {
                    o[0] = nd->mbr[e].lx;
                    o[1] = nd->mbr[e].ly;
                    o[2] = nd->mbr[e].hx;
                    o[3] = nd->mbr[e].hy;
                } else {
                    o[0] = INFINITY;
                    o[1] = INFINITY;
                    o[2] = -INFINITY;
                    o[3] = -INFINITY;
                }
                if (e < nd->count) {
                    if (nd->height == 0)
                        leaf_ids[li++] = nd->id[e];
                    else
                        nxt[nn++] = nd->child[e];
                }
            }
        }
        const onode **sw = cur;
        cur = nxt;
        nxt = sw;
        nc = nn;
    }
    free(cur);
    free(nxt);
    return 0;
}

/* ----------------------------------------------------------------- select */

static int select_rec(const onode *nd, box q, ivec *out)
{
    for (int e = 0; e < nd->count; e++) {
        box c = nd->mbr[e];
        if (c.lx <= q.hx && q.lx <= c.hx && c.ly <= q.hy && q.ly <= c.hy) {
            if (nd->height == 0) {
                if (ivec_push(out, nd->id[e]))
                    return -1;
            } else if (select_rec(nd->child[e], q, out)) {
                return -1;
            }
        }
    }
    return 0;
}

/*
 * Range select for a batch of queries.  offsets[Q+1] receives CSR offsets;
 * *ids_out receives a malloc'd array of all ids (free with orc_free), each
 * query's ids sorted ascending.  Returns the total, or -1 on failure.
 */
int64_t orc_select(const otree *t, const float *queries, int64_t Q, int64_t *offsets,
                   int32_t **ids_out)
{
    ivec out = {0, 0, 0};
    offsets[0] = 0;
    for (int64_t i = 0; i < Q; i++) {
        box q = {queries[4 * i], queries[4 * i + 1], queries[4 * i + 2], queries[4 * i + 3]};
        int64_t start = out.n;
        if (t && t->root && select_rec(t->root, q, &out)) {
            free(out.v);
            return -1;
        }
        qsort(out.v + start, (size_t)(out.n - start), sizeof(int32_t), cmp_i32);
        offsets[i + 1] = out.n;
    }
    *ids_out = out.v;
    return out.n;
}

/* Brute-force range select: every rectangle against every query. */
int64_t orc_brute_select(const float *rects, const int32_t *ids, int64_t n,
                         const float *queries, int64_t Q, int64_t *offsets, int32_t **ids_out)
{
    ivec out = {0, 0, 0};
    offsets[0] = 0;
    for (int64_t i = 0; i < Q; i++) {
        box q = {queries[4 * i], queries[4 * i + 1], queries[4 * i + 2], queries[4 * i + 3]};
        int64_t start = out.n;
        for (int64_t k = 0; k < n; k++) {
            box r = {rects[4 * k], rects[4 * k + 1], rects[4 * k + 2], rects[4 * k + 3]};
            if (intersects(r, q) && ivec_push(&out, ids[k])) {
                free(out.v);
                return -1;
            }
        }
        qsort(out.v + start, (size_t)(out.n - start), sizeof(int32_t), cmp_i32);
        offsets[i + 1] = out.n;
    }
    *ids_out = out.v;
    return out.n;
}

/* ------------------------------------------------------------------- join */

static int emit_pair(ivec *out, int32_t r, int32_t s)
{
    return ivec_push(out, r) || ivec_push(out, s) ? -1 : 0;
}

static int join_rec(const onode *a, box amb, const onode *b, box bmb, ivec *out)
{
    if (a->height == b->height) {
        for (int i = 0; i < a->count; i++) {
            for (int j = 0; j < b->count; j++) {
                if (!intersects(a->mbr[i], b->mbr[j]))
                    continue;
                if (a->height == 0) {
                    if (emit_pair(out, a->id[i], b->id[j]))
                        return -1;
                } else if (join_rec(a->child[i], a->mbr[i], b->child[j], b->mbr[j], out)) {
                    return -1;
                }
            }
        }
    } else if (a->height > b->height) {
        for (int i = 0; i < a->count; i++)
            if (intersects(a->mbr[i], bmb) && join_rec(a->child[i], a->mbr[i], b, bmb, out))
                return -1;
    } else {
        for (int j = 0; j < b->count; j++)
            if (intersects(amb, b->mbr[j]) && join_rec(a, amb, b->child[j], b->mbr[j], out))
                return -1;
    }
    return 0;
}

/*
 * R-tree join.  *pairs_out receives a malloc'd int32 array of 2*total
 * values, (r_id, s_id) pairs sorted lexicographically.  Returns the number
 * of pairs, or -1 on failure.
 */
int64_t orc_join(const otree *r, const otree *s, int32_t **pairs_out)
{
    ivec out = {0, 0, 0};
    if (r && s && r->root && s->root &&
        join_rec(r->root, r->root_mbr, s->root, s->root_mbr, &out)) {
        free(out.v);
        return -1;
    }
    qsort(out.v, (size_t)(out.n / 2), 2 * sizeof(int32_t), cmp_pair);
    *pairs_out = out.v;
    return out.n / 2;
}

/* ------------------------------------------- all-cores forms (for timing) */

typedef struct {
    const otree *t;
    const float *queries;
    int64_t q0, q1;
    int64_t *counts; /* counts[i - q0] = hits of query i */
    ivec out;
    int rc;
} sel_job;

static void *sel_worker(void *p)
{
    sel_job *j = (sel_job *)p;
    for (int64_t i = j->q0; i < j->q1; i++) {
        box q = {j->queries[4 * i], j->queries[4 * i + 1], j->queries[4 * i + 2],
                 j->queries[4 * i + 3]};
        int64_t start = j->out.n;
        if (j->t && j->t->root && select_rec(j->t->root, q, &j->out)) {
            j->rc = -1;
            return NULL;
        }
        qsort(j->out.v + start, (size_t)(j->out.n - start), sizeof(int32_t), cmp_i32);
        j->counts[i - j->q0] = j->out.n - start;
    }
    return NULL;
}

/* orc_select on `threads` POSIX threads, each taking a contiguous run of the
 * queries; same contract and result as orc_select. */
int64_t orc_select_mt(const otree *t, const float *queries, int64_t Q, int64_t *offsets,
                      int32_t **ids_out, int threads)
{
    if (threads < 1)
        threads = 1;
    if ((int64_t)threads > Q)
        threads = Q > 0 ? (int)Q : 1;
    sel_job *jobs = (sel_job *)calloc((size_t)threads, sizeof(sel_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    char *started = (char *)calloc((size_t)threads, 1);
    if (!jobs || !tid || !started) {
        free(jobs);
        free(tid);
        free(started);
        return -1;
    }
    offsets[0] = 0;
    for (int k = 0; k < threads; k++) {
        jobs[k].t = t;
        jobs[k].queries = queries;
        jobs[k].q0 = Q * k / threads;
        jobs[k].q1 = Q * (k + 1) / threads;
        jobs[k].counts = offsets + 1 + jobs[k].q0;
        started[k] = pthread_create(&tid[k], NULL, sel_worker, &jobs[k]) == 0;
        if (!started[k])
            sel_worker(&jobs[k]);
    }
    int64_t total = 0;
    int rc = 0;
    for (int k = 0; k < threads; k++) {
        if (started[k])
            pthread_join(tid[k], NULL);
        rc |= jobs[k].rc;
        total += jobs[k].out.n;
    }
    int32_t *ids = rc ? NULL : (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t at = 0;
    for (int k = 0; k < threads; k++) {
        if (ids && jobs[k].out.n)
            memcpy(ids + at, jobs[k].out.v, (size_t)jobs[k].out.n * sizeof(int32_t));
        at += jobs[k].out.n;
        free(jobs[k].out.v);
    }
    free(jobs);
    free(tid);
    free(started);
    if (!ids)
        return -1;
    for (int64_t i = 0; i < Q; i++)
        offsets[i + 1] += offsets[i];
    *ids_out = ids;
    return total;
}

typedef struct {
    const onode *a, *b;
    box amb, bmb;
} jcall;

typedef struct {
    jcall *v;
    int64_t n, cap;
} jvec;

static int jvec_push(jvec *c, jcall x)
{
    if (c->n == c->cap) {
        int64_t nc = c->cap ? c->cap * 2 : 64;
        jcall *p = (jcall *)realloc(c->v, (size_t)nc * sizeof(jcall));
        if (!p)
            return -1;
        c->v = p;
        c->cap = nc;
    }
    c->v[c->n++] = x;
    return 0;
}

/* One step of join_rec on a node pair, with the same branching: leaf pairs
 * go to out, and every recursive call join_rec would make goes to next. */
static int join_expand(jcall c, ivec *out, jvec *next)
{
    const onode *a = c.a, *b = c.b;
    if (a->height == b->height) {
        for (int i = 0; i < a->count; i++)
            for (int j = 0; j < b->count; j++) {
                if (!intersects(a->mbr[i], b->mbr[j]))
                    continue;
                if (a->height == 0) {
                    if (emit_pair(out, a->id[i], b->id[j]))
                        return -1;
                } else {
                    jcall d = {a->child[i], b->child[j], a->mbr[i], b->mbr[j]};
                    if (jvec_push(next, d))
                        return -1;
                }
            }
    } else if (a->height > b->height) {
        for (int i = 0; i < a->count; i++)
            if (intersects(a->mbr[i], c.bmb)) {
                jcall d = {a->child[i], b, a->mbr[i], c.bmb};
                if (jvec_push(next, d))
                    return -1;
            }
    } else {
        for (int j = 0; j < b->count; j++)
            if (intersects(c.amb, b->mbr[j])) {
                jcall d = {a, b->child[j], c.amb, b->mbr[j]};
                if (jvec_push(next, d))
                    return -1;
            }
    }
    return 0;
}

typedef struct {
    const jcall *calls;
    int64_t c0, c1;
    ivec out;
    int rc;
} join_job;

static void *join_worker(void *p)
{
    join_job *j = (join_job *)p;
    for (int64_t k = j->c0; k < j->c1; k++) {
        const jcall *c = &j->calls[k];
        if (join_rec(c->a, c->amb, c->b, c->bmb, &j->out)) {
            j->rc = -1;
            return NULL;
        }
    }
    return NULL;
}

/* orc_join on `threads` POSIX threads: the traversal is expanded level by
 * level from the roots until there are at least 8 node pairs per thread (or
 * none left), then each thread runs join_rec on a contiguous run of them.
 * Same contract and result as orc_join. */
int64_t orc_join_mt(const otree *r, const otree *s, int32_t **pairs_out, int threads)
{
    if (threads < 1)
        threads = 1;
    ivec out = {0, 0, 0};
    jvec cur = {0, 0, 0}, next = {0, 0, 0};
    int rc = 0;
    if (r && s && r->root && s->root) {
        jcall root = {r->root, s->root, r->root_mbr, s->root_mbr};
        rc = jvec_push(&cur, root);
        while (!rc && cur.n > 0 && cur.n < 8 * (int64_t)threads) {
            next.n = 0;
            for (int64_t k = 0; k < cur.n && !rc; k++)
                rc = join_expand(cur.v[k], &out, &next);
            jvec t = cur;
            cur = next;
            next = t;
        }
    }
    int nt = (int64_t)threads > cur.n ? (int)(cur.n > 0 ? cur.n : 1) : threads;
    join_job *jobs = (join_job *)calloc((size_t)nt, sizeof(join_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
    char *started = (char *)calloc((size_t)nt, 1);
    if (!jobs || !tid || !started)
        rc = -1;
    for (int k = 0; !rc && k < nt; k++) {
        jobs[k].calls = cur.v;
        jobs[k].c0 = cur.n * k / nt;
        jobs[k].c1 = cur.n * (k + 1) / nt;
        started[k] = pthread_create(&tid[k], NULL, join_worker, &jobs[k]) == 0;
        if (!started[k])
            join_worker(&jobs[k]);
    }
    int64_t total = out.n;
    for (int k = 0; jobs && tid && started && k < nt; k++) {
        if (started[k])
            pthread_join(tid[k], NULL);
        rc |= jobs[k].rc;
        total += jobs[k].out.n;
    }
    int32_t *v = rc ? NULL : (int32_t *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
    int64_t at = 0;
    if (v && out.n)
        memcpy(v, out.v, (size_t)out.n * sizeof(int32_t));
    at = out.n;
    for (int k = 0; jobs && k < nt; k++) {
        if (v && jobs[k].out.n)
            memcpy(v + at, jobs[k].out.v, (size_t)jobs[k].out.n * sizeof(int32_t));
        at += jobs[k].out.n;
        free(jobs[k].out.v);
    }
    free(jobs);
    free(tid);
    free(started);
    free(out.v);
    free(cur.v);
    free(next.v);
    if (!v)
        return -1;
    qsort(v, (size_t)(total / 2), 2 * sizeof(int32_t), cmp_pair);
    *pairs_out = v;
    return total / 2;
}

/* --------------------------------------------- join with sorted-node pruning */

/*
 * The one-to-many join of Section 4.1 with the two prunings of Section 4.2,
 * for trees whose node entries ascend by lx:
 *   O3 -- outer children are taken in ascending lx.  If the key test
 *         out.lx <= in.hx fails against every inner child, no later outer
 *         child (whose lx is no smaller) can pass it: the rest of the outer
 *         node is skipped.
 *   O4 -- for one outer child, inner children are scanned in ascending lx;
 *         the first with in.lx > out.hx ends the scan, as every later inner
 *         child starts even further right.
 * Where heights differ, the taller side's children are scanned in ascending
 * lx against the other node's MBR and the scan ends at the first child that
 * starts right of it (O4 with a single outer MBR).  *tests counts the full
 * predicate evaluations, to show what the pruning saves.
 */
static int join_rec_pruned(const onode *a, box amb, const onode *b, box bmb, ivec *out,
                           int64_t *tests)
{
    if (a->height == b->height) {
        for (int i = 0; i < a->count; i++) {
            int any = 0; /* O3: the lx key test against all inner children */
            for (int j = 0; j < b->count; j++)
                if (a->mbr[i].lx <= b->mbr[j].hx)
                    any = 1;
            if (!any)
                break;
            for (int j = 0; j < b->count; j++) {
                if (b->mbr[j].lx > a->mbr[i].hx) /* O4 */
                    break;
                (*tests)++;
                if (!intersects(a->mbr[i], b->mbr[j]))
                    continue;
                if (a->height == 0) {
                    if (emit_pair(out, a->id[i], b->id[j]))
                        return -1;
                } else if (join_rec_pruned(a->child[i], a->mbr[i], b->child[j], b->mbr[j], out,
                                           tests)) {
                    return -1;
                }
            }
        }
    } else if (a->height > b->height) {
        for (int i = 0; i < a->count; i++) {
            if (a->mbr[i].lx > bmb.hx)
                break;
            (*tests)++;
            if (intersects(a->mbr[i], bmb) &&
                join_rec_pruned(a->child[i], a->mbr[i], b, bmb, out, tests))
                return -1;
        }
    } else {
        for (int j = 0; j < b->count; j++) {
            if (b->mbr[j].lx > amb.hx)
                break;
            (*tests)++;
            if (intersects(amb, b->mbr[j]) &&
                join_rec_pruned(a, amb, b->child[j], b->mbr[j], out, tests))
                return -1;
        }
    }
    return 0;
}

/* Same contract as orc_join; both trees must have been built with
 * sort_children (else -1).  *tests receives the predicate evaluations. */
int64_t orc_join_pruned(const otree *r, const otree *s, int32_t **pairs_out, int64_t *tests)
{
    ivec out = {0, 0, 0};
    *tests = 0;
    if (r && s && r->root && s->root) {
        if (!r->sorted || !s->sorted)
            return -1;
        if (join_rec_pruned(r->root, r->root_mbr, s->root, s->root_mbr, &out, tests)) {
            free(out.v);
            return -1;
        }
    }
    qsort(out.v, (size_t)(out.n / 2), 2 * sizeof(int32_t), cmp_pair);
    *pairs_out = out.v;
    return out.n / 2;
}

/* Predicate evaluations of the plain join (for comparison with the above). */
static void count_rec(const onode *a, box amb, const onode *b, box bmb, int64_t *tests)
{
    if (a->height == b->height) {
        for (int i = 0; i < a->count; i++)
            for (int j = 0; j < b->count; j++) {
                (*tests)++;
                if (a->height > 0 && intersects(a->mbr[i], b->mbr[j]))
                    count_rec(a->child[i], a->mbr[i], b->child[j], b->mbr[j], tests);
            }
    } else if (a->height > b->height) {
        for (int i = 0; i < a->count; i++) {
            (*tests)++;
            if (intersects(a->mbr[i], bmb))
                count_rec(a->child[i], a->mbr[i], b, bmb, tests);
        }
    } else {
        for (int j = 0; j < b->count; j++) {
            (*tests)++;
            if (intersects(amb, b->mbr[j]))
                count_rec(a, amb, b->child[j], b->mbr[j], tests);
        }
    }
}

int64_t orc_join_tests(const otree *r, const otree *s)
{
    int64_t tests = 0;
    if (r && s && r->root && s->root)
        count_rec(r->root, r->root_mbr, s->root, s->root_mbr, &tests);
    return tests;
}

/*
 * O5, the batched form of O4 (Section 4.2, many-to-many comparison): for
 * every outer child at once, find the index beyond which the inner children
 * (ascending lx) cannot qualify, i.e. the first inner index with
 * in.lx > out.hx, by a search that all lanes run in step.
 *   P = n_in rounded up to a power of two; every lane starts at gather index
 *   g = P/2 with its flip index undefined (all inner children qualify);
 *   each of the log2(P)+1 rounds compares out.hx >= in[g].lx (an index past
 *   the node counts as failing); a failing lane records g as its flip index
 *   (keeping the smallest), then every lane moves g up by the step if it
 *   passed and down if it failed; the step starts at P/4 and halves each
 *   round, but never below 1.
 * flip[i] receives the bound for outer child i (n_in when every inner child
 * qualifies).  If trace_g / trace_f are not NULL they receive, for every
 * round, the gather indices used and the flip indices after the round
 * (-1 = undefined), n_out per round.  Returns the number of rounds.
 */
int orc_o5_bounds(const float *out_hx, int n_out, const float *in_lx, int n_in, int32_t *flip,
                  int32_t *trace_g, int32_t *trace_f)
{
    int P = 1, logp = 0;
    while (P < n_in) {
        P *= 2;
        logp++;
    }
    for (int i = 0; i < n_out; i++)
        flip[i] = -1;
    int32_t *g = (int32_t *)malloc((size_t)(n_out > 0 ? n_out : 1) * sizeof(int32_t));
    if (!g)
        return -1;
    for (int i = 0; i < n_out; i++)
        g[i] = P / 2;
    int step = P / 4 > 1 ? P / 4 : 1;
    int rounds = logp + 1;
    for (int t = 0; t < rounds; t++) {
        for (int i = 0; i < n_out; i++) {
            if (trace_g)
                trace_g[t * n_out + i] = g[i];
            int pass = g[i] >= 0 && g[i] < n_in && out_hx[i] >= in_lx[g[i]];
            if (!pass && g[i] < n_in && (flip[i] < 0 || g[i] < flip[i]))
                flip[i] = g[i];
            g[i] = pass ? g[i] + step : g[i] - step;
            if (trace_f)
                trace_f[t * n_out + i] = flip[i];
        }
        step = step / 2 > 1 ? step / 2 : 1;
    }
    for (int i = 0; i < n_out; i++)
        if (flip[i] < 0)
            flip[i] = n_in;
    free(g);
    return rounds;
}

/* Brute-force join: every (r, s) pair. */
int64_t orc_brute_join(const float *ra, const int32_t *rid, int64_t nr, const float *sa,
                       const int32_t *sid, int64_t ns, int32_t **pairs_out)
{
    ivec out = {0, 0, 0};
    for (int64_t i = 0; i < nr; i++) {
        box a = {ra[4 * i], ra[4 * i + 1], ra[4 * i + 2], ra[4 * i + 3]};
        for (int64_t j = 0; j < ns; j++) {
            box b = {sa[4 * j], sa[4 * j + 1], sa[4 * j + 2], sa[4 * j + 3]};
            if (intersects(a, b) && emit_pair(&out, rid[i], sid[j])) {
                free(out.v);
                return -1;
            }
        }
    }
    qsort(out.v, (size_t)(out.n / 2), 2 * sizeof(int32_t), cmp_pair);
    *pairs_out = out.v;
    return out.n / 2;
}
