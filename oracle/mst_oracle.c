/*
 * CPU oracle for minimum spanning trees — TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, obviously-correct reference that the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it; the product library never does.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes.  The paper defines the minimum spanning tree as the tree
 * joining every vertex of a connected graph whose total edge weight is
 * smallest (Section 1) and assumes distinct weights (Section 2.1, inputs),
 * which makes that tree unique.  Ties are resolved here by one reading: an
 * edge is lighter than another if its weight is smaller, or the weights are
 * equal and its edge id (index in the input arrays) is smaller.  Under that
 * total order the tree is unique for every input.  A disconnected input gets
 * its minimum spanning forest.
 *
 * Functions (each independent of the others except the shared comparison
 * and the union-find helpers):
 *   orc_kruskal     — Kruskal: edges in increasing order, keep an edge whose
 *                     ends are in different sets (textbook; Section 1 names it).
 *   orc_boruvka     — sequential Boruvka exactly as Section 2.1 lays it out:
 *                     per round reset minimum[], sweep all edges keeping each
 *                     component's lightest outgoing edge, then for each vertex
 *                     with a minimum re-check the two components and join them
 *                     (bigger component's root wins).  With covered_opt it
 *                     also applies the Section 2.1 "Optimization": internal
 *                     and chosen edges are marked covered and skipped.
 *   orc_prim        — Prim with a binary heap (textbook; Section 1 names it).
 *   orc_components  — number of connected components (union-find).
 *   orc_check_cycle_property — certificate: the marked edges form a spanning
 *                     forest of the graph and every unmarked edge is heavier
 *                     than every edge on the forest path between its ends.
 *   orc_check_cut_property   — certificate for small graphs: removing any
 *                     marked edge splits its tree in two, and that edge is the
 *                     lightest graph edge across the split (the exchange
 *                     argument of the Section 2.2.1 correctness proof).
 *
 * Weight types: 0 = uint32, 1 = float32 (compared as floats; NaN is the
 * caller's error and is rejected by the Python wrapper).
 *
 * Return values: edge counts >= 0; -1 = bad vertex id; -2 = out of memory.
 * Certificates return 0 when the certificate holds, > 0 naming the first
 * violated condition.
 */
#define _GNU_SOURCE /* qsort_r */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_U32 0
#define ORC_F32 1

/* ---- the edge order: weight, then edge id -------------------------------- */

/* Returns 1 when edge a is lighter than edge b. */
static int lighter(const void *w, int wt, int64_t a, int64_t b)
{
    if (wt == ORC_U32) {
        uint32_t x = ((const uint32_t *)w)[a], y = ((const uint32_t *)w)[b];
        if (x != y)
            return x < y;
    } else {
        float x = ((const float *)w)[a], y = ((const float *)w)[b];
        if (x < y)
            return 1;
        if (y < x)
            return 0;
    }
    return a < b;
}

static int check_ids(int64_t n, int64_t m, const int32_t *src, const int32_t *dst)
{
    if (n < 0 || m < 0)
        return -1;
    for (int64_t e = 0; e < m; e++)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
            return -1;
    return 0;
}

/* ---- union-find (path halving, union by size) ----------------------------- */

static int64_t uf_find(int64_t *parent, int64_t v)
{
    while (parent[v] != v) {
        parent[v] = parent[parent[v]];
        v = parent[v];
    }
    return v;
}

/* Joins the sets of roots a and b; the root of the bigger set stays root. */
static void uf_union(int64_t *parent, int64_t *size, int64_t a, int64_t b)
{
    if (size[a] < size[b]) {
        int64_t t = a;
        a = b;
        b = t;
    }
    parent[b] = a;
    size[a] += size[b];
}

static int uf_init(int64_t n, int64_t **parent, int64_t **size)
{
    *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    *size = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!*parent || !*size) {
        free(*parent);
        free(*size);
        return -2;
    }
    for (int64_t v = 0; v < n; v++) {
        (*parent)[v] = v;
        (*size)[v] = 1;
    }
    return 0;
}

/* ---- Kruskal ------------------------------------------------------------- */

typedef struct {
    const void *w;
    int wt;
} order_ctx;

static int cmp_edges(const void *pa, const void *pb, void *ctx)
{
    const order_ctx *c = (const order_ctx *)ctx;
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (lighter(c->w, c->wt, a, b))
        return -1;
    if (lighter(c->w, c->wt, b, a))
        return 1;
    return 0;
}

int64_t orc_kruskal(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const void *w, int wt, uint8_t *in_tree)
{
    if (check_ids(n, m, src, dst))
        return -1;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *parent, *size;
    if (!order || uf_init(n, &parent, &size)) {
        free(order);
        return -2;
    }
    for (int64_t e = 0; e < m; e++)
        order[e] = e;
    order_ctx ctx = {w, wt};
    qsort_r(order, (size_t)m, sizeof(int64_t), cmp_edges, &ctx);
    for (int64_t e = 0; e < m; e++)
        in_tree[e] = 0;
    int64_t count = 0;
    for (int64_t i = 0; i < m; i++) {
        int64_t e = order[i];
        int64_t a = uf_find(parent, src[e]), b = uf_find(parent, dst[e]);
        if (a != b) {
            uf_union(parent, size, a, b);
            in_tree[e] = 1;
            count++;
        }
    }
    free(order);
    free(parent);
    free(size);
    return count;
}

/* ---- sequential Boruvka, Section 2.1 ------------------------------------- */

/*
 * components[] of the paper is the union-find forest; find() walks it with
 * path halving (the paper leaves compression unspecified).  minimum[v] = -1
 * means "no edge".  The loop runs while the previous round joined anything:
 * for a connected input that is exactly "while F has more than one
 * component"; for a disconnected input it stops with the spanning forest.
 * rounds_out receives the number of rounds that joined components.
 */
int64_t orc_boruvka(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                    const void *w, int wt, int covered_opt, uint8_t *in_tree,
                    int64_t *rounds_out)
{
    if (check_ids(n, m, src, dst))
        return -1;
    int64_t *components, *size;
    int64_t *minimum = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *covered = (uint8_t *)calloc((size_t)(m > 0 ? m : 1), 1);
    if (!minimum || !covered || uf_init(n, &components, &size)) {
        free(minimum);
        free(covered);
        return -2;
    }
    for (int64_t e = 0; e < m; e++)
        in_tree[e] = 0;
    int64_t count = 0, rounds = 0;
    int64_t ncomp = n;
    while (ncomp > 1) {
        /* Initialize minimum[] to -1 for all vertices */
        for (int64_t v = 0; v < n; v++)
            minimum[v] = -1;
        /* For all edges: keep the lightest edge leaving each component */
        for (int64_t e = 0; e < m; e++) {
            if (covered_opt && covered[e])
                continue;
            int64_t c1 = uf_find(components, src[e]);
            int64_t c2 = uf_find(components, dst[e]);
            if (c1 == c2) {
                if (covered_opt)
                    covered[e] = 1;
                continue;
            }
            if (minimum[c1] == -1 || lighter(w, wt, e, minimum[c1]))
                minimum[c1] = e;
            if (minimum[c2] == -1 || lighter(w, wt, e, minimum[c2]))
                minimum[c2] = e;
        }
        /* For each vertex with a minimum: re-check, add to M, join */
        int64_t joined = 0;
        for (int64_t v = 0; v < n; v++) {
            if (minimum[v] == -1)
                continue;
            int64_t e = minimum[v];
            int64_t c1 = uf_find(components, src[e]);
            int64_t c2 = uf_find(components, dst[e]);
            if (c1 == c2)
                continue;
            in_tree[e] = 1;
            count++;
            uf_union(components, size, c1, c2);
            if (covered_opt)
                covered[e] = 1;
            joined++;
        }
        if (joined == 0)
            break; /* no edge leaves any component: spanning forest done */
        ncomp -= joined;
        rounds++;
    }
    if (rounds_out)
        *rounds_out = rounds;
    free(minimum);
    free(covered);
    free(components);
    free(size);
    return count;
}

/* ---- Prim with a binary heap ---------------------------------------------- */

typedef struct {
    int64_t *heap; /* edge ids */
    int64_t len;
    const void *w;
    int wt;
} edge_heap;

static void heap_push(edge_heap *h, int64_t e)
{
    int64_t i = h->len++;
    h->heap[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!lighter(h->w, h->wt, h->heap[i], h->heap[p]))
            break;
        int64_t t = h->heap[i];
        h->heap[i] = h->heap[p];
        h->heap[p] = t;
        i = p;
    }
}

static int64_t heap_pop(edge_heap *h)
{
    int64_t top = h->heap[0];
    h->heap[0] = h->heap[--h->len];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->len && lighter(h->w, h->wt, h->heap[l], h->heap[s]))
            s = l;
        if (r < h->len && lighter(h->w, h->wt, h->heap[r], h->heap[s]))
            s = r;
        if (s == i)
            break;
        int64_t t = h->heap[i];
        h->heap[i] = h->heap[s];
        h->heap[s] = t;
        i = s;
    }
    return top;
}

/* CSR adjacency: for vertex v, adj[off[v] .. off[v+1]) are incident edge ids. */
static int build_adjacency(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const uint8_t *mask, int64_t **off_out, int64_t **adj_out)
{
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off)
        return -2;
    for (int64_t e = 0; e < m; e++) {
        if (mask && !mask[e])
            continue;
        off[src[e] + 1]++;
        if (dst[e] != src[e])
            off[dst[e] + 1]++;
    }
    for (int64_t v = 0; v < n; v++)
        off[v + 1] += off[v];
    int64_t *adj = (int64_t *)malloc(sizeof(int64_t) * (size_t)(off[n] > 0 ? off[n] : 1));
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!adj || !fill) {
        free(off);
        free(adj);
        free(fill);
        return -2;
    }
    memcpy(fill, off, sizeof(int64_t) * (size_t)n);
    for (int64_t e = 0; e < m; e++) {
        if (mask && !mask[e])
            continue;
        adj[fill[src[e]]++] = e;
        if (dst[e] != src[e])
            adj[fill[dst[e]]++] = e;
    }
    free(fill);
    *off_out = off;
    *adj_out = adj;
    return 0;
}

int64_t orc_prim(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                 const void *w, int wt, uint8_t *in_tree)
{
    if (check_ids(n, m, src, dst))
        return -1;
    int64_t *off, *adj;
    if (build_adjacency(n, m, src, dst, NULL, &off, &adj))
        return -2;
    uint8_t *seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    edge_heap h = {(int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1)), 0, w, wt};
    if (!seen || !h.heap) {
        free(off);
        free(adj);
        free(seen);
        free(h.heap);
        return -2;
    }
    for (int64_t e = 0; e < m; e++)
        in_tree[e] = 0;
    int64_t count = 0;
    for (int64_t s = 0; s < n; s++) {
        if (seen[s])
            continue;
        seen[s] = 1;
        for (int64_t i = off[s]; i < off[s + 1]; i++)
            heap_push(&h, adj[i]);
        while (h.len > 0) {
            int64_t e = heap_pop(&h);
            int64_t x = seen[src[e]] ? dst[e] : src[e];
            if (seen[x])
                continue; /* both ends already in the tree */
            seen[x] = 1;
            in_tree[e] = 1;
            count++;
            for (int64_t i = off[x]; i < off[x + 1]; i++) {
                int64_t f = adj[i];
                int64_t y = src[f] == x ? dst[f] : src[f];
                if (!seen[y])
                    heap_push(&h, f);
            }
        }
    }
    free(off);
    free(adj);
    free(seen);
    free(h.heap);
    return count;
}

/* ---- connected components ------------------------------------------------- */

int64_t orc_components(int64_t n, int64_t m, const int32_t *src, const int32_t *dst)
{
    if (check_ids(n, m, src, dst))
        return -1;
    int64_t *parent, *size;
    if (uf_init(n, &parent, &size))
        return -2;
    int64_t comps = n;
    for (int64_t e = 0; e < m; e++) {
        int64_t a = uf_find(parent, src[e]), b = uf_find(parent, dst[e]);
        if (a != b) {
            uf_union(parent, size, a, b);
            comps--;
        }
    }
    free(parent);
    free(size);
    return comps;
}

/* ---- certificate: spanning forest + cycle property ------------------------ */

/*
 * Returns 0 if in_tree marks a spanning forest of the graph (acyclic, one
 * tree per connected component) and every unmarked non-loop edge (u,v) is
 * heavier than the heaviest marked edge on the forest path u..v.  Together
 * these certify that in_tree is the minimum spanning forest under the edge
 * order.  Codes: 1 marked self-loop, 2 cycle among marked edges, 3 unmarked
 * edge joins two different trees (forest not spanning), 4 cycle property
 * violated, -1 bad ids, -2 no memory.
 */
int orc_check_cycle_property(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                             const void *w, int wt, const uint8_t *in_tree)
{
    if (check_ids(n, m, src, dst))
        return -1;
    for (int64_t e = 0; e < m; e++)
        if (in_tree[e] && src[e] == dst[e])
            return 1;
    int64_t *off, *adj;
    if (build_adjacency(n, m, src, dst, in_tree, &off, &adj))
        return -2;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t *tree_id = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *depth = (int64_t *)malloc(sizeof(int64_t) * nn);
    int64_t *up0 = (int64_t *)malloc(sizeof(int64_t) * nn);   /* parent vertex */
    int64_t *upe0 = (int64_t *)malloc(sizeof(int64_t) * nn);  /* parent edge id */
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * nn);
    int rc = 0;
    if (!tree_id || !depth || !up0 || !upe0 || !queue) {
        rc = -2;
        goto out0;
    }
    for (int64_t v = 0; v < n; v++)
        tree_id[v] = -1;
    int64_t maxdepth = 0;
    for (int64_t s = 0; s < n && rc == 0; s++) {
        if (tree_id[s] != -1)
            continue;
        int64_t qh = 0, qt = 0;
        queue[qt++] = s;
        tree_id[s] = s;
        depth[s] = 0;
        up0[s] = s;
        upe0[s] = -1;
        while (qh < qt && rc == 0) {
            int64_t x = queue[qh++];
            for (int64_t i = off[x]; i < off[x + 1]; i++) {
                int64_t e = adj[i];
                if (e == upe0[x])
                    continue;
                int64_t y = src[e] == x ? dst[e] : src[e];
                if (tree_id[y] != -1) {
                    rc = 2; /* reached a vertex twice: marked edges have a cycle */
                    break;
                }
                tree_id[y] = s;
                depth[y] = depth[x] + 1;
                if (depth[y] > maxdepth)
                    maxdepth = depth[y];
                up0[y] = x;
                upe0[y] = e;
                queue[qt++] = y;
            }
        }
    }
    if (rc)
        goto out0;
    /* binary lifting: up[k][v] = 2^k-th ancestor, mx[k][v] = heaviest edge on the way */
    int levels = 1;
    while (((int64_t)1 << levels) <= maxdepth)
        levels++;
    int64_t **up = (int64_t **)calloc((size_t)levels, sizeof(int64_t *));
    int64_t **mx = (int64_t **)calloc((size_t)levels, sizeof(int64_t *));
    if (!up || !mx) {
        free(up);
        free(mx);
        rc = -2;
        goto out0;
    }
    up[0] = up0;
    mx[0] = upe0;
    for (int k = 1; k < levels && rc == 0; k++) {
        up[k] = (int64_t *)malloc(sizeof(int64_t) * nn);
        mx[k] = (int64_t *)malloc(sizeof(int64_t) * nn);
        if (!up[k] || !mx[k]) {
            rc = -2;
            break;
        }
        for (int64_t v = 0; v < n; v++) {
            int64_t mid = up[k - 1][v];
            up[k][v] = up[k - 1][mid];
            int64_t a = mx[k - 1][v], b = mx[k - 1][mid];
            if (a == -1)
                mx[k][v] = b;
            else if (b == -1)
                mx[k][v] = a;
            else
                mx[k][v] = lighter(w, wt, a, b) ? b : a;
        }
    }
    for (int64_t e = 0; e < m && rc == 0; e++) {
        if (in_tree[e] || src[e] == dst[e])
            continue;
        int64_t a = src[e], b = dst[e];
        if (tree_id[a] != tree_id[b]) {
            rc = 3;
            break;
        }
        int64_t heaviest = -1;
#define TAKE(f)                                                                  \
    do {                                                                         \
        int64_t f_ = (f);                                                        \
        if (f_ != -1 && (heaviest == -1 || lighter(w, wt, heaviest, f_)))        \
            heaviest = f_;                                                       \
    } while (0)
        if (depth[a] < depth[b]) {
            int64_t t = a;
            a = b;
            b = t;
        }
        for (int k = levels - 1; k >= 0; k--)
            if (depth[a] - ((int64_t)1 << k) >= depth[b]) {
                TAKE(mx[k][a]);
                a = up[k][a];
            }
        if (a != b) {
            for (int k = levels - 1; k >= 0; k--)
                if (up[k][a] != up[k][b]) {
                    TAKE(mx[k][a]);
                    TAKE(mx[k][b]);
                    a = up[k][a];
                    b = up[k][b];
                }
            TAKE(mx[0][a]);
            TAKE(mx[0][b]);
        }
#undef TAKE
        if (heaviest == -1 || !lighter(w, wt, heaviest, e))
            rc = 4;
    }
    for (int k = 1; k < levels; k++) {
        free(up[k]);
        free(mx[k]);
    }
    free(up);
    free(mx);
out0:
    free(off);
    free(adj);
    free(tree_id);
    free(depth);
    free(up0);
    free(upe0);
    free(queue);
    return rc;
}

/* ---- certificate: cut property (small graphs) ----------------------------- */

/*
 * For every marked edge t: remove t from the marked forest, collect the side
 * S holding src[t] (search over marked edges), and require that t is the
 * lightest of all graph edges with exactly one end in S.  O(n * (n + m)).
 * Codes: 5 a marked edge is not the lightest across its cut, 6 the marked
 * edges contain a cycle (t's ends stay connected without t), -1, -2.
 */
int orc_check_cut_property(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const void *w, int wt, const uint8_t *in_tree)
{
    if (check_ids(n, m, src, dst))
        return -1;
    int64_t *off, *adj;
    if (build_adjacency(n, m, src, dst, in_tree, &off, &adj))
        return -2;
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint8_t *side = (uint8_t *)malloc(nn);
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * nn);
    int rc = 0;
    if (!side || !stack)
        rc = -2;
    for (int64_t t = 0; t < m && rc == 0; t++) {
        if (!in_tree[t])
            continue;
        memset(side, 0, nn);
        int64_t sp = 0;
        stack[sp++] = src[t];
        side[src[t]] = 1;
        while (sp > 0) {
            int64_t x = stack[--sp];
            for (int64_t i = off[x]; i < off[x + 1]; i++) {
                int64_t e = adj[i];
                if (e == t)
                    continue;
                int64_t y = src[e] == x ? dst[e] : src[e];
                if (!side[y]) {
                    side[y] = 1;
                    stack[sp++] = y;
                }
            }
        }
        if (side[dst[t]]) {
            rc = 6;
            break;
        }
        int64_t best = -1;
        for (int64_t e = 0; e < m; e++)
            if (side[src[e]] != side[dst[e]] && (best == -1 || lighter(w, wt, e, best)))
                best = e;
        if (best != t)
            rc = 5;
    }
    free(off);
    free(adj);
    free(side);
    free(stack);
    return rc;
}
