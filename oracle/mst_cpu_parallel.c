/*
 * The paper's parallel Boruvka with atomic compare-and-swap (Section 2.2.2)
 * on the host's cores, with POSIX threads — TEST INFRASTRUCTURE ONLY.
 *
 * This is a CPU baseline that the benchmark times beside the GPU path, not
 * the parity oracle (that is mst_oracle.c's Kruskal); its own tests check it
 * against Kruskal.  It shares nothing with the CUDA path.
 *
 * The structure follows Section 2.2.2:
 *   - every vertex has an owning thread (owner_tid[], initially v mod T);
 *   - a round resets minimum[] of the owned vertices, then every thread
 *     sweeps all edges from its own spaced start, skipping covered edges,
 *     marking internal ones covered, and keeping the lightest outgoing edge
 *     of each component whose root it owns;
 *   - then every thread takes its owned roots with a minimum, finds the
 *     two components of that edge again, and joins them with one
 *     compare-and-swap of a root's parent; the thread whose swap succeeds
 *     takes ownership of the surviving root, adds the edge to the tree and
 *     marks it covered.
 * Two readings, both of them forced by running the steps concurrently:
 *   - the three steps of a round are separated by barriers (the minima must
 *     be complete before any join reads them);
 *   - the higher-numbered root is hooked under the lower one, not the
 *     destination's component under the source's.  With a fixed direction a
 *     root found first can be joined to the other endpoint's tree before the
 *     swap, and the swap then closes a cycle; pointers that only go to lower
 *     ids cannot.  A failed swap is retried after fresh finds.
 * The edge order is the oracle's: smaller weight, then smaller edge id.
 * The rounds end when no join happened (the spanning forest is complete).
 *
 * Returns the number of tree edges, -1 for a bad vertex id, -2 when out of
 * memory, -3 when a thread cannot be started.
 */
#define _GNU_SOURCE
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CAS_U32 0
#define CAS_F32 1
#define CAS_MAX_THREADS 256

typedef struct {
    int64_t n, m;
    const int32_t *src, *dst;
    const void *w;
    int wt, nthreads;
    int64_t *parent;   /* components[]: the forest, by vertex */
    int64_t *minimum;  /* lightest outgoing edge of a root, or -1 */
    int32_t *owner;    /* owner_tid[] */
    uint8_t *covered;
    uint8_t *in_tree;
    int64_t joined[3]; /* joins per round, rotated by round mod 3 */
    int64_t rounds;
    pthread_barrier_t bar;
    pthread_mutex_t gate_mu; /* threads start together, or not at all */
    pthread_cond_t gate_cv;
    int gate; /* 0 = wait, 1 = run, -1 = abort */
} cas_ctx;

typedef struct {
    cas_ctx *c;
    int tid;
} cas_arg;

static int cas_lighter(const void *w, int wt, int64_t a, int64_t b)
{
    if (wt == CAS_U32) {
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

static int64_t ld(const int64_t *p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
static void st(int64_t *p, int64_t v) { __atomic_store_n(p, v, __ATOMIC_RELAXED); }

/* Root of v with path halving.  Pointers only move to ancestors and only a
 * root's pointer is swapped, so concurrent halving and joins are safe. */
static int64_t cas_find(int64_t *parent, int64_t v)
{
    for (;;) {
        int64_t p = ld(parent + v);
        if (p == v)
            return v;
        int64_t gp = ld(parent + p);
        if (gp != p)
            st(parent + v, gp);
        v = gp;
    }
}

static void *cas_thread(void *argp)
{
    cas_arg *a = (cas_arg *)argp;
    cas_ctx *c = a->c;
    pthread_mutex_lock(&c->gate_mu);
    while (c->gate == 0)
        pthread_cond_wait(&c->gate_cv, &c->gate_mu);
    const int go = c->gate;
    pthread_mutex_unlock(&c->gate_mu);
    if (go < 0)
        return NULL;
    const int tid = a->tid, T = c->nthreads;
    const int64_t n = c->n, m = c->m;
    for (int64_t r = 0;; r++) {
        /* every thread resets minimum[] of the vertices it owns */
        for (int64_t v = 0; v < n; v++)
            if (__atomic_load_n(c->owner + v, __ATOMIC_RELAXED) == tid)
                c->minimum[v] = -1;
        if (tid == 0)
            __atomic_store_n(&c->joined[(r + 1) % 3], 0, __ATOMIC_RELAXED);
        pthread_barrier_wait(&c->bar);
        /* every thread sweeps all edges from a spaced start */
        const int64_t start = m > 0 ? (int64_t)((double)m * tid / T) : 0;
        for (int64_t k = 0; k < m; k++) {
            int64_t e = start + k;
            if (e >= m)
                e -= m;
            if (__atomic_load_n(c->covered + e, __ATOMIC_RELAXED))
                continue;
            int64_t c1 = cas_find(c->parent, c->src[e]);
            int64_t c2 = cas_find(c->parent, c->dst[e]);
            if (c1 == c2) {
                __atomic_store_n(c->covered + e, 1, __ATOMIC_RELAXED);
                continue;
            }
            if (__atomic_load_n(c->owner + c1, __ATOMIC_RELAXED) == tid &&
                (c->minimum[c1] == -1 || cas_lighter(c->w, c->wt, e, c->minimum[c1])))
                c->minimum[c1] = e;
            if (__atomic_load_n(c->owner + c2, __ATOMIC_RELAXED) == tid &&
                (c->minimum[c2] == -1 || cas_lighter(c->w, c->wt, e, c->minimum[c2])))
                c->minimum[c2] = e;
        }
        pthread_barrier_wait(&c->bar);
        /* every thread joins along the minima of the roots it owns */
        int64_t joined = 0;
        for (int64_t v = 0; v < n; v++) {
            if (__atomic_load_n(c->owner + v, __ATOMIC_RELAXED) != tid || ld(c->parent + v) != v)
                continue;
            const int64_t e = c->minimum[v];
            if (e == -1)
                continue;
            for (;;) {
                int64_t c1 = cas_find(c->parent, c->src[e]);
                int64_t c2 = cas_find(c->parent, c->dst[e]);
                if (c1 == c2) {
                    __atomic_store_n(c->covered + e, 1, __ATOMIC_RELAXED);
                    break;
                }
                int64_t lo = c1 < c2 ? c1 : c2, hi = c1 < c2 ? c2 : c1, expect = hi;
                if (__atomic_compare_exchange_n(c->parent + hi, &expect, lo, 0, __ATOMIC_RELAXED,
                                                __ATOMIC_RELAXED)) {
                    __atomic_store_n(c->owner + lo, tid, __ATOMIC_RELAXED);
                    c->in_tree[e] = 1;
                    __atomic_store_n(c->covered + e, 1, __ATOMIC_RELAXED);
                    joined++;
                    break;
                }
            }
        }
        __atomic_fetch_add(&c->joined[r % 3], joined, __ATOMIC_RELAXED);
        pthread_barrier_wait(&c->bar);
        if (__atomic_load_n(&c->joined[r % 3], __ATOMIC_RELAXED) == 0) {
            if (tid == 0)
                c->rounds = r;
            return NULL;
        }
    }
}

int64_t orc_boruvka_cas_mt(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           const void *w, int wt, int nthreads, uint8_t *in_tree,
                           int64_t *rounds_out)
{
    if (n < 0 || m < 0 || nthreads < 1 || nthreads > CAS_MAX_THREADS)
        return -1;
    for (int64_t e = 0; e < m; e++)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
            return -1;
    cas_ctx c;
    memset(&c, 0, sizeof(c));
    c.n = n;
    c.m = m;
    c.src = src;
    c.dst = dst;
    c.w = w;
    c.wt = wt;
    c.nthreads = nthreads;
    const size_t nv = (size_t)(n > 0 ? n : 1), ne = (size_t)(m > 0 ? m : 1);
    c.parent = (int64_t *)malloc(sizeof(int64_t) * nv);
    c.minimum = (int64_t *)malloc(sizeof(int64_t) * nv);
    c.owner = (int32_t *)malloc(sizeof(int32_t) * nv);
    c.covered = (uint8_t *)calloc(ne, 1);
    c.in_tree = in_tree;
    pthread_t th[CAS_MAX_THREADS];
    cas_arg args[CAS_MAX_THREADS];
    int64_t rc = -2;
    if (!c.parent || !c.minimum || !c.owner || !c.covered)
        goto out;
    for (int64_t v = 0; v < n; v++) {
        c.parent[v] = v;
        c.minimum[v] = -1;
        c.owner[v] = (int32_t)(v % nthreads);
    }
    for (int64_t e = 0; e < m; e++) {
        in_tree[e] = 0;
        if (src[e] == dst[e])
            c.covered[e] = 1; /* a self-loop is internal from the start */
    }
    if (pthread_barrier_init(&c.bar, NULL, (unsigned)nthreads)) {
        rc = -3;
        goto out;
    }
    pthread_mutex_init(&c.gate_mu, NULL);
    pthread_cond_init(&c.gate_cv, NULL);
    for (int t = 0; t < nthreads; t++) {
        args[t].c = &c;
        args[t].tid = t;
    }
    /* every thread must exist before the first barrier: the threads wait at
     * a gate until all are started, and leave if one could not be */
    int started = 0;
    for (int t = 1; t < nthreads; t++) {
        if (pthread_create(&th[t], NULL, cas_thread, &args[t]))
            break;
        started++;
    }
    pthread_mutex_lock(&c.gate_mu);
    c.gate = started == nthreads - 1 ? 1 : -1;
    pthread_cond_broadcast(&c.gate_cv);
    pthread_mutex_unlock(&c.gate_mu);
    if (c.gate > 0)
        cas_thread(&args[0]);
    for (int t = 1; t <= started; t++)
        pthread_join(th[t], NULL);
    pthread_barrier_destroy(&c.bar);
    pthread_mutex_destroy(&c.gate_mu);
    pthread_cond_destroy(&c.gate_cv);
    if (c.gate < 0) {
        rc = -3;
        goto out;
    }
    rc = 0;
    for (int64_t e = 0; e < m; e++)
        rc += in_tree[e];
    if (rounds_out)
        *rounds_out = c.rounds;
out:
    free(c.parent);
    free(c.minimum);
    free(c.owner);
    free(c.covered);
    return rc;
}
