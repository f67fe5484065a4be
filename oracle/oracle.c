/*
 * CPU oracle for the traversal results: TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It shares no code, header, table or helper with the CUDA
 * library; it is deliberately plain, single-threaded and slow so that each
 * function can be checked against its definition by eye.
 *
 * Every result here is the exact textbook answer, so each function is that
 * definition written out:
 *   oracle_bfs  - FIFO-queue breadth-first search (Sec. 2.1, Algorithm
 *                 "High-level Graph Traversal Flow" with BFS as the workload:
 *                 unvisited neighbours of the active set become active at
 *                 the next depth).  level[src] = 0, unreachable = UINT32_MAX.
 *   oracle_sssp - Dijkstra with a binary heap and 64-bit accumulation
 *                 (single-source shortest path with non-negative integer
 *                 weights, Sec. 5.1.2 / Sec. 5.4).  Unreachable = UINT32_MAX;
 *                 a finite distance >= UINT32_MAX is reported as overflow.
 *   oracle_cc   - union-find (path halving; the larger root is linked under
 *                 the smaller), connected components of an undirected graph
 *                 (Sec. 5.4).  label[v] = the smallest vertex id in v's
 *                 component.
 *   oracle_pagerank - PageRank by power iteration in double precision (the
 *                 fourth application of Sec. 5.4), every vertex active each
 *                 iteration.  This is an iteration, not a closed form, so it
 *                 follows the steps in order: start from 1/n; each iteration
 *                 gives every vertex (1 - d)/n, plus d times the rank of the
 *                 vertices without out-edges divided by n, plus d times
 *                 rank(v)/outdeg(v) for each edge v -> u it receives; stop
 *                 after max_iter iterations or once the L1 change is below
 *                 tol.  Parallel edges and self-loops count as edges.
 *
 * Build: gcc -O2 -shared -fPIC oracle.c -o _oracle.so
 */
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_INF 0xFFFFFFFFu

/* Returns 0 on success, 1 if src is out of range, 2 on allocation failure. */
int oracle_bfs(uint64_t n, const uint64_t* offsets, const uint64_t* cols, uint64_t src,
               uint32_t* level) {
    if (src >= n) return 1;
    uint64_t* queue = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!queue) return 2;
    for (uint64_t v = 0; v < n; v++) level[v] = ORACLE_INF;
    uint64_t head = 0, tail = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint64_t v = queue[head++];
        for (uint64_t i = offsets[v]; i < offsets[v + 1]; i++) {
            uint64_t u = cols[i];
            if (level[u] == ORACLE_INF) {
                level[u] = level[v] + 1;
                queue[tail++] = u;
            }
        }
    }
    free(queue);
    return 0;
}

/* ---- binary min-heap of (distance, vertex) pairs, lazy deletion ---- */
typedef struct { uint64_t d, v; } hitem;

static int hless(hitem a, hitem b) { return a.d < b.d || (a.d == b.d && a.v < b.v); }

static void hpush(hitem* h, uint64_t* sz, hitem x) {
    uint64_t i = (*sz)++;
    h[i] = x;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!hless(h[i], h[p])) break;
        hitem t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static hitem hpop(hitem* h, uint64_t* sz) {
    hitem top = h[0];
    h[0] = h[--(*sz)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *sz && hless(h[l], h[s])) s = l;
        if (r < *sz && hless(h[r], h[s])) s = r;
        if (s == i) break;
        hitem t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/* Returns 0 on success, 1 bad src, 2 no memory, 3 a finite distance does not
 * fit below UINT32_MAX (dist[] then holds the low 32 bits clamped to
 * UINT32_MAX - 1 for such vertices; callers treat it as an error). */
int oracle_sssp(uint64_t n, const uint64_t* offsets, const uint64_t* cols, const uint32_t* w,
                uint64_t src, uint32_t* dist) {
    if (src >= n) return 1;
    uint64_t m = offsets[n];
    uint64_t* d = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    unsigned char* done = (unsigned char*)calloc(n ? n : 1, 1);
    hitem* heap = (hitem*)malloc((m + 1) * sizeof(hitem));
    if (!d || !done || !heap) { free(d); free(done); free(heap); return 2; }
    const uint64_t UNREACHED = UINT64_MAX;
    for (uint64_t v = 0; v < n; v++) d[v] = UNREACHED;
    uint64_t sz = 0;
    d[src] = 0;
    hitem s0 = {0, src};
    hpush(heap, &sz, s0);
    while (sz) {
        hitem x = hpop(heap, &sz);
        if (done[x.v] || x.d != d[x.v]) continue;
        done[x.v] = 1;
        for (uint64_t i = offsets[x.v]; i < offsets[x.v + 1]; i++) {
            uint64_t u = cols[i];
            uint64_t nd = x.d + (uint64_t)w[i];
            if (nd < d[u]) {
                d[u] = nd;
                hitem y = {nd, u};
                hpush(heap, &sz, y);
            }
        }
    }
    int overflow = 0;
    for (uint64_t v = 0; v < n; v++) {
        if (d[v] == UNREACHED) dist[v] = ORACLE_INF;
        else if (d[v] >= (uint64_t)ORACLE_INF) { dist[v] = ORACLE_INF - 1; overflow = 1; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(done); free(heap);
    return overflow ? 3 : 0;
}

static uint64_t uf_find(uint64_t* parent, uint64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]]; /* path halving */
        x = parent[x];
    }
    return x;
}

/* Returns 0 on success, 2 on allocation failure.  Treats every stored edge as
 * undirected. */
int oracle_cc(uint64_t n, const uint64_t* offsets, const uint64_t* cols, uint32_t* label) {
    uint64_t* parent = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!parent) return 2;
    for (uint64_t v = 0; v < n; v++) parent[v] = v;
    for (uint64_t v = 0; v < n; v++) {
        for (uint64_t i = offsets[v]; i < offsets[v + 1]; i++) {
            uint64_t a = uf_find(parent, v), b = uf_find(parent, cols[i]);
            if (a == b) continue;
            if (a < b) parent[b] = a; else parent[a] = b;
        }
    }
    for (uint64_t v = 0; v < n; v++) label[v] = (uint32_t)uf_find(parent, v);
    free(parent);
    return 0;
}

/* PageRank, power iteration (see the header).  rank: n doubles, output.
 * Returns the iterations run through *iters; 0 on success, 2 on allocation
 * failure. */
int oracle_pagerank(uint64_t n, const uint64_t* offsets, const uint64_t* cols, double damping, double tol,
                    uint32_t max_iter, double* rank, uint32_t* iters) {
    *iters = 0;
    if (n == 0) return 0;
    double* next = (double*)malloc(n * sizeof(double));
    if (!next) return 2;
    for (uint64_t v = 0; v < n; v++) rank[v] = 1.0 / (double)n;
    for (uint32_t it = 0; it < max_iter; it++) {
        double dangling = 0.0;
        for (uint64_t v = 0; v < n; v++)
            if (offsets[v + 1] == offsets[v]) dangling += rank[v];
        const double base = (1.0 - damping) / (double)n + damping * dangling / (double)n;
        for (uint64_t u = 0; u < n; u++) next[u] = base;
        for (uint64_t v = 0; v < n; v++) {
            const uint64_t deg = offsets[v + 1] - offsets[v];
            for (uint64_t i = offsets[v]; i < offsets[v + 1]; i++)
                next[cols[i]] += damping * rank[v] / (double)deg;
        }
        double change = 0.0;
        for (uint64_t v = 0; v < n; v++) {
            change += next[v] > rank[v] ? next[v] - rank[v] : rank[v] - next[v];
            rank[v] = next[v];
        }
        *iters = it + 1;
        if (change < tol) break;
    }
    free(next);
    return 0;
}
