/*
 * Seeded synthetic graph generators (Kronecker and uniform random) and a CSR
 * builder.  This module only makes inputs: it holds none of the traversal
 * arithmetic, and both the CPU oracle and the CUDA path consume what it makes.
 *
 * Randomness is counter based: value i of a stream with seed s is the i-th
 * output of a SplitMix64 generator seeded with s (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), so any
 * sample can be regenerated independently and the result does not depend on
 * thread count or scheduling.
 *
 * Graph recipe (stands in for the GAP-kron and GAP-urand graphs of the
 * paper's Table "Graph Datasets", Sec. 5.2):
 *   Kronecker: 2^scale vertices, ef * 2^scale samples; each sample picks one
 *     quadrant per bit level with probabilities (0.57, 0.19, 0.19, 0.05);
 *     vertex ids are relabelled by a seeded Fisher-Yates permutation.
 *   Uniform: n vertices, samples with both endpoints iid uniform on [0, n).
 *   Cleaning (both): self-loops dropped, every sample stored in both
 *     directions, each row sorted ascending and de-duplicated.
 *   Weights: w(u,v) = w(v,u) = 1 + (hash(min,max) mod 255), in [1, 255].
 *
 * Build: gcc -O3 -fopenmp -shared -fPIC graphgen.c -o _graphgen.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th output (0-based) of a SplitMix64 stream seeded with `seed`. */
uint64_t gg_rand(uint64_t seed, uint64_t i) { return gg_mix(seed + (i + 1) * GG_GAMMA); }

/* Map a 64-bit random value to [0, bound) by a 64x64->128 multiply. */
static inline uint64_t gg_bounded(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)bound) >> 64);
}

/* Sub-stream seeds, so that the edge, permutation and weight streams differ. */
static inline uint64_t seed_edges(uint64_t s) { return gg_mix(s ^ 0x45444745ULL); }
static inline uint64_t seed_perm(uint64_t s) { return gg_mix(s ^ 0x5045524DULL); }

enum { GG_KRON = 0, GG_UNIFORM = 1 };

/* Kronecker quadrant thresholds on a 53-bit uniform integer. */
#define GG_P53 9007199254740992.0 /* 2^53 */
static inline void kron_sample(uint64_t seed, int scale, uint64_t k, uint64_t* pu, uint64_t* pv) {
    const uint64_t t_a = (uint64_t)(0.57 * GG_P53);
    const uint64_t t_ab = (uint64_t)(0.76 * GG_P53);
    const uint64_t t_abc = (uint64_t)(0.95 * GG_P53);
    uint64_t u = 0, v = 0;
    const uint64_t base = k * (uint64_t)scale;
    for (int l = 0; l < scale; l++) {
        uint64_t x = gg_rand(seed, base + (uint64_t)l) >> 11;
        uint64_t ru, rv;
        if (x < t_a) { ru = 0; rv = 0; }
        else if (x < t_ab) { ru = 0; rv = 1; }
        else if (x < t_abc) { ru = 1; rv = 0; }
        else { ru = 1; rv = 1; }
        u |= ru << l;
        v |= rv << l;
    }
    *pu = u;
    *pv = v;
}

/* Sample k of the graph (before permutation and cleaning). */
static inline void sample(int kind, uint64_t n, int scale, uint64_t es, uint64_t k, uint64_t* u, uint64_t* v) {
    if (kind == GG_KRON) {
        kron_sample(es, scale, k, u, v);
    } else {
        *u = gg_bounded(gg_rand(es, 2 * k), n);
        *v = gg_bounded(gg_rand(es, 2 * k + 1), n);
    }
}

/* Seeded Fisher-Yates permutation of [0, n). */
void gg_perm(uint64_t n, uint64_t seed, uint64_t* perm) {
    uint64_t ps = seed_perm(seed);
    for (uint64_t i = 0; i < n; i++) perm[i] = i;
    for (uint64_t i = n; i > 1; i--) {
        uint64_t j = gg_bounded(gg_rand(ps, i - 1), i);
        uint64_t t = perm[i - 1];
        perm[i - 1] = perm[j];
        perm[j] = t;
    }
}

/* Raw samples k0 .. k0+count-1, after relabelling by perm (NULL = identity). */
void gg_sample(int kind, uint64_t n, int scale, uint64_t seed, const uint64_t* perm,
               uint64_t k0, uint64_t count, uint64_t* src, uint64_t* dst) {
    uint64_t es = seed_edges(seed);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        uint64_t u, v;
        sample(kind, n, scale, es, k0 + (uint64_t)i, &u, &v);
        if (perm) { u = perm[u]; v = perm[v]; }
        src[i] = u;
        dst[i] = v;
    }
}

/* Pass 1: raw (symmetrised, self-loops dropped, duplicates kept) degree of each
 * vertex.  deg[] must hold n zeros. */
void gg_count(int kind, uint64_t n, int scale, uint64_t seed, const uint64_t* perm,
              uint64_t nsamples, uint64_t* deg) {
    uint64_t es = seed_edges(seed);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)nsamples; k++) {
        uint64_t u, v;
        sample(kind, n, scale, es, (uint64_t)k, &u, &v);
        if (perm) { u = perm[u]; v = perm[v]; }
        if (u == v) continue;
#pragma omp atomic
        deg[u]++;
#pragma omp atomic
        deg[v]++;
    }
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

static void sort_row(uint64_t* a, uint64_t len) {
    if (len < 24) {
        for (uint64_t i = 1; i < len; i++) {
            uint64_t x = a[i];
            uint64_t j = i;
            while (j > 0 && a[j - 1] > x) { a[j] = a[j - 1]; j--; }
            a[j] = x;
        }
    } else {
        qsort(a, (size_t)len, sizeof(uint64_t), cmp_u64);
    }
}

/* Pass 2: scatter every cleaned sample into its raw row (off_raw from pass 1),
 * then sort and de-duplicate each row in place.  cursor[] is scratch of n
 * entries.  deg_out[v] receives the de-duplicated degree. */
void gg_fill(int kind, uint64_t n, int scale, uint64_t seed, const uint64_t* perm,
             uint64_t nsamples, const uint64_t* off_raw, uint64_t* cursor,
             uint64_t* cols_raw, uint64_t* deg_out) {
    uint64_t es = seed_edges(seed);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; v++) cursor[v] = off_raw[v];
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < (int64_t)nsamples; k++) {
        uint64_t u, v, p, q;
        sample(kind, n, scale, es, (uint64_t)k, &u, &v);
        if (perm) { u = perm[u]; v = perm[v]; }
        if (u == v) continue;
#pragma omp atomic capture
        p = cursor[u]++;
#pragma omp atomic capture
        q = cursor[v]++;
        cols_raw[p] = v;
        cols_raw[q] = u;
    }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        uint64_t b = off_raw[v], len = off_raw[v + 1] - b;
        uint64_t* row = cols_raw + b;
        sort_row(row, len);
        uint64_t w = 0;
        for (uint64_t i = 0; i < len; i++)
            if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
        deg_out[v] = w;
    }
}

/* Pass 3: move each de-duplicated row to its final place (rows only move
 * towards lower addresses, so an in-order sequential memmove is safe) and
 * write the final offsets. */
void gg_compact(uint64_t n, const uint64_t* off_raw, const uint64_t* deg, uint64_t* cols,
                uint64_t* off_out) {
    uint64_t o = 0;
    for (uint64_t v = 0; v < n; v++) {
        off_out[v] = o;
        if (o != off_raw[v] && deg[v]) memmove(cols + o, cols + off_raw[v], deg[v] * sizeof(uint64_t));
        o += deg[v];
    }
    off_out[n] = o;
}

/* Symmetric edge weights in [1, 255] for every stored edge. */
void gg_weights(uint64_t n, const uint64_t* off, const uint64_t* cols, uint64_t seed, uint32_t* w) {
    uint64_t ws = gg_mix(seed ^ 0x57474854ULL);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        for (uint64_t i = off[v]; i < off[v + 1]; i++) {
            uint64_t u = cols[i];
            uint64_t a = (uint64_t)v < u ? (uint64_t)v : u;
            uint64_t b = (uint64_t)v < u ? u : (uint64_t)v;
            uint64_t h = gg_mix(gg_mix(ws ^ a) + b * GG_GAMMA);
            w[i] = 1u + (uint32_t)(h % 255u);
        }
    }
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
