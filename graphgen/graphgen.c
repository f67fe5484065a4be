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
 *     quadrant per bit level with probabilities (0.57, 0.19, 0.19, 0.05),
 *     quantised to multiples of 2^-16 (four levels per 64-bit random value);
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

/* Kronecker quadrant choice of one bit level from a 16-bit uniform integer x:
 * (u bit, v bit) = (0,0) below 0.57, (0,1) below 0.76, (1,0) below 0.95, else
 * (1,1); thresholds are the probabilities times 2^16, rounded.  Each 64-bit
 * output of the sample's stream gives four levels (bits 0-15 the lowest
 * level), so a scale-27 sample takes 7 outputs.  Written without branches:
 * the four outcomes are about equally hard to predict. */
#define GG_KRON_A 37356u   /* 0.57 * 2^16 */
#define GG_KRON_AB 49807u  /* 0.76 * 2^16 */
#define GG_KRON_ABC 62259u /* 0.95 * 2^16 */
static inline int kron_draws(int scale) { return (scale + 3) / 4; }
static inline void kron_sample(uint64_t seed, int scale, uint64_t k, uint64_t* pu, uint64_t* pv) {
    const int draws = kron_draws(scale);
    uint64_t u = 0, v = 0;
    /* output i of the stream is gg_mix(seed + (i + 1) * GAMMA): step z by GAMMA */
    uint64_t z = seed + (k * (uint64_t)draws + 1) * GG_GAMMA;
    for (int d = 0; d < draws; d++, z += GG_GAMMA) {
        const uint64_t r = gg_mix(z);
        for (int j = 0; j < 4; j++) {
            const uint32_t x = (uint32_t)(r >> (16 * j)) & 0xFFFFu;
            const uint64_t ru = x >= GG_KRON_AB;
            const uint64_t rv = (uint64_t)(x >= GG_KRON_A) ^ ru ^ (uint64_t)(x >= GG_KRON_ABC);
            u |= ru << (4 * d + j);
            v |= rv << (4 * d + j);
        }
    }
    const uint64_t mask = scale >= 64 ? ~0ull : ((1ull << scale) - 1ull);
    *pu = u & mask;
    *pv = v & mask;
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

/* Seeded relabelling of Kronecker vertex ids: a bijection of [0, 2^scale)
 * computed from the id (no table lookup, so placing a sample costs no random
 * memory access).  Four rounds of x -> (a x + b) mod 2^scale with a odd,
 * then x ^= x >> ceil(scale / 2); each step is a bijection on scale-bit
 * integers, so their composition is one.  The round keys come from the
 * permutation stream of the seed. */
#define GG_RELABEL_ROUNDS 4
typedef struct {
    uint64_t a[GG_RELABEL_ROUNDS], b[GG_RELABEL_ROUNDS], mask;
    int shift;
} gg_relabel_key;

static gg_relabel_key relabel_key(uint64_t seed, int scale) {
    gg_relabel_key k;
    uint64_t ps = seed_perm(seed);
    k.mask = scale >= 64 ? ~0ull : ((1ull << scale) - 1ull);
    k.shift = (scale + 1) / 2;
    for (int r = 0; r < GG_RELABEL_ROUNDS; r++) {
        k.a[r] = gg_rand(ps, 2 * (uint64_t)r) | 1ull;
        k.b[r] = gg_rand(ps, 2 * (uint64_t)r + 1);
    }
    return k;
}

static inline uint64_t relabel(const gg_relabel_key* k, uint64_t x) {
    for (int r = 0; r < GG_RELABEL_ROUNDS; r++) {
        x = (x * k->a[r] + k->b[r]) & k->mask;
        if (k->shift > 0) x ^= x >> k->shift;
    }
    return x;
}

/* The relabelling as a table: perm[x] = new id of x, for x < 2^scale. */
void gg_relabel_table(int scale, uint64_t seed, uint64_t* perm) {
    gg_relabel_key k = relabel_key(seed, scale);
    const uint64_t n = 1ull << scale;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < (int64_t)n; x++) perm[x] = relabel(&k, (uint64_t)x);
}

/* Sample k of the graph after relabelling (Kronecker with `permute`). */
static inline void sample_final(int kind, uint64_t n, int scale, uint64_t es, const gg_relabel_key* rk,
                                uint64_t k, uint64_t* u, uint64_t* v) {
    sample(kind, n, scale, es, k, u, v);
    if (rk) { *u = relabel(rk, *u); *v = relabel(rk, *v); }
}

/* Raw samples k0 .. k0+count-1 (relabelled when `permute`; Kronecker only). */
void gg_sample(int kind, uint64_t n, int scale, uint64_t seed, int permute,
               uint64_t k0, uint64_t count, uint64_t* src, uint64_t* dst) {
    uint64_t es = seed_edges(seed);
    gg_relabel_key rk = relabel_key(seed, scale);
    const gg_relabel_key* prk = (permute && kind == GG_KRON) ? &rk : NULL;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < (int64_t)count; i++) {
        uint64_t u, v;
        sample_final(kind, n, scale, es, prk, k0 + (uint64_t)i, &u, &v);
        src[i] = u;
        dst[i] = v;
    }
}

/* The samples are split into T contiguous parts; part t (taken by one thread,
 * the same part in both passes) keeps its own uint32 count per vertex in
 * cnt[t * n + v], so neither pass needs an atomic update: a thread counts and
 * later places only its own samples.  With fewer threads than parts, a thread
 * takes parts t, t + threads, ... (the result does not depend on which
 * thread takes a part). */
static inline uint64_t part_begin(uint64_t nsamples, int T, int t) {
    return (uint64_t)(((unsigned __int128)nsamples * (unsigned)t) / (unsigned)T);
}

#ifdef _OPENMP
#define GG_THREAD_ID() omp_get_thread_num()
#define GG_THREADS() omp_get_num_threads()
#else
#define GG_THREAD_ID() 0
#define GG_THREADS() 1
#endif

/* Both passes take a part's samples in batches: a batch is generated first
 * (prefetching the counters it will touch), then its updates run back to
 * back, so that a core keeps many random memory accesses in flight instead
 * of one per sample (the generation work between two updates otherwise fills
 * the out-of-order window).  The order of the updates within a part is the
 * samples' order either way. */
#define GG_BATCH 512

/* Pass 1: raw (symmetrised, self-loops dropped, duplicates kept) degree of
 * each vertex.  cnt[] is T * n uint32 of scratch (zeroed here, each part's
 * counts by the thread that takes the part); on return deg[v] is the raw
 * degree of v and cnt[t * n + v] is the number of row-v entries that parts
 * before t place (part t's first slot within row v). */
void gg_count(int kind, uint64_t n, int scale, uint64_t seed, int permute, uint64_t nsamples, int T,
              uint32_t* cnt, uint64_t* deg) {
    uint64_t es = seed_edges(seed);
    gg_relabel_key rk = relabel_key(seed, scale);
    const gg_relabel_key* prk = (permute && kind == GG_KRON) ? &rk : NULL;
#pragma omp parallel
    {
        const int nt = GG_THREADS(), me = GG_THREAD_ID();
        uint64_t bu[GG_BATCH], bv[GG_BATCH];
        for (int t = me; t < T; t += nt) {
            uint32_t* c = cnt + (uint64_t)t * n;
            memset(c, 0, n * sizeof(uint32_t));
            const uint64_t k1 = part_begin(nsamples, T, t + 1);
            uint64_t k = part_begin(nsamples, T, t);
            while (k < k1) {
                int nb = 0;
                for (; nb < GG_BATCH && k < k1; k++) {
                    uint64_t u, v;
                    sample_final(kind, n, scale, es, prk, k, &u, &v);
                    if (u == v) continue;
                    __builtin_prefetch(c + u, 1);
                    __builtin_prefetch(c + v, 1);
                    bu[nb] = u;
                    bv[nb] = v;
                    nb++;
                }
                for (int i = 0; i < nb; i++) {
                    c[bu[i]]++;
                    c[bv[i]]++;
                }
            }
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < (int64_t)n; v++) {
        uint64_t run = 0;
        for (int t = 0; t < T; t++) {
            const uint32_t x = cnt[(uint64_t)t * n + (uint64_t)v];
            cnt[(uint64_t)t * n + (uint64_t)v] = (uint32_t)run;
            run += x;
        }
        deg[v] = run;
    }
}

/* Pass 2: place every cleaned sample in its raw row (off_raw from the raw
 * degrees of pass 1; part t writes row v from slot cnt[t * n + v] on).  The
 * rows' contents do not depend on the parts' order; the sort of pass 3 makes
 * the result canonical. */
void gg_fill(int kind, uint64_t n, int scale, uint64_t seed, int permute, uint64_t nsamples, int T,
             uint32_t* cnt, const uint64_t* off_raw, uint64_t* cols_raw) {
    uint64_t es = seed_edges(seed);
    gg_relabel_key rk = relabel_key(seed, scale);
    const gg_relabel_key* prk = (permute && kind == GG_KRON) ? &rk : NULL;
#pragma omp parallel
    {
        const int nt = GG_THREADS(), me = GG_THREAD_ID();
        uint64_t bu[GG_BATCH], bv[GG_BATCH], pu[GG_BATCH], pv[GG_BATCH];
        for (int t = me; t < T; t += nt) {
            uint32_t* c = cnt + (uint64_t)t * n;
            const uint64_t k1 = part_begin(nsamples, T, t + 1);
            uint64_t k = part_begin(nsamples, T, t);
            while (k < k1) {
                int nb = 0;
                for (; nb < GG_BATCH && k < k1; k++) {
                    uint64_t u, v;
                    sample_final(kind, n, scale, es, prk, k, &u, &v);
                    if (u == v) continue;
                    __builtin_prefetch(c + u, 1);
                    __builtin_prefetch(c + v, 1);
                    __builtin_prefetch(off_raw + u, 0);
                    __builtin_prefetch(off_raw + v, 0);
                    bu[nb] = u;
                    bv[nb] = v;
                    nb++;
                }
                for (int i = 0; i < nb; i++) {
                    pu[i] = off_raw[bu[i]] + c[bu[i]]++;
                    pv[i] = off_raw[bv[i]] + c[bv[i]]++;
                    __builtin_prefetch(cols_raw + pu[i], 1);
                    __builtin_prefetch(cols_raw + pv[i], 1);
                }
                for (int i = 0; i < nb; i++) {
                    cols_raw[pu[i]] = bv[i];
                    cols_raw[pv[i]] = bu[i];
                }
            }
        }
    }
}

/* Ascending sort of one row: insertion sort for short rows, else quicksort
 * (median of three, Hoare partition, the smaller side by recursion and the
 * larger by looping) with a heapsort fallback once the depth passes
 * 2 log2(len). */
static void insertion_u64(uint64_t* a, uint64_t len) {
    for (uint64_t i = 1; i < len; i++) {
        uint64_t x = a[i];
        uint64_t j = i;
        while (j > 0 && a[j - 1] > x) { a[j] = a[j - 1]; j--; }
        a[j] = x;
    }
}

static void sift_down_u64(uint64_t* a, uint64_t root, uint64_t len) {
    for (;;) {
        uint64_t c = 2 * root + 1;
        if (c >= len) return;
        if (c + 1 < len && a[c + 1] > a[c]) c++;
        if (a[root] >= a[c]) return;
        uint64_t t = a[root]; a[root] = a[c]; a[c] = t;
        root = c;
    }
}

static void heapsort_u64(uint64_t* a, uint64_t len) {
    for (uint64_t i = len / 2; i-- > 0;) sift_down_u64(a, i, len);
    for (uint64_t end = len; end-- > 1;) {
        uint64_t t = a[0]; a[0] = a[end]; a[end] = t;
        sift_down_u64(a, 0, end);
    }
}

static void introsort_u64(uint64_t* a, uint64_t len, int depth) {
    while (len > 24) {
        if (depth-- <= 0) { heapsort_u64(a, len); return; }
        uint64_t x = a[0], y = a[len / 2], z = a[len - 1];
        uint64_t pivot = x < y ? (y < z ? y : (x < z ? z : x)) : (x < z ? x : (y < z ? z : y));
        /* the median of three keeps 1 <= left <= len - 1, so both sides shrink */
        uint64_t i = 0, j = len - 1;
        for (;;) {
            while (a[i] < pivot) i++;
            while (a[j] > pivot) j--;
            if (i >= j) break;
            uint64_t t = a[i]; a[i] = a[j]; a[j] = t;
            i++; j--;
        }
        uint64_t left = j + 1; /* a[0..left) <= pivot <= a[left..len) */
        if (left < len - left) { introsort_u64(a, left, depth); a += left; len -= left; }
        else { introsort_u64(a + left, len - left, depth); len = left; }
    }
    insertion_u64(a, len);
}

static void sort_row(uint64_t* a, uint64_t len) {
    int depth = 0;
    for (uint64_t l = len; l > 1; l >>= 1) depth += 2;
    introsort_u64(a, len, depth);
}

/* Sorts and de-duplicates the rows of v in [lo, hi) (raw rows from off_raw)
 * and packs them, in order, from cols[off_raw[lo]] on; deg[v] receives the
 * de-duplicated degree.  Returns the packed length.  Rows only move towards
 * lower addresses inside the block, so a forward memmove is safe. */
static uint64_t sort_pack_block(uint64_t lo, uint64_t hi, const uint64_t* off_raw, uint64_t* cols, uint64_t* deg) {
    uint64_t o = off_raw[lo];
    for (uint64_t v = lo; v < hi; v++) {
        const uint64_t b = off_raw[v], len = off_raw[v + 1] - b;
        uint64_t* row = cols + b;
        sort_row(row, len);
        uint64_t w = 0;
        for (uint64_t i = 0; i < len; i++)
            if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
        if (o != b && w) memmove(cols + o, row, w * sizeof(uint64_t));
        deg[v] = w;
        o += w;
    }
    return o - off_raw[lo];
}

/* Pass 3: sort and de-duplicate every row and pack the rows into the final
 * CSR in place; off_out[v] receives the final offsets (n + 1 entries).
 * blk_len is scratch of nblocks entries.  Vertices are cut into nblocks
 * blocks; each block is packed at the start of its own raw region in
 * parallel, then the blocks move to their final places in order (a block's
 * destination can only overlap its own source or the source of a block
 * already moved).  A block whose shift is at least its length overlaps
 * nothing and is copied by all threads at once; otherwise one memmove. */
void gg_finish(uint64_t n, const uint64_t* off_raw, uint64_t* cols, uint64_t nblocks, uint64_t* blk_len,
               uint64_t* deg, uint64_t* off_out) {
    if (nblocks < 1) nblocks = 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < (int64_t)nblocks; b++) {
        const uint64_t lo = n * (uint64_t)b / nblocks, hi = n * (uint64_t)(b + 1) / nblocks;
        blk_len[b] = sort_pack_block(lo, hi, off_raw, cols, deg);
    }
    uint64_t dst = 0;
    for (uint64_t b = 0; b < nblocks; b++) {
        const uint64_t lo = n * b / nblocks, hi = n * (b + 1) / nblocks;
        const uint64_t src = off_raw[lo], len = blk_len[b];
        uint64_t o = dst;
        for (uint64_t v = lo; v < hi; v++) { off_out[v] = o; o += deg[v]; }
        if (src != dst && len) {
            if (src - dst >= len) {
                const uint64_t chunk = 1u << 14;
                const int64_t nchunks = (int64_t)((len + chunk - 1) / chunk);
#pragma omp parallel for schedule(static) if (nchunks > 4)
                for (int64_t c = 0; c < nchunks; c++) {
                    const uint64_t a = (uint64_t)c * chunk, e = a + chunk < len ? a + chunk : len;
                    memcpy(cols + dst + a, cols + src + a, (e - a) * sizeof(uint64_t));
                }
            } else {
                memmove(cols + dst, cols + src, len * sizeof(uint64_t));
            }
        }
        dst += len;
    }
    off_out[n] = dst;
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
