/*
 * Seeded synthetic graph generators shared by the tests, the oracle's test
 * inputs and the benchmark.  This file holds none of the sampling method's
 * arithmetic: no Philox, no liveness rule, no traversal.  Its random numbers
 * come from the SplitMix64 output function applied to a counter (Steele,
 * Lea and Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014), so every draw is a pure function of (seed, stream, index) and
 * the generated graph is identical on any machine and any thread count.
 *
 * Graph layout produced here (the library's input format): an in-edge CSR.
 * Row v of (row_ptr, col) lists the sources w of the edges w -> v, strictly
 * ascending, with self-loops and duplicate edges removed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Draw number `i` of stream `stream` under `seed`. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t base = mix64(seed ^ mix64(stream + 0x9E3779B97F4A7C15ULL));
    return mix64(base + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Uniform integer in [0, bound) by the 64x64 -> high-64 multiply. */
static inline uint64_t below(uint64_t r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)r * bound) >> 64);
}

uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i) { return draw(seed, stream, i); }

int synth_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* Sort every row ascending and drop duplicates in place, then close the gaps.
 * `cnt` holds the raw row lengths; rows start at `start`.  Writes the final
 * row_ptr and compacts `col`.  Returns the final edge count. */
static uint64_t finish_rows(uint32_t n, uint64_t* start, uint32_t* col, uint64_t* row_ptr) {
    uint64_t* keep = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        uint32_t* r = col + start[v];
        uint64_t len = start[v + 1] - start[v];
        if (len > 1) qsort(r, len, sizeof(uint32_t), cmp_u32);
        uint64_t k = 0;
        for (uint64_t j = 0; j < len; ++j)
            if (k == 0 || r[j] != r[k - 1]) r[k++] = r[j];
        keep[v] = k;
    }
    row_ptr[0] = 0;
    for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] = row_ptr[v] + keep[v];
    /* Compact left to right: row v moves from start[v] to row_ptr[v] <= start[v]. */
    for (uint32_t v = 0; v < n; ++v)
        if (row_ptr[v] != start[v]) memmove(col + row_ptr[v], col + start[v], keep[v] * sizeof(uint32_t));
    free(keep);
    return row_ptr[n];
}

/* Directed Erdos-Renyi G(n, m): m distinct ordered pairs (u, v), u != v, drawn
 * uniformly by rejection.  n <= 65536 (an n*n bitmap marks drawn pairs).
 * Output: in-CSR (row_ptr[n+1], col[m]).  Returns 0, or -1 on bad arguments. */
int synth_er(uint32_t n, uint64_t m, uint64_t seed, uint64_t* row_ptr, uint32_t* col) {
    if (n < 2 || n > 65536 || m > (uint64_t)n * (n - 1)) return -1;
    uint64_t words = ((uint64_t)n * n + 63) / 64;
    uint64_t* seen = (uint64_t*)calloc(words, sizeof(uint64_t));
    uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * m);
    uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * m);
    if (!seen || !src || !dst) { free(seen); free(src); free(dst); return -2; }
    uint64_t got = 0, i = 0;
    while (got < m) {
        uint64_t r = draw(seed, 1, i++);
        uint32_t u = (uint32_t)below(r, n);
        uint32_t v = (uint32_t)below(draw(seed, 2, i), n);
        if (u == v) continue;
        uint64_t key = (uint64_t)u * n + v;
        if (seen[key >> 6] >> (key & 63) & 1) continue;
        seen[key >> 6] |= 1ULL << (key & 63);
        src[got] = u; dst[got] = v; ++got;
    }
    memset(row_ptr, 0, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t j = 0; j < m; ++j) row_ptr[dst[j] + 1]++;
    for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    uint64_t* cur = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    memcpy(cur, row_ptr, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t j = 0; j < m; ++j) col[cur[dst[j]]++] = src[j];
    for (uint32_t v = 0; v < n; ++v)
        qsort(col + row_ptr[v], row_ptr[v + 1] - row_ptr[v], sizeof(uint32_t), cmp_u32);
    free(cur); free(seen); free(src); free(dst);
    return 0;
}

/* Seeded random permutation of [0, n) (Fisher-Yates, sequential). */
static void permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n - 1; i > 0; --i) {
        uint32_t j = (uint32_t)below(draw(seed, 7, i), (uint64_t)i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): 2^scale vertices,
 * ef * 2^scale raw edges.  Each raw edge picks one of the four quadrants
 * (a: src 0 dst 0, b: src 0 dst 1, c: src 1 dst 0, d: src 1 dst 1) at every
 * level, most significant bit first, from a 32-bit draw compared with the
 * cumulative integer thresholds floor(a*2^32) etc.  Vertex ids are then
 * relabelled by a seeded random permutation (when `permute`), self-loops and
 * duplicates are dropped and each in-row is sorted by source.
 * `col` must hold ef * 2^scale entries; row_ptr holds 2^scale + 1.
 * Returns the final edge count, or UINT64_MAX on bad arguments. */
uint64_t synth_rmat(uint32_t scale, uint32_t ef, double a, double b, double c, uint64_t seed,
                    int permute, uint64_t* row_ptr, uint32_t* col) {
    if (scale < 1 || scale > 30 || ef < 1) return UINT64_MAX;
    const uint32_t n = 1u << scale;
    const uint64_t m_raw = (uint64_t)ef * n;
    const uint64_t ta = (uint64_t)(a * 4294967296.0);
    const uint64_t tab = (uint64_t)((a + b) * 4294967296.0);
    const uint64_t tabc = (uint64_t)((a + b + c) * 4294967296.0);
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * m_raw);
    uint32_t* dst = (uint32_t*)malloc(sizeof(uint32_t) * m_raw);
    uint64_t* start = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!perm || !src || !dst || !start) { free(perm); free(src); free(dst); free(start); return UINT64_MAX; }
    if (permute) permutation(n, seed, perm);
    else for (uint32_t i = 0; i < n; ++i) perm[i] = i;

    #pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < (int64_t)m_raw; ++j) {
        uint32_t u = 0, v = 0;
        uint64_t r = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            if ((lvl & 1) == 0) r = draw(seed, 3, (uint64_t)j * 16 + (lvl >> 1));
            uint64_t x = (lvl & 1) ? (r >> 32) : (r & 0xFFFFFFFFULL);
            uint32_t su = 0, sv = 0;
            if (x < ta) { su = 0; sv = 0; }
            else if (x < tab) { su = 0; sv = 1; }
            else if (x < tabc) { su = 1; sv = 0; }
            else { su = 1; sv = 1; }
            u = (u << 1) | su;
            v = (v << 1) | sv;
        }
        src[j] = perm[u];
        dst[j] = perm[v];
    }
    /* Counting sort by destination (self-loops dropped). */
    for (uint64_t j = 0; j < m_raw; ++j)
        if (src[j] != dst[j]) start[dst[j] + 1]++;
    for (uint32_t v = 0; v < n; ++v) start[v + 1] += start[v];
    uint64_t* cur = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    memcpy(cur, start, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t j = 0; j < m_raw; ++j)
        if (src[j] != dst[j]) col[cur[dst[j]]++] = src[j];
    free(cur); free(src); free(dst); free(perm);
    uint64_t m = finish_rows(n, start, col, row_ptr);
    free(start);
    return m;
}

/* Per-edge independent-cascade thresholds.  The library takes the edge
 * probability p(e) as the integer floor(p * 2^32); 0xFFFFFFFF marks an edge
 * that is always live (p = 1). */
static inline uint32_t thr_of(double p) {
    if (!(p > 0.0)) return 0;
    if (p >= 1.0) return 0xFFFFFFFFu;
    double t = p * 4294967296.0;          /* exact: scaling by a power of two */
    uint64_t f = (uint64_t)t;              /* floor for t >= 0 */
    return f >= 0xFFFFFFFFULL ? 0xFFFFFFFFu : (uint32_t)f;
}

void synth_thr_uniform(uint64_t m, double p, uint32_t* thr) {
    uint32_t t = thr_of(p);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; ++e) thr[e] = t;
}

/* Weighted cascade: p(w -> v) = 1 / indeg(v), as floor(2^32 / d) in integer
 * arithmetic; indeg 1 gives the always-live marker. */
void synth_thr_wc(uint32_t n, const uint64_t* row_ptr, uint32_t* thr) {
    #pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < (int64_t)n; ++v) {
        uint64_t d = row_ptr[v + 1] - row_ptr[v];
        uint32_t t = d == 1 ? 0xFFFFFFFFu : (uint32_t)(4294967296ULL / (d ? d : 1));
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) thr[e] = t;
    }
}

/* Trivalency: each edge gets one of the given probabilities, uniformly. */
void synth_thr_choice(uint64_t m, const double* ps, uint32_t k, uint64_t seed, uint32_t* thr) {
    uint32_t ts[16];
    for (uint32_t i = 0; i < k && i < 16; ++i) ts[i] = thr_of(ps[i]);
    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < (int64_t)m; ++e) thr[e] = ts[below(draw(seed, 11, (uint64_t)e), k)];
}

uint32_t synth_thr_of(double p) { return thr_of(p); }
