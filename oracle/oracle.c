/*
 * CPU oracle for fused breadth-first probabilistic traversals (BPTs) under
 * the independent-cascade (IC) model.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the graft entry's smoke check and
 * the benchmark's CPU-baseline leg load this code.  It shares no source with
 * the CUDA library: its Philox, its liveness test, its traversals and its
 * greedy selection are written out here, plainly, from their definitions.
 *
 * What it computes (all integer arithmetic, so results are exact):
 *
 *  - Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror and
 *    Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): ten rounds
 *    of the Philox S-box over a 4x32-bit counter with a 2x32-bit key that is
 *    bumped by the Weyl constants between rounds.
 *
 *  - Edge liveness for sample s and edge e (the paper's Listing 1 draws
 *    random(0,1) per colour and edge and drops the colour when it exceeds
 *    e.prob; Section 2 fixes that the draws are independent per edge and per
 *    sample).  Here the draw is the Philox word out[e & 3] of the counter
 *    (lo(s), hi(s), lo(e>>2), hi(e>>2)) under key (lo(seed), hi(seed)), and
 *    the edge is live iff thr[e] == 0xFFFFFFFF or draw < thr[e], where
 *    thr[e] = floor(p(e) * 2^32) is given as input.
 *
 *  - Start vertex of sample s (Section 3: BPTs start at vertices chosen
 *    uniformly at random): R = out[1] << 32 | out[0] of the counter
 *    (lo(s), hi(s), 0, 0x80000000), start = floor(R * n / 2^64).
 *
 *  - RR sets (Definition 2): RR(s) = { u : a path u -> ... -> start(s) of
 *    edges live for s }.  oracle_rr runs one plain FIFO BFS per sample over
 *    the in-edges, and returns the rows in sample-id order, each sorted
 *    ascending.  This is the definition written out.
 *
 *  - oracle_rr_fused follows Listing 1 (Section 3) literally: colours of 64
 *    samples per mask word share one frontier array; an active vertex v
 *    takes fr_v = frontier[v] (and clears it), ORs it into visited[v], and
 *    pushes fr_v & ~visited[u] filtered by liveness into frontier[u] for every
 *    edge of v; RR sets are read off the visited masks vertex by vertex.  It
 *    also counts edge accesses (one per edge scanned per processing of an
 *    active vertex), the quantity Theorem 1 bounds.
 *
 *  - oracle_rr_lt: RR sets under the linear-threshold (LT) model (Section 2
 *    names IC and LT; Kempe et al.'s live-edge form of LT): each vertex v
 *    keeps at most one in-edge, edge e of its row with probability
 *    w(e) = thr[e] / 2^32 (0xFFFFFFFF read as 1), none with the rest.  For
 *    sample s the choice is one Philox draw r = out[0] of the counter
 *    (lo(s), hi(s), v, 0x40000000): the first edge e of the row with
 *    r < w(rs) + ... + w(e) (sums in units of 2^-32), none if r is beyond the
 *    row's total.  The RR set of s is the walk start(s) <- u1 <- u2 ... along
 *    the chosen in-edges, which ends at a vertex with no edge or at a vertex
 *    already on the walk.
 *
 *  - oracle_greedy: greedy maximum k-coverage over the RR sets (Section 2:
 *    seed selection reduces to max-k-cover).  Each round recounts, for every
 *    vertex, the RR sets that contain it and are not yet covered, and takes
 *    the largest count, the smallest vertex id on a tie; if every set is
 *    covered it takes the smallest unselected id.  Always k seeds.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Philox4x32-10 (Salmon et al., SC'11) --------------------------------- */

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)PHILOX_M0 * c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void oracle_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += PHILOX_W0; k[1] += PHILOX_W1; }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* ---- The liveness rule and the start draw ---------------------------------- */

uint32_t oracle_edge_draw(uint64_t seed, uint64_t s, uint64_t e) {
    uint64_t q = e >> 2;
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)q, (uint32_t)(q >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox(ctr, key, out);
    return out[e & 3];
}

int oracle_live(uint64_t seed, uint64_t s, uint64_t e, uint32_t thr) {
    if (thr == 0xFFFFFFFFu) return 1;
    return oracle_edge_draw(seed, s, e) < thr;
}

uint32_t oracle_start(uint64_t seed, uint64_t s, uint32_t n) {
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), 0u, 0x80000000u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox(ctr, key, out);
    uint64_t r = ((uint64_t)out[1] << 32) | out[0];
    return (uint32_t)(((unsigned __int128)r * n) >> 64);
}

/* ---- Plain per-sample BFS ------------------------------------------------- */

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

typedef struct {
    uint32_t* data;
    uint64_t len, cap;
} vec32;

static int vec_push(vec32* v, uint32_t x) {
    if (v->len == v->cap) {
        uint64_t nc = v->cap ? v->cap * 2 : 1024;
        uint32_t* d = (uint32_t*)realloc(v->data, nc * sizeof(uint32_t));
        if (!d) return -1;
        v->data = d; v->cap = nc;
    }
    v->data[v->len++] = x;
    return 0;
}

/* RR set of one sample: BFS from start(s) over in-edges, keeping an edge only
 * when it is live for s.  Appends the sorted set to `out`; returns its size.
 * `mark` (n entries) must hold values != tag on entry for every vertex. */
static uint64_t rr_one(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
                       uint64_t seed, uint64_t s, uint64_t* mark, uint64_t tag, vec32* queue,
                       vec32* out, uint32_t* start_out) {
    uint32_t st = oracle_start(seed, s, n);
    if (start_out) *start_out = st;
    queue->len = 0;
    vec_push(queue, st);
    mark[st] = tag;
    for (uint64_t head = 0; head < queue->len; ++head) {
        uint32_t v = queue->data[head];
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            uint32_t w = col[e];
            if (mark[w] == tag) continue;
            if (!oracle_live(seed, s, e, thr[e])) continue;
            mark[w] = tag;
            vec_push(queue, w);
        }
    }
    qsort(queue->data, queue->len, sizeof(uint32_t), cmp_u32);
    uint64_t base = out->len;
    for (uint64_t i = 0; i < queue->len; ++i) vec_push(out, queue->data[i]);
    return out->len - base;
}

/* ---- The linear-threshold model: one reverse walk per sample --------------- */

uint32_t oracle_vertex_draw(uint64_t seed, uint64_t s, uint32_t v) {
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), v, 0x40000000u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox(ctr, key, out);
    return out[0];
}

/* The in-edge vertex v keeps for sample s, or -1 for none. */
int64_t oracle_lt_choice(const uint64_t* row_ptr, const uint32_t* thr, uint64_t seed, uint64_t s, uint32_t v) {
    const uint64_t r = oracle_vertex_draw(seed, s, v);
    uint64_t acc = 0;
    for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        acc += thr[e] == 0xFFFFFFFFu ? (1ull << 32) : (uint64_t)thr[e];
        if (r < acc) return (int64_t)e;
    }
    return -1;
}

static uint64_t rr_one_lt(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
                          uint64_t seed, uint64_t s, uint64_t* mark, uint64_t tag, vec32* queue,
                          vec32* out, uint32_t* start_out) {
    uint32_t v = oracle_start(seed, s, n);
    if (start_out) *start_out = v;
    queue->len = 0;
    for (;;) {
        vec_push(queue, v);
        mark[v] = tag;
        const int64_t e = oracle_lt_choice(row_ptr, thr, seed, s, v);
        if (e < 0) break;
        const uint32_t u = col[e];
        if (mark[u] == tag) break;
        v = u;
    }
    qsort(queue->data, queue->len, sizeof(uint32_t), cmp_u32);
    uint64_t base = out->len;
    for (uint64_t i = 0; i < queue->len; ++i) vec_push(out, queue->data[i]);
    return out->len - base;
}

/* RR sets for `count` samples.  Sample j has id ids[j] when ids is non-NULL,
 * else first_id + j.  On success *offsets_out (count+1 entries) and *verts_out
 * are malloc'd (free with oracle_free); starts_out (count entries) is
 * optional.  threads <= 0 uses the OpenMP default.  Returns 0, or -1 when
 * memory runs out. */
static int rr_many(int lt, uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
                   uint64_t seed, uint64_t first_id, const uint64_t* ids, uint64_t count, int threads,
                   uint64_t** offsets_out, uint32_t** verts_out, uint32_t* starts_out) {
    const uint64_t CH = 256;
    uint64_t nchunks = (count + CH - 1) / CH;
    vec32* chunk = (vec32*)calloc(nchunks ? nchunks : 1, sizeof(vec32));
    uint64_t* sizes = (uint64_t*)calloc(count + 1, sizeof(uint64_t));
    if (!chunk || !sizes) { free(chunk); free(sizes); return -1; }
    int fail = 0;
#ifdef _OPENMP
    if (threads <= 0) threads = omp_get_max_threads();
#else
    threads = 1;
#endif
    #pragma omp parallel num_threads(threads)
    {
        uint64_t* mark = (uint64_t*)calloc(n, sizeof(uint64_t));
        vec32 queue = {0, 0, 0};
        #pragma omp for schedule(dynamic, 1)
        for (int64_t c = 0; c < (int64_t)nchunks; ++c) {
            if (!mark) { fail = 1; continue; }
            for (uint64_t j = (uint64_t)c * CH; j < count && j < (uint64_t)(c + 1) * CH; ++j) {
                uint64_t s = ids ? ids[j] : first_id + j;
                sizes[j] = (lt ? rr_one_lt : rr_one)(n, row_ptr, col, thr, seed, s, mark, j + 1, &queue, &chunk[c],
                                                     starts_out ? &starts_out[j] : NULL);
            }
        }
        free(mark);
        free(queue.data);
    }
    uint64_t* off = (uint64_t*)malloc((count + 1) * sizeof(uint64_t));
    if (!off || fail) { free(off); for (uint64_t c = 0; c < nchunks; ++c) free(chunk[c].data); free(chunk); free(sizes); return -1; }
    off[0] = 0;
    for (uint64_t j = 0; j < count; ++j) off[j + 1] = off[j] + sizes[j];
    uint32_t* verts = (uint32_t*)malloc((off[count] ? off[count] : 1) * sizeof(uint32_t));
    if (!verts) { free(off); for (uint64_t c = 0; c < nchunks; ++c) free(chunk[c].data); free(chunk); free(sizes); return -1; }
    for (uint64_t c = 0; c < nchunks; ++c) {
        uint64_t j0 = c * CH;
        if (chunk[c].len) memcpy(verts + off[j0], chunk[c].data, chunk[c].len * sizeof(uint32_t));
        free(chunk[c].data);
    }
    free(chunk);
    free(sizes);
    *offsets_out = off;
    *verts_out = verts;
    return 0;
}

int oracle_rr(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
              uint64_t seed, uint64_t first_id, const uint64_t* ids, uint64_t count, int threads,
              uint64_t** offsets_out, uint32_t** verts_out, uint32_t* starts_out) {
    return rr_many(0, n, row_ptr, col, thr, seed, first_id, ids, count, threads, offsets_out, verts_out, starts_out);
}

/* As oracle_rr, under the linear-threshold model (one reverse walk per sample). */
int oracle_rr_lt(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
                 uint64_t seed, uint64_t first_id, const uint64_t* ids, uint64_t count, int threads,
                 uint64_t** offsets_out, uint32_t** verts_out, uint32_t* starts_out) {
    return rr_many(1, n, row_ptr, col, thr, seed, first_id, ids, count, threads, offsets_out, verts_out, starts_out);
}

void oracle_free(void* p) { free(p); }

/* ---- Listing 1: fused traversal with colour masks --------------------------- */

/* Samples first_id .. first_id+count-1 are processed in groups of 64*W colours
 * (colour c of group g is sample first_id + g*64*W + c).  Rows are emitted in
 * sample order, each ascending.  *edge_accesses receives the number of
 * (active vertex, edge) pairs scanned over all groups.  Output as oracle_rr. */
int oracle_rr_fused(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* thr,
                    uint64_t seed, uint64_t first_id, uint64_t count, uint32_t W,
                    uint64_t** offsets_out, uint32_t** verts_out, uint64_t* edge_accesses) {
    if (W == 0) return -1;
    const uint64_t C = 64ull * W;
    uint64_t* frontier = (uint64_t*)calloc((size_t)n * W, sizeof(uint64_t));
    uint64_t* visited = (uint64_t*)calloc((size_t)n * W, sizeof(uint64_t));
    uint32_t* queue = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint8_t* queued = (uint8_t*)calloc(n, 1);
    uint64_t* off = (uint64_t*)malloc((count + 1) * sizeof(uint64_t));
    vec32* rows = (vec32*)calloc(C, sizeof(vec32));
    vec32 all = {0, 0, 0};
    if (!frontier || !visited || !queue || !queued || !off || !rows) {
        free(frontier); free(visited); free(queue); free(queued); free(off); free(rows);
        return -1;
    }
    uint64_t acc = 0;
    off[0] = 0;
    for (uint64_t g0 = 0; g0 < count; g0 += C) {
        uint64_t colours = count - g0 < C ? count - g0 : C;
        /* Frontier initialization: one colour per sample at its start. */
        uint64_t qh = 0, qt = 0;  /* ring buffer over n+1 slots */
        for (uint64_t c = 0; c < colours; ++c) {
            uint32_t st = oracle_start(seed, first_id + g0 + c, n);
            frontier[(size_t)st * W + c / 64] |= 1ull << (c % 64);
            if (!queued[st]) { queued[st] = 1; queue[qt] = st; qt = (qt + 1) % (n + 1); }
        }
        /* Fused random traversals. */
        while (qh != qt) {
            uint32_t v = queue[qh]; qh = (qh + 1) % (n + 1);
            queued[v] = 0;
            uint64_t fr_v[8];
            for (uint32_t i = 0; i < W; ++i) {
                fr_v[i] = frontier[(size_t)v * W + i];
                frontier[(size_t)v * W + i] = 0;
                visited[(size_t)v * W + i] |= fr_v[i];
            }
            for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                uint32_t u = col[e];
                ++acc;
                int any = 0;
                for (uint32_t i = 0; i < W; ++i) {
                    uint64_t fr_u = fr_v[i] & ~visited[(size_t)u * W + i];
                    for (int b = 0; b < 64; ++b) {
                        if (!(fr_u >> b & 1)) continue;
                        uint64_t s = first_id + g0 + 64ull * i + (uint64_t)b;
                        if (!oracle_live(seed, s, e, thr[e])) fr_u &= ~(1ull << b);
                    }
                    frontier[(size_t)u * W + i] |= fr_u;
                    any |= fr_u != 0;
                }
                if (any && !queued[u]) { queued[u] = 1; queue[qt] = u; qt = (qt + 1) % (n + 1); }
            }
        }
        /* RRR sets construction: vertex by vertex, colour by colour. */
        for (uint32_t v = 0; v < n; ++v)
            for (uint32_t i = 0; i < W; ++i) {
                uint64_t x = visited[(size_t)v * W + i];
                if (!x) continue;
                visited[(size_t)v * W + i] = 0;
                for (int b = 0; b < 64; ++b)
                    if (x >> b & 1) vec_push(&rows[64 * i + b], v);
            }
        for (uint64_t c = 0; c < colours; ++c) {
            for (uint64_t j = 0; j < rows[c].len; ++j) vec_push(&all, rows[c].data[j]);
            off[g0 + c + 1] = all.len;
            rows[c].len = 0;
        }
    }
    for (uint64_t c = 0; c < C; ++c) free(rows[c].data);
    free(rows); free(frontier); free(visited); free(queue); free(queued);
    if (!all.data) all.data = (uint32_t*)malloc(sizeof(uint32_t));
    *offsets_out = off;
    *verts_out = all.data;
    if (edge_accesses) *edge_accesses = acc;
    return 0;
}

/* ---- Greedy maximum k-coverage --------------------------------------------- */

/* seeds_out[k]; gains_out[k] (optional) receives the number of newly covered
 * sets each pick added.  Returns 0, -1 on k > n, -2 when memory runs out. */
int oracle_greedy(uint32_t n, uint64_t S, const uint64_t* offsets, const uint32_t* verts, uint32_t k,
                  uint32_t* seeds_out, uint64_t* gains_out) {
    if (k > n) return -1;
    uint8_t* covered = (uint8_t*)calloc(S ? S : 1, 1);
    uint8_t* selected = (uint8_t*)calloc(n, 1);
    uint64_t* count = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!covered || !selected || !count) { free(covered); free(selected); free(count); return -2; }
    for (uint32_t r = 0; r < k; ++r) {
        memset(count, 0, sizeof(uint64_t) * (size_t)n);
        for (uint64_t s = 0; s < S; ++s) {
            if (covered[s]) continue;
            for (uint64_t j = offsets[s]; j < offsets[s + 1]; ++j) count[verts[j]]++;
        }
        int64_t best = -1;
        for (uint32_t v = 0; v < n; ++v) {
            if (selected[v]) continue;
            if (best < 0 || count[v] > count[best]) best = v;
        }
        uint32_t u = (uint32_t)best;
        selected[u] = 1;
        seeds_out[r] = u;
        if (gains_out) gains_out[r] = count[u];
        for (uint64_t s = 0; s < S; ++s) {
            if (covered[s]) continue;
            for (uint64_t j = offsets[s]; j < offsets[s + 1]; ++j)
                if (verts[j] == u) { covered[s] = 1; break; }
        }
    }
    free(covered); free(selected); free(count);
    return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
