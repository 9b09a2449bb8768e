// The fused-BPT sampling engine (Section 3, Listing 1), with the adaptive
// future-work items of Section 9: (b) finished traversals hand their RR sets
// over early and new starts are injected mid-traversal.
//
// Colour lanes.  A vertex row holds WB 64-bit words, i.e. 64*WB colour lanes.
// Each lane carries one sample at a time: bit c of word i of visited[v] means
// "the sample held by lane 64i+c has reached v".  All lanes share one
// frontier: a frontier unit is a vertex with the non-zero words of its new
// mask, and the in-edges of a unit are read once per level for all of its
// colours (Listing 1's fusing update, over every sample in flight).  When a
// lane's sample stops (no unit carries its bit), the next level sweeps the
// lane's own list of reached vertices (a segment of seg_cap entries, then a
// shared spill log) into (sample, vertex) pairs, clears the lane's bit from
// visited[], and the lane takes the next sample id (lane refill); or, in
// batch mode, lanes wait until the whole row has finished, which is the plain
// fused algorithm of Listing 1 with 64*WB colours per group.
//
// One level ("tick") has five phases:
//   sweep    finished lanes: RR pairs out, bits cleared, spill log compacted
//   expand   frontier units x 4-edge groups -> next rows, pending vertices
//   commit   pending vertices -> visited, new frontier list, lane entry lists
//   schedule (one CTA) finished lanes, refills, loop condition
//   init     start vertices of lanes assigned a new sample
// They run as three kernels per level (host loop or CUDA-graph WHILE loop):
// init, expand and sweep in one kernel (init first, the sweep in its tail), the
// commit, and the scheduler CTA; a level that expands by filtered push or pull
// adds a second expand kernel.  Or inside one persistent cooperative kernel,
// where sweep, init and expand of a level share a phase and bounded grid
// barriers separate the phases.
//
// Liveness never reads visited[]: the expand draws for every colour of the
// frontier mask and the commit removes colours a vertex has already seen.
// The result is the same closure (each colour reaches each vertex once), and
// the hot loop streams col/thr with 128-bit loads instead of gathering masks.
#include <algorithm>
#include <cstring>
#include <vector>
#include <string>

#include "internal.cuh"

namespace fbpt {
namespace {

constexpr int kThreads = 256;
// dynamic shared memory of the expand kernels: two slots per warp of 32 lanes x
// four 16-byte vectors (the next wide chunk's thresholds and sources)
constexpr size_t kStageBytes = (kThreads / 32) * 2 * 32 * 4 * sizeof(uint4);
#ifndef FBPT_EXPAND_ILP
#define FBPT_EXPAND_ILP 1   // chunks a warp works on at once in the expand
#endif
#ifndef FBPT_COMMIT_VPW_MIN
#define FBPT_COMMIT_VPW_MIN 8  // fewest pending vertices a commit warp takes
#endif
#ifndef FBPT_EXPAND_MINB
#define FBPT_EXPAND_MINB 3  // resident CTAs per SM the expand kernel is compiled for
#endif


__device__ __forceinline__ uint64_t row_groups(uint64_t rs, uint64_t re) {
    return re > rs ? ((re - 1) >> 2) - (rs >> 2) + 1 : 0;
}

// Data written by other CTAs in an earlier phase of the persistent kernel is
// read through L2 (ld.global.cg), never from a possibly stale L1 line.
template <typename T>
__device__ __forceinline__ T L2(const T* p) { return __ldcg(p); }

// Loads of data no kernel writes while the expand runs (frontier list, chunk
// map, stage words): through the read-only cache in the per-level kernels,
// through L2 in the persistent kernel, whose levels rewrite them in place.
template <bool ro, typename T>
__device__ __forceinline__ T LD(const T* p) {
    if constexpr (ro) return __ldg(p);
    else return __ldcg(p);
}

// Commit scratch of one warp: its 32 pending vertices and what their words add.
struct CommitWarp {
    uint64_t m[32];                 // words of next[w] that changed this level
    uint32_t w[32];
    uint32_t start[32];             // first (vertex, word) item of each vertex
    uint32_t row[32];               // stage row of each vertex
    uint32_t occ_lo[32], occ_hi[32];
    uint32_t bits[32];
    uint32_t he[32];                // vertex has in-edges
    // RR-list entries of the current 32 items, flattened across the warp
    uint64_t ex[32];                // new colours of each item
    uint32_t el[32];                // its first lane (64 * word)
    uint32_t ev[32];                // its vertex
    uint32_t es[32];                // its first entry
};

struct SchedHead {
    unsigned long long next_j, pair_cursor, new_packed, new_colours, tick, tick_limit;
    unsigned long long list_count, list_groups, list_colours;
    unsigned long long wide_packed, wide_gnew, wide_units, wide_groups;
    unsigned long long ph_t0[3], ph_t1[3], spill_len[2];
    uint32_t err, refill, sched, dir, frontier_lanes, pend_count, spill_cur, mode, scan_rows;
};

struct Smem {
    uint32_t lane[kMaxLanes + 1];   // expand: sample index per lane; sweep, schedule: entry prefixes
    uint32_t act[2 * kMaxWords];    // commit: lanes seen in this CTA's new units (32-bit halves)
    CommitWarp cw[kThreads / 32];   // commit
    uint64_t fin[kMaxWords];        // sweep: finished lanes (spill-log sweep)
    // schedule: the control fields it reads (loaded in parallel), lane masks
    // per word, block-scan scratch
    SchedHead h;
    unsigned long long still[kMaxWords], sfin[kMaxWords], init[kMaxWords];
    unsigned long long mscan[33][6];  // schedule: block-scan scratch (32 warps + totals)
    float rawf[8], feat[8], h1[kPolicyHidden], h2[kPolicyHidden], out[kPolicyOut];
    float pol[2 * kPolicyIn + kPolicyParams];  // schedule: the network's parameters
    uint32_t last, abort, nstill, dir, mode;
    uint32_t pcnt[kThreads / 32], pbuf[kThreads / 32 * kPendBuf];  // expand: per-warp pending buffers
};

// dst[0 .. count) = src[0 .. count) (count <= kMaxLanes + 1), all loads of a
// thread issued before any store so that they are in flight together.
// ro: src does not change while the kernel runs (read through L1, so that the
// CTAs of an SM share one fetch).
template <bool ro = false>
__device__ __forceinline__ void fill_smem(uint32_t* dst, const uint32_t* src, uint32_t count) {
    constexpr uint32_t kPer = (kMaxLanes + 1 + kThreads - 1) / kThreads;
    uint32_t v[kPer];
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        const uint32_t i = threadIdx.x + k * kThreads;
        v[k] = i < count ? LD<ro>(&src[i]) : 0u;
    }
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        const uint32_t i = threadIdx.x + k * kThreads;
        if (i < count) dst[i] = v[k];
    }
}

__device__ __forceinline__ void phase_begin(Ctl* ctl, int p) {
    if (threadIdx.x == 0) atomicMin(&ctl->ph_t0[p], globaltimer_ns());
}
__device__ __forceinline__ void phase_end(Ctl* ctl, int p) {
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&ctl->ph_t1[p], globaltimer_ns());
}

// w becomes pending (once per level) when the first word of next[w] turns non-zero.
__device__ __forceinline__ void or_next(const Eng& E, uint32_t w, uint32_t i, uint64_t y) {
    const unsigned long long old =
        atomicOr((unsigned long long*)&E.next[(uint64_t)w * E.WB + i], (unsigned long long)y);
    if (old != 0) return;
    const unsigned long long o2 = atomicOr((unsigned long long*)&E.nocc[w], 1ull << i);
    if (o2 != 0) return;
    const uint32_t p = atomicAdd(&E.ctl->pend_count, 1u);
    if (p < E.pend_cap)
        E.pend_v[p] = w;
    else
        atomicOr(&E.ctl->error, (unsigned)kErrPendOverflow);
}

// ---- sweep: RR rows of finished lanes (Listing 1's RRR-set construction) -------------------

// Every entry of a finished lane (its segment, plus the spill log when the
// segment overflowed) is one vertex of its sample's RR set.  The scheduler gave
// the lane a staging range of the row's length; entry p of the lane's list
// goes to position p of that range (vertices in discovery order; the final
// CSR pass sorts each row).  The lane's bit is cleared from visited[] so that
// the lane can carry its next sample.
// The finished lanes' bits of one word of visited[v] are cleared and counted
// once per (vertex, word), by the entry of the lowest finished lane the word
// still holds: when many lanes that share a word end together (their RR sets
// overlapping in a giant component), one atomic per word replaces one per lane.
// Only that entry writes the word during the sweep, so every other entry of
// the word reads either all of the finished bits (and is not the lowest) or
// none of them.
// v is the vertex's label in the sampler's order, vo its caller id (the same
// without a vertex order).
__device__ __forceinline__ void sweep_entry(const Eng& E, const uint64_t* fin, uint32_t l, uint32_t v, uint32_t vo) {
    const uint32_t w = l >> 6;
    unsigned long long* p = (unsigned long long*)&E.visited[(uint64_t)v * E.WB + w];
    const uint64_t m = L2(p) & fin[w];
    if (m == 0 || (uint32_t)(__ffsll((long long)m) - 1) != (l & 63u)) return;
    atomicAnd(p, ~(unsigned long long)m);
    atomicAdd(&E.vcount[vo], (uint32_t)__popcll(m));
}

// pre: shared memory for the finished lanes' entry prefixes (kMaxLanes + 1);
// fin: shared memory for the finished-lane masks (kMaxWords).
template <bool ro>
__device__ void dev_sweep(const Eng& E, uint32_t* pre, uint64_t* fin) {
    Ctl* ctl = E.ctl;
    const uint32_t F = LD<ro>(&ctl->fin_count);
    const uint32_t spill = LD<ro>(&ctl->spill_sweep);
    // a CTA whose first index lies beyond both entry ranges has nothing to do
    const uint64_t work = LD<ro>(&ctl->sweep_work);
    if (F == 0 && !spill) return;
    if ((uint64_t)blockIdx.x * blockDim.x >= work) return;
    phase_begin(ctl, 2);
    __syncthreads();
    fill_smem<ro>(pre, ctl->fin_pre, F + 1);
    for (uint32_t i = threadIdx.x; i < E.WB; i += blockDim.x) fin[i] = LD<ro>(&ctl->fin_mask[i]);
    __syncthreads();
    const uint32_t total = pre[F];
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t cap = LD<ro>(&ctl->pair_cap);
    for (uint64_t base = wid * 32; base < total; base += nwarp * 32) {
        const uint32_t idx = (uint32_t)(base + lane);
        if (idx < total) {
            uint32_t lo = 0, hi = F;  // largest k < F with prefix[k] <= idx
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (pre[mid] <= idx) lo = mid; else hi = mid;
            }
            const uint32_t l = LD<ro>(&ctl->fin_lane[lo]);
            const uint32_t p = idx - pre[lo];
            const uint32_t v = L2(&E.seg[(uint64_t)l * E.seg_cap + p]);
            const uint64_t dst = LD<ro>(&ctl->lane_base[l]) + p;
            const uint32_t vo = E.inv ? __ldg(&E.inv[v]) : v;
            if (dst < cap) E.rows_v[dst] = vo;
            sweep_entry(E, fin, l, v, vo);
        }
    }
    if (spill) {
        const uint32_t dst = LD<ro>(&ctl->spill_cur), src = dst ^ 1u;
        const uint64_t len = min((uint64_t)LD<ro>(&ctl->spill_len[src]), E.spill_cap);
        for (uint64_t base = wid * 32; base < len; base += nwarp * 32) {
            const uint64_t idx = base + lane;
            const bool ok = idx < len;
            uint32_t l = 0, v = 0;
            uint64_t p = 0;
            bool done = false;
            uint64_t ent = 0;
            if (ok) {
                ent = L2(&E.spill[(uint64_t)src * E.spill_cap + idx]);
                l = (uint32_t)(ent >> (2 * kSpillPosBits));
                p = (ent >> kSpillPosBits) & kSpillMask;
                v = (uint32_t)(ent & kSpillMask);
                done = (fin[l >> 6] >> (l & 63)) & 1ull;
            }
            const uint64_t kp = warp_alloc<unsigned long long>(&ctl->spill_len[dst], (ok && !done) ? 1ull : 0ull);
            if (ok && done) {
                const uint64_t d = LD<ro>(&ctl->lane_base[l]) + p;
                const uint32_t vo = E.inv ? __ldg(&E.inv[v]) : v;
                if (d < cap) E.rows_v[d] = vo;
                sweep_entry(E, fin, l, v, vo);
            } else if (ok) {
                if (kp < E.spill_cap) E.spill[(uint64_t)dst * E.spill_cap + kp] = ent;
                else atomicOr(&ctl->error, (unsigned)kErrSpillOverflow);
            }
        }
    }
    phase_end(ctl, 2);
}

// ---- init: start vertices of lanes given a new sample (Listing 1's frontier initialization) ------
// Runs over all CTAs of the level's first kernel (the persistent kernel, or the
// per-level expand) from the lanes the last schedule marked in init_w.

__device__ void dev_init(const Eng& E) {
    Ctl* ctl = E.ctl;
    const uint64_t lanes = 64ull * E.WB;
    for (uint64_t l = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; l < lanes;
         l += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(l >> 6), c = (uint32_t)(l & 63);
        if (!((L2(&ctl->init_w[i]) >> c) & 1ull)) continue;
        const uint32_t j = L2(&ctl->lane_j[l]);
        const uint32_t v = start_vertex(E.seed, E.first_id + j, E.n);
        E.starts[j] = v;
        or_next(E, E.perm ? __ldg(&E.perm[v]) : v, i, 1ull << c);
    }
}

// ---- expand (push over in-edges) -----------------------------------------------------
//
// Liveness test of a 4-edge group: edge k is live for a colour iff
// draw_k < T_k or bit k of `sure` is set.  T_k is the edge's threshold when
// the edge lies in the unit's in-row and 0 < thr < 2^32 - 1, 0 for an edge
// outside the row or with thr = 0 (never live); an always-live edge
// (thr = 0xFFFFFFFF) keeps T = 0xFFFFFFFF and sets its `sure` bit, since a
// draw of 0xFFFFFFFF would fail the strict test.

// New pending vertices of a warp are collected in its shared-memory buffer and
// appended to the global list with one atomic per chunk (pend_flush); a vertex
// that finds the buffer full goes to the list directly.
__device__ __forceinline__ void pend_push(const Eng& E, uint32_t* cnt, uint32_t* buf, uint32_t w) {
    const uint32_t p = atomicAdd(cnt, 1u);
    if (p < kPendBuf) {
        buf[p] = w;
        return;
    }
    const uint32_t g = atomicAdd(&E.ctl->pend_count, 1u);
    if (g < E.pend_cap)
        E.pend_v[g] = w;
    else
        atomicOr(&E.ctl->error, (unsigned)kErrPendOverflow);
}

// All 32 lanes call, converged.
__device__ __forceinline__ void pend_flush(const Eng& E, uint32_t* cnt, uint32_t* buf) {
    __syncwarp();
    const uint32_t n = min(*cnt, kPendBuf);
    if (n == 0) return;
    const uint32_t lane = lane_id();
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&E.ctl->pend_count, n);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (lane < n) {
        if (base + lane < E.pend_cap)
            E.pend_v[base + lane] = buf[lane];
        else
            atomicOr(&E.ctl->error, (unsigned)kErrPendOverflow);
    }
    __syncwarp();
    if (lane == 0) *cnt = 0;
    __syncwarp();
}

// Colours y of word i reach w: next[w][i] |= y and bit i of nocc[w] is set,
// both as reductions that return nothing.  Queue compaction: the nocc update
// returns the old mask instead, and w becomes pending (once per level) when it
// was zero, i.e. on the level's first live edge into w.  Scan compaction: the
// commit finds w by its non-zero nocc mask.
__device__ __forceinline__ void push_live(const Eng& E, uint32_t w, uint32_t i, uint64_t y, bool scan, uint32_t* cnt,
                                          uint32_t* buf) {
    atomicOr((unsigned long long*)&E.next[(uint64_t)w * E.WB + i], (unsigned long long)y);
    if (scan) {
        atomicOr((unsigned long long*)&E.nocc[w], 1ull << i);
        return;
    }
    if (atomicOr((unsigned long long*)&E.nocc[w], 1ull << i) != 0) return;
    pend_push(E, cnt, buf, w);
}

// T and sure of a group whose in-row edges are vm (bits 0..3) and thresholds t.
__device__ __forceinline__ uint32_t group_thresholds(uint32_t vm, const uint4& t, uint4& T) {
    const bool in0 = vm & 1u, in1 = vm & 2u, in2 = vm & 4u, in3 = vm & 8u;
    T = make_uint4(in0 ? t.x : 0u, in1 ? t.y : 0u, in2 ? t.z : 0u, in3 ? t.w : 0u);
    return (in0 && t.x == 0xFFFFFFFFu ? 1u : 0u) | (in1 && t.y == 0xFFFFFFFFu ? 2u : 0u) |
           (in2 && t.z == 0xFFFFFFFFu ? 4u : 0u) | (in3 && t.w == 0xFFFFFFFFu ? 8u : 0u);
}

// Edges of the group that need a draw (in the row, 0 < thr < 2^32 - 1).
__device__ __forceinline__ uint32_t draw_edges(const uint4& T, uint32_t sure) {
    return ((T.x ? 1u : 0u) | (T.y ? 2u : 0u) | (T.z ? 4u : 0u) | (T.w ? 8u : 0u)) & ~sure;
}

// The draws of one group for the colours x (bits of word i, lane ids
// 64i + bit): one Philox call per colour decides the four edges (Listing 1's
// per-colour liveness draw); the live colours of each edge are gathered per
// half-word and ORed into the source's next row (Listing 1's fusing update).
// Filtered: vis_k are the sources' visited words; a colour a source already
// has is not sent to it (and needs no draw if every source has it).
template <bool filtered>
__device__ __forceinline__ void group_draws(const Eng& E, const uint32_t* lj, uint64_t x, uint32_t i, uint64_t q,
                                            const uint4& c4, const uint4& T, uint32_t sure, const PhiloxKeys& K,
                                            const uint64_t (&vis)[4], bool scan, uint32_t* cnt, uint32_t* buf) {
    const uint32_t f_lo = (uint32_t)E.first_id, f_hi = (uint32_t)(E.first_id >> 32);
    const uint32_t qlo = (uint32_t)q, qhi = (uint32_t)(q >> 32);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t xx = (uint32_t)(x >> (32 * h));
        uint32_t z0 = 0, z1 = 0, z2 = 0, z3 = 0;
        const uint32_t* l = lj + 32 * h;
        while (xx) {
            const uint32_t c = __ffs(xx) - 1;
            xx &= xx - 1;
            const uint32_t j = l[c];
            const uint32_t slo = f_lo + j;
            const uint32_t shi = f_hi + (slo < j ? 1u : 0u);
            const uint4 r = philox4x32_10(make_uint4(slo, shi, qlo, qhi), K);
            if ((r.x < T.x) | (r.y < T.y) | (r.z < T.z) | (r.w < T.w) | (sure != 0u)) {
                const uint32_t bit = 1u << c;
                if ((r.x < T.x) || (sure & 1u)) z0 |= bit;
                if ((r.y < T.y) || (sure & 2u)) z1 |= bit;
                if ((r.z < T.z) || (sure & 4u)) z2 |= bit;
                if ((r.w < T.w) || (sure & 8u)) z3 |= bit;
            }
        }
        if (filtered) {
            z0 &= ~(uint32_t)(vis[0] >> (32 * h));
            z1 &= ~(uint32_t)(vis[1] >> (32 * h));
            z2 &= ~(uint32_t)(vis[2] >> (32 * h));
            z3 &= ~(uint32_t)(vis[3] >> (32 * h));
        }
        if (z0 | z1 | z2 | z3) {
            if (z0) push_live(E, c4.x, i, (uint64_t)z0 << (32 * h), scan, cnt, buf);
            if (z1) push_live(E, c4.y, i, (uint64_t)z1 << (32 * h), scan, cnt, buf);
            if (z2) push_live(E, c4.z, i, (uint64_t)z2 << (32 * h), scan, cnt, buf);
            if (z3) push_live(E, c4.w, i, (uint64_t)z3 << (32 * h), scan, cnt, buf);
        }
    }
}

// The set bits of x after dropping its lowest `skip` set bits, at most `take`
// of them (the lowest).
__device__ __forceinline__ uint64_t colour_slice(uint64_t x, uint32_t skip, uint32_t take) {
    for (uint32_t k = 0; k < skip; ++k) x &= x - 1;
    uint64_t rest = x;
    for (uint32_t k = 0; k < take && rest; ++k) rest &= rest - 1;
    return x & ~rest;
}

// Visited words (word i) of the four sources of group q, for filtered push;
// ~0 for edges outside the row, so that they never veto a draw.
__device__ __forceinline__ void source_visited(const Eng& E, uint64_t q, uint32_t vm, uint32_t i, uint64_t (&vis)[4]) {
    const uint4 c4 = __ldg(reinterpret_cast<const uint4*>(E.col) + q);
    vis[0] = (vm & 1u) ? L2(&E.visited[(uint64_t)c4.x * E.WB + i]) : ~0ull;
    vis[1] = (vm & 2u) ? L2(&E.visited[(uint64_t)c4.y * E.WB + i]) : ~0ull;
    vis[2] = (vm & 4u) ? L2(&E.visited[(uint64_t)c4.z * E.WB + i]) : ~0ull;
    vis[3] = (vm & 8u) ? L2(&E.visited[(uint64_t)c4.w * E.WB + i]) : ~0ull;
}

// The draws of two groups (q and q + 32: one lane's pair in a wide chunk) for
// the colours x of word i: two independent Philox chains per colour, sharing
// the colour's sample id; live colours gathered per half-word and edge.
__device__ __forceinline__ void pair_draws(const Eng& E, const uint32_t* lj, uint64_t x, uint32_t i, uint64_t q,
                                           const uint4& ca, const uint4& Ta, uint32_t sa, const uint4& cb,
                                           const uint4& Tb, uint32_t sb, const PhiloxKeys& K, bool scan,
                                           uint32_t* cnt, uint32_t* buf) {
    const uint32_t f_lo = (uint32_t)E.first_id, f_hi = (uint32_t)(E.first_id >> 32);
    const uint64_t qb = q + kChunk;
    const uint32_t qalo = (uint32_t)q, qahi = (uint32_t)(q >> 32), qblo = (uint32_t)qb, qbhi = (uint32_t)(qb >> 32);
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        uint32_t xx = (uint32_t)(x >> (32 * h));
        uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
        const uint32_t* l = lj + 32 * h;
        while (xx) {
            const uint32_t c = __ffs(xx) - 1;
            xx &= xx - 1;
            const uint32_t j = l[c];
            const uint32_t slo = f_lo + j;
            const uint32_t shi = f_hi + (slo < j ? 1u : 0u);
            const uint4 r = philox4x32_10(make_uint4(slo, shi, qalo, qahi), K);
            const uint4 t = philox4x32_10(make_uint4(slo, shi, qblo, qbhi), K);
            const uint32_t bit = 1u << c;
            if ((r.x < Ta.x) | (r.y < Ta.y) | (r.z < Ta.z) | (r.w < Ta.w) | (sa != 0u)) {
                if ((r.x < Ta.x) || (sa & 1u)) a0 |= bit;
                if ((r.y < Ta.y) || (sa & 2u)) a1 |= bit;
                if ((r.z < Ta.z) || (sa & 4u)) a2 |= bit;
                if ((r.w < Ta.w) || (sa & 8u)) a3 |= bit;
            }
            if ((t.x < Tb.x) | (t.y < Tb.y) | (t.z < Tb.z) | (t.w < Tb.w) | (sb != 0u)) {
                if ((t.x < Tb.x) || (sb & 1u)) b0 |= bit;
                if ((t.y < Tb.y) || (sb & 2u)) b1 |= bit;
                if ((t.z < Tb.z) || (sb & 4u)) b2 |= bit;
                if ((t.w < Tb.w) || (sb & 8u)) b3 |= bit;
            }
        }
        if (a0 | a1 | a2 | a3) {
            if (a0) push_live(E, ca.x, i, (uint64_t)a0 << (32 * h), scan, cnt, buf);
            if (a1) push_live(E, ca.y, i, (uint64_t)a1 << (32 * h), scan, cnt, buf);
            if (a2) push_live(E, ca.z, i, (uint64_t)a2 << (32 * h), scan, cnt, buf);
            if (a3) push_live(E, ca.w, i, (uint64_t)a3 << (32 * h), scan, cnt, buf);
        }
        if (b0 | b1 | b2 | b3) {
            if (b0) push_live(E, cb.x, i, (uint64_t)b0 << (32 * h), scan, cnt, buf);
            if (b1) push_live(E, cb.y, i, (uint64_t)b1 << (32 * h), scan, cnt, buf);
            if (b2) push_live(E, cb.z, i, (uint64_t)b2 << (32 * h), scan, cnt, buf);
            if (b3) push_live(E, cb.w, i, (uint64_t)b3 << (32 * h), scan, cnt, buf);
        }
    }
}

// Asynchronous 16-byte global -> shared copies (no register holds the data).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Where chunk c of wide unit (ra, rb) puts this lane: its two groups q and
// q + 32 with their in-row edge masks, and the chunk's colour block.
struct WidePos {
    uint64_t q;
    uint32_t vma, vmb, cb;
};
__device__ __forceinline__ WidePos wide_pos(uint32_t c, const uint4& ra, const uint4& rb, uint32_t lane) {
    WidePos p;
    const uint32_t r = c - rb.y, ngb = (rb.x + kWideSpan - 1) / kWideSpan;
    uint32_t gb = r;
    p.cb = 0;
    if (r >= ngb) {
        p.cb = r / ngb;
        gb = r - p.cb * ngb;
    }
    const uint32_t gl = kWideSpan * gb + lane;
    p.q = (((uint64_t)ra.y << 32) | ra.x) + gl;
    p.vma = gl < rb.x ? 0xFu : 0u;
    p.vmb = gl + kChunk < rb.x ? 0xFu : 0u;
    if (gl == 0) p.vma &= rb.w & 0xFu;
    if (gl + 1 == rb.x) p.vma &= (rb.w >> 4) & 0xFu;
    if (gl + kChunk + 1 == rb.x) p.vmb &= (rb.w >> 4) & 0xFu;
    return p;
}

// Wide units: a chunk is kWideSpan consecutive groups of ONE unit (lane l
// takes groups l and l + 32 of it), times a block of at most kColourBlock of
// the unit's colours, so the unit record, its colour words and each draw's
// colour are warp-uniform.  A warp's first grab is static (warp index), later
// ones come from the level's counter.  While a chunk draws, the threshold and
// source vectors of the next chunk of the grab, when it belongs to the same
// unit, travel into one of the warp's two shared-memory slots (stage: 2 x 32
// lanes x 4 vectors; the slot a chunk reads is never the one being filled).
template <bool filtered, bool ro>
__device__ __forceinline__ void expand_wide(const Eng& E, const uint32_t* lane_j, const PhiloxKeys& K, uint64_t NC,
                                            bool scan, uint32_t* cnt, uint32_t* buf, uint4* stage,
                                            uint64_t& n_edges, uint64_t& n_calls) {
    Ctl* ctl = E.ctl;
    const uint32_t lane = lane_id();
    const uint4* thr4 = reinterpret_cast<const uint4*>(E.thr);
    const uint4* col4 = reinterpret_cast<const uint4*>(E.col);
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t sl = 0;  // slot holding the current chunk's vectors (when pre)
    for (uint32_t grab = 0;; ++grab) {
        uint32_t c0 = 0;
        if (grab == 0) {
            c0 = wid * kChunksPerGrab;
        } else {
            if (lane == 0) c0 = nwarps * kChunksPerGrab + atomicAdd(&ctl->wchunk_next, kChunksPerGrab);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
        }
        if (c0 >= NC) break;
        const uint32_t c1 = (uint32_t)min((uint64_t)c0 + kChunksPerGrab, NC);
        uint32_t u = 0xFFFFFFFFu;
        uint4 ra = make_uint4(0u, 0u, 0u, 0u), rb = ra;
        bool pre = false;  // this chunk's vectors are in the slot
        for (uint32_t c = c0; c < c1; ++c) {
            // the level's chunks are taken from the last allocated down: the
            // commit warps that allocate last are those with the most items,
            // i.e. the units reached by the most colours, whose chunks are the
            // longest; started first, they no longer make the level's tail
            const uint32_t cr = (uint32_t)(NC - 1) - c;
            const uint32_t uc = LD<ro>(&E.wide_chunk[cr]);
            if (uc != u) {
                u = uc;
                ra = LD<ro>(&E.wide_rec[2ull * u]);
                rb = LD<ro>(&E.wide_rec[2ull * u + 1]);
            }
            const WidePos P = wide_pos(cr, ra, rb, lane);
            uint4 ta = make_uint4(0u, 0u, 0u, 0u), tb = ta, ca = ta, cbv = ta;
            if (pre) {
                cp_async_wait_all();
                const uint4* slot = stage + (sl * 32 + lane) * 4;
                if (P.vma) {
                    ta = slot[0];
                    ca = slot[1];
                }
                if (P.vmb) {
                    tb = slot[2];
                    cbv = slot[3];
                }
            } else {
                if (P.vma) {
                    ta = __ldg(thr4 + P.q);
                    ca = __ldg(col4 + P.q);
                }
                if (P.vmb) {
                    tb = __ldg(thr4 + P.q + kChunk);
                    cbv = __ldg(col4 + P.q + kChunk);
                }
            }
            // the next chunk of the grab, if it continues this unit: its vectors
            // head for the slot while this chunk draws
            pre = false;
            if (c + 1 < c1 && LD<ro>(&E.wide_chunk[cr - 1]) == u) {
                sl ^= 1u;
                uint4* slot = stage + (sl * 32 + lane) * 4;
                const WidePos Pn = wide_pos(cr - 1, ra, rb, lane);
                if (Pn.vma) {
                    cp_async16(&slot[0], thr4 + Pn.q);
                    cp_async16(&slot[1], col4 + Pn.q);
                }
                if (Pn.vmb) {
                    cp_async16(&slot[2], thr4 + Pn.q + kChunk);
                    cp_async16(&slot[3], col4 + Pn.q + kChunk);
                }
                cp_async_commit();
                pre = true;
            }
            uint4 Ta, Tb;
            const uint32_t sa = group_thresholds(P.vma, ta, Ta), sb = group_thresholds(P.vmb, tb, Tb);
            if (P.cb == 0) n_edges += __popc(P.vma) + __popc(P.vmb);
            const uint32_t need = (draw_edges(Ta, sa) != 0u ? 1u : 0u) + (draw_edges(Tb, sb) != 0u ? 1u : 0u);
            const bool any_a = (Ta.x | Ta.y | Ta.z | Ta.w) != 0u, any_b = (Tb.x | Tb.y | Tb.z | Tb.w) != 0u;
            if (__any_sync(0xffffffffu, any_a || any_b)) {
                uint64_t words = ((uint64_t)ra.w << 32) | ra.z;
                // the unit's colours in (word, bit) order: skip cb blocks, take one
                uint32_t skip = P.cb * kColourBlock, take = kColourBlock;
                while (words && take) {
                    const uint32_t i = __ffsll((long long)words) - 1;
                    words &= words - 1;
                    const uint32_t only = rb.w >> 8;  // unfused: the unit's single colour (lane + 1)
                    uint64_t x = only ? 1ull << ((only - 1u) & 63u) : LD<ro>(&E.stage[(uint64_t)rb.z * E.WB + i]);
                    const uint32_t pc = __popcll(x);
                    if (skip >= pc) {
                        skip -= pc;
                        continue;
                    }
                    if (skip || pc - skip > take) x = colour_slice(x, skip, take);
                    skip = 0;
                    take -= __popcll(x);
                    n_calls += (uint64_t)need * __popcll(x);
                    if (!filtered) {
                        pair_draws(E, lane_j + (i << 6), (any_a || any_b) ? x : 0ull, i, P.q, ca, Ta, sa, cbv, Tb, sb,
                                   K, scan, cnt, buf);
                    } else {
#pragma unroll 1
                        for (int g2 = 0; g2 < 2; ++g2) {
                            const uint32_t vm = g2 ? P.vmb : P.vma;
                            const uint64_t qq = g2 ? P.q + kChunk : P.q;
                            uint64_t vis[4] = {~0ull, ~0ull, ~0ull, ~0ull};
                            if (vm) source_visited(E, qq, vm, i, vis);
                            const uint64_t xs = (g2 ? any_b : any_a) ? x & ~(vis[0] & vis[1] & vis[2] & vis[3]) : 0ull;
                            group_draws<true>(E, lane_j + (i << 6), xs, i, qq, g2 ? cbv : ca, g2 ? Tb : Ta,
                                              g2 ? sb : sa, K, vis, scan, cnt, buf);
                        }
                    }
                }
            }
            pend_flush(E, cnt, buf);
        }
        if (pre) cp_async_wait_all();  // nothing may still be landing in the slot
    }
}

// Narrow units (fewer than kWideMin groups): their groups form one index
// space, 32 consecutive groups per chunk, one group per lane; a lane finds its
// unit among the chunk's (at most 32) units.
struct Grp {
    uint64_t q, occ;
    uint4 c4, T;
    uint32_t mrow, only, sure, vm;
};

template <bool ro>
__device__ __forceinline__ bool grp_load(const Eng& E, uint32_t u, uint64_t j, Grp& G, uint64_t& n_edges) {
    G.occ = LD<ro>(&E.list_occ[u]);
    G.mrow = LD<ro>(&E.list_mrow[u]);
    const uint64_t rs = LD<ro>(&E.list_rs[u]), re = LD<ro>(&E.list_re[u]);
    G.only = E.unfused ? LD<ro>(&E.list_only[u]) : 0u;
    G.q = (rs >> 2) + j;
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(E.thr) + G.q);
    G.c4 = __ldg(reinterpret_cast<const uint4*>(E.col) + G.q);
    const uint32_t first = j == 0 ? (uint32_t)(rs & 3) : 0u;
    const uint32_t last = G.q == ((re - 1) >> 2) ? (uint32_t)((re - 1) & 3) : 3u;
    G.vm = (0xFu << first) & (0xFu >> (3u - last));
    n_edges += __popc(G.vm);
    G.sure = group_thresholds(G.vm, t, G.T);
    return (G.T.x | G.T.y | G.T.z | G.T.w) != 0u;
}

template <bool filtered, bool ro>
__device__ __forceinline__ void grp_run(const Eng& E, const uint32_t* lane_j, const Grp& G, const PhiloxKeys& K,
                                        bool scan, uint32_t* cnt, uint32_t* buf, uint64_t& n_calls) {
    const bool need = draw_edges(G.T, G.sure) != 0u;
    uint64_t words = G.occ;
    while (words) {
        const uint32_t i = __ffsll((long long)words) - 1;
        words &= words - 1;
        uint64_t x = G.only ? (1ull << ((G.only - 1u) & 63u)) : LD<ro>(&E.stage[(uint64_t)G.mrow * E.WB + i]);
        uint64_t vis[4] = {0ull, 0ull, 0ull, 0ull};
        if (filtered) {
            source_visited(E, G.q, G.vm, i, vis);
            x &= ~(vis[0] & vis[1] & vis[2] & vis[3]);
            if (!x) continue;
        }
        if (need) n_calls += __popcll(x);
        group_draws<filtered>(E, lane_j + (i << 6), x, i, G.q, G.c4, G.T, G.sure, K, vis, scan, cnt, buf);
    }
}

// The unit holding group g of chunk c: chunk_u0[c] names the unit holding
// group 32c; the lanes find their own unit among the (at most 32) units of the
// chunk by binary lifting over shuffled group offsets.  All lanes must call.
template <bool ro>
__device__ __forceinline__ uint32_t chunk_unit(const Eng& E, uint32_t c, uint64_t nchunks, uint64_t U, uint64_t g,
                                               uint64_t& j) {
    const uint32_t lane = lane_id();
    const uint32_t u0 = LD<ro>(&E.chunk_u0[c]);
    const uint32_t ul = (c + 1 < nchunks) ? LD<ro>(&E.chunk_u0[c + 1]) : (uint32_t)(U - 1);
    const uint32_t nu = min(ul - u0 + 1u, 32u);
    const uint64_t gb = lane < nu ? LD<ro>(&E.list_g[u0 + lane]) : ~0ull;
    uint32_t k = 0;
#pragma unroll
    for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint64_t gs = __shfl_sync(0xffffffffu, gb, (k + step) & 31u);
        if (k + step < nu && gs <= g) k += step;
    }
    j = g - __shfl_sync(0xffffffffu, gb, k);
    return u0 + k;
}

// Pull (Section 9 (a), direction switching): every vertex w that some
// frontier colour has not reached yet scans its out-edges (w -> v, edge e).  A
// colour of the frontier row of v that w lacks is live by the same draw as in
// push (word e & 3 of Philox(sample, e >> 2)), so the closure is unchanged.  A
// warp owns w and stops once every missing colour has been found; no draw is
// spent on a colour w already has.  Needs WB <= kPullMaxWords.
__device__ __forceinline__ void dev_pull(const Eng& E, const uint32_t* lane_j, const PhiloxKeys& K, uint64_t& n_edges,
                                      uint64_t& n_calls) {
    Ctl* ctl = E.ctl;
    const uint32_t WB = E.WB;
    const uint32_t tick = (uint32_t)L2(&ctl->tick);
    uint64_t still[kPullMaxWords];
#pragma unroll
    for (uint32_t i = 0; i < kPullMaxWords; ++i) still[i] = i < WB ? L2(&ctl->still_w[i]) : 0ull;
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t f_lo = (uint32_t)E.first_id, f_hi = (uint32_t)(E.first_id >> 32);
    for (uint64_t w = wid; w < E.n; w += nwarp) {
        uint64_t cand[kPullMaxWords];
        bool any = false;
#pragma unroll
        for (uint32_t i = 0; i < kPullMaxWords; ++i) {
            cand[i] = still[i] ? (still[i] & ~L2(&E.visited[w * WB + i])) : 0ull;
            any |= cand[i] != 0;
        }
        if (!any) continue;
        const uint64_t a = __ldg(&E.orow[w]), b = __ldg(&E.orow[w + 1]);
        uint64_t acc[kPullMaxWords];
#pragma unroll
        for (uint32_t i = 0; i < kPullMaxWords; ++i) acc[i] = 0;
        for (uint64_t base = a; base < b; base += 32) {
            const uint64_t p = base + lane;
            if (p < b) {
                const uint32_t v = __ldg(&E.odst[p]);
                if (L2(&E.fstamp[v]) == tick) {
                    const uint32_t e = __ldg(&E.oeid[p]);
                    const uint32_t t = __ldg(&E.thr[e]);
                    ++n_edges;
#pragma unroll
                    for (uint32_t i = 0; i < kPullMaxWords; ++i) {
                        if (!cand[i] || !t) continue;
                        uint64_t f = L2(&E.frontd[(uint64_t)v * WB + i]) & cand[i] & ~acc[i];
                        if (t == 0xFFFFFFFFu) {
                            acc[i] |= f;
                            continue;
                        }
                        while (f) {
                            const uint32_t c = __ffsll((long long)f) - 1;
                            f &= f - 1;
                            const uint32_t j = lane_j[(i << 6) + c];
                            const uint32_t slo = f_lo + j;
                            const uint32_t shi = f_hi + (slo < j ? 1u : 0u);
                            const uint4 r = philox4x32_10(make_uint4(slo, shi, e >> 2, 0u), K);
                            ++n_calls;
                            const uint32_t k = e & 3u;
                            const uint32_t draw = k == 0 ? r.x : k == 1 ? r.y : k == 2 ? r.z : r.w;
                            if (draw < t) acc[i] |= 1ull << c;
                        }
                    }
                }
            }
            bool left = false;
#pragma unroll
            for (uint32_t i = 0; i < kPullMaxWords; ++i) {
                acc[i] = warp_or64(acc[i]);
                left |= (cand[i] & ~acc[i]) != 0;
            }
            if (!left) break;
        }
        if (lane == 0) {
#pragma unroll
            for (uint32_t i = 0; i < kPullMaxWords; ++i)
                if (acc[i]) or_next(E, (uint32_t)w, i, acc[i]);
        }
    }
}

// Narrow units: the packed group space, a warp taking kChunksPerGrab chunks of
// 32 consecutive groups per atomic, one group per lane.  One instance per
// push variant, so that the plain push loop carries no register of the
// filtered one.
template <bool filtered, bool ro>
__device__ __forceinline__ void expand_push(const Eng& E, const uint32_t* lane_j, const PhiloxKeys& K, uint64_t G,
                                            uint64_t U, uint64_t nchunks, bool scan, uint32_t* cnt, uint32_t* buf,
                                            uint64_t& n_edges, uint64_t& n_calls) {
    Ctl* ctl = E.ctl;
    const uint32_t lane = lane_id();
    for (;;) {
        uint32_t c0 = 0;
        if (lane == 0) c0 = atomicAdd(&ctl->chunk_next, kChunksPerGrab);
        c0 = __shfl_sync(0xffffffffu, c0, 0);
        if (c0 >= nchunks) break;
        const uint32_t c1 = (uint32_t)min((uint64_t)c0 + kChunksPerGrab, nchunks);
        for (uint32_t c = c0; c < c1; ++c) {
            const uint64_t g = (uint64_t)c * kChunk + lane;
            uint64_t j = 0;
            const uint32_t u = chunk_unit<ro>(E, c, nchunks, U, g, j);
            Grp A;
            if (g < G && grp_load<ro>(E, u, j, A, n_edges))
                grp_run<filtered, ro>(E, lane_j, A, K, scan, cnt, buf, n_calls);
            pend_flush(E, cnt, buf);
        }
    }
}

// LT levels (the live-edge form of the linear-threshold model): every
// frontier colour at vertex v follows v's kept in-edge for its sample, one
// Philox draw per (sample, vertex) against the row's weight prefix (binary
// search for the first edge whose prefix passes the draw); the source gets the
// colour.  Each colour has at most one frontier vertex (its walk), so one
// thread per frontier unit is enough.
template <bool ro>
__device__ __forceinline__ void expand_lt(const Eng& E, const uint32_t* lane_j, const PhiloxKeys& K, uint64_t U,
                                          uint64_t& n_edges, uint64_t& n_calls) {
    const uint32_t f_lo = (uint32_t)E.first_id, f_hi = (uint32_t)(E.first_id >> 32);
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < U;
         u += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t occ = LD<ro>(&E.list_occ[u]);
        const uint32_t mrow = LD<ro>(&E.list_mrow[u]);
        const uint32_t v = LD<ro>(&E.list_v[u]);
        const uint32_t vid = E.inv ? __ldg(&E.inv[v]) : v;  // the draw is keyed by the caller's vertex id
        const uint64_t rs = LD<ro>(&E.list_rs[u]), re = LD<ro>(&E.list_re[u]);
        const uint64_t base = __ldg(&E.wpre[rs]);
        const uint64_t total = __ldg(&E.wpre[re]) - base;
        uint64_t words = occ;
        while (words) {
            const uint32_t i = __ffsll((long long)words) - 1;
            words &= words - 1;
            uint64_t x = LD<ro>(&E.stage[(uint64_t)mrow * E.WB + i]);
            while (x) {
                const uint32_t c = __ffsll((long long)x) - 1;
                x &= x - 1;
                const uint32_t j = lane_j[(i << 6) + c];
                const uint32_t slo = f_lo + j;
                const uint32_t shi = f_hi + (slo < j ? 1u : 0u);
                const uint4 rnd = philox4x32_10(make_uint4(slo, shi, vid, 0x40000000u), K);
                ++n_calls;
                const uint64_t r = rnd.x;
                if (r >= total) continue;  // v keeps no in-edge for this sample
                const uint64_t key = base + r;
                uint64_t lo = rs, hi = re - 1;  // first e with wpre[e + 1] > key
                while (lo < hi) {
                    const uint64_t mid = (lo + hi) >> 1;
                    if (__ldg(&E.wpre[mid + 1]) > key) hi = mid; else lo = mid + 1;
                }
                ++n_edges;
                or_next(E, __ldg(&E.col[lo]), i, 1ull << c);
            }
        }
    }
}

// The expand phase.  part selects which directions this instance runs (the
// per-level kernels split them so that the plain push kernel carries no
// register of the others): kPartPush, kPartAlt (filtered push and pull) or
// kPartAll (the persistent kernel).  cnt / buf: the CTA's per-warp pending
// buffers (one counter and kPendBuf entries per warp).
enum ExpandPart : int { kPartPush = 0, kPartAlt = 1, kPartAll = 2 };

template <int part>
__device__ void dev_expand(const Eng& E, uint32_t* lane_j, uint32_t* pcnt, uint32_t* pbuf, uint4* pstage) {
    Ctl* ctl = E.ctl;
    // the level's control fields do not change during a per-level kernel:
    // read through L1 there, so that an SM's warps share one fetch
    constexpr bool ro = part != kPartAll;
    const uint64_t G = LD<ro>(&ctl->list_groups);
    const uint64_t NW = LD<ro>(&ctl->wide_chunks);
    const uint32_t dir = LD<ro>(&ctl->dir);
    const bool pull = dir == kDirPull && E.frontd;
    if (part == kPartPush && dir != kDirPush) return;
    if (part == kPartAlt && (dir == kDirPush || E.model == FBPT_MODEL_LT)) return;
    if (G == 0 && NW == 0) return;
    const uint64_t U = LD<ro>(&ctl->list_count);
    const uint64_t nchunks = (G + kChunk - 1) / kChunk;
    // overflow already flagged by commit
    if (nchunks > E.chunk_cap || U > E.list_cap || NW > E.wide_chunk_cap || LD<ro>(&ctl->wide_units) > E.list_cap)
        return;
    phase_begin(ctl, 0);
    __syncthreads();
    fill_smem<ro>(lane_j, ctl->lane_j, 64u * E.WB);
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    uint32_t* cnt = pcnt + warp;
    uint32_t* buf = pbuf + warp * kPendBuf;
    uint4* wstage = pstage + warp * 2 * 32 * 4;
    if (lane == 0) *cnt = 0;
    __syncthreads();
#ifdef FBPT_KEYS_COMPUTED
    const PhiloxKeys K = philox_keys(E.seed);
#else
    // round keys read from the kernel parameters, which the draws can take as
    // constant operands instead of holding them in registers
    PhiloxKeys K;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        K.k0[k] = E.key0[k];
        K.k1[k] = E.key1[k];
    }
#endif
    uint64_t n_edges = 0, n_calls = 0;
    const bool scan = LD<ro>(&ctl->mode) == FBPT_COMPACT_SCAN;
    if (E.model == FBPT_MODEL_LT) {
        expand_lt<part != kPartAll>(E, lane_j, K, U, n_edges, n_calls);
    } else if (part != kPartPush && pull) {
        dev_pull(E, lane_j, K, n_edges, n_calls);
    } else if (part != kPartPush && dir == kDirFiltered) {
        expand_wide<true, part != kPartAll>(E, lane_j, K, NW, scan, cnt, buf, wstage, n_edges, n_calls);
        expand_push<true, part != kPartAll>(E, lane_j, K, G, U, nchunks, scan, cnt, buf, n_edges, n_calls);
    } else if (part != kPartAlt) {
        expand_wide<false, part != kPartAll>(E, lane_j, K, NW, scan, cnt, buf, wstage, n_edges, n_calls);
        expand_push<false, part != kPartAll>(E, lane_j, K, G, U, nchunks, scan, cnt, buf, n_edges, n_calls);
    }
    // one reduction per CTA for the statistics (the lane table's shared
    // memory holds the warps' sums once every warp is done with it)
    n_edges = warp_sum(n_edges);
    n_calls = warp_sum(n_calls);
    __syncthreads();
    if (lane == 0) {
        lane_j[2 * warp] = (uint32_t)n_edges;
        lane_j[2 * warp + 1] = (uint32_t)n_calls;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long e = 0, c = 0;
        for (uint32_t k = 0; k < (blockDim.x >> 5); ++k) {
            e += lane_j[2 * k];
            c += lane_j[2 * k + 1];
        }
        if (e) atomicAdd(&ctl->st_edges, e);
        if (c) atomicAdd(&ctl->st_calls, c);
    }
    phase_end(ctl, 0);
}

// ---- commit -------------------------------------------------------------------------

__device__ __forceinline__ void write_unit(const Eng& E, uint64_t pos, uint32_t w, uint32_t mrow, uint64_t occ,
                                           uint32_t only, uint64_t rs, uint64_t re, uint64_t gbeg, uint64_t ng,
                                           bool chunks) {
    E.list_v[pos] = w;
    E.list_mrow[pos] = mrow;
    E.list_occ[pos] = occ;
    E.list_rs[pos] = rs;
    E.list_re[pos] = re;
    E.list_g[pos] = gbeg;
    if (E.unfused) E.list_only[pos] = only;
    if (!chunks) return;
    // chunks whose first group falls inside this unit start their search here
    const uint64_t end = gbeg + ng;
    for (uint64_t c = (gbeg + kChunk - 1) / kChunk; c * kChunk < end; ++c) {
        if (c < E.chunk_cap) E.chunk_u0[c] = (uint32_t)pos;
        else atomicOr(&E.ctl->error, (unsigned)kErrChunkOverflow);
    }
}

// Position of the r-th (0-based) set bit of m.
__device__ __forceinline__ uint32_t nth_bit64(uint64_t m, uint32_t r) {
    const uint32_t lo = (uint32_t)m, pl = __popc(lo);
    return r < pl ? __fns(lo, 0, (int)r + 1) : 32u + __fns((uint32_t)(m >> 32), 0, (int)(r - pl) + 1);
}

// For every pending vertex w and every word i with next[w][i] != 0:
// nx = next[w][i] & ~visited[w][i]; next[w][i] = 0; visited[w][i] |= nx; each
// new colour appends w to its lane's entries.  The (vertex, word) items of a
// warp's 32 vertices are spread over its lanes, so a hub reached by many
// colours at once is not left to one thread.  Non-empty rows become frontier
// units (if w has in-edges).
// ro: the per-level kernel, in which the level's control fields do not change
// (read through L1); the persistent kernel reads them through L2.
template <bool ro>
__device__ void dev_commit(const Eng& E, Smem& sm) {
    Ctl* ctl = E.ctl;
    const bool scan = LD<ro>(&ctl->mode) == FBPT_COMPACT_SCAN;
    const uint32_t P = scan ? 0u : (uint32_t)min((uint64_t)LD<ro>(&ctl->pend_count), E.pend_cap);
    // queue: vertices per warp: spread a small level over more warps of the
    // grid (the work is a chain of dependent loads per vertex), but at least
    // FBPT_COMMIT_VPW_MIN per warp so that each warp's fixed bookkeeping stays
    // amortised; up to one per lane.  A warp takes every nused-th pending
    // vertex (nused: the warps a round needs): the hubs, which many frontier
    // units reach early in the expand and so head the pending list, are spread
    // over the warps instead of lengthening the first warps' item loops.
    // scan: every warp takes 32 consecutive vertices at a time and handles
    // those whose word-occupancy mask is set.
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t vpw =
        (uint32_t)min((uint64_t)32, max((uint64_t)FBPT_COMMIT_VPW_MIN, (P + nwarp - 1) / nwarp));
    if (!scan && (uint64_t)blockIdx.x * (blockDim.x >> 5) * vpw >= P) return;  // no pending vertex for this CTA
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < 2 * E.WB; i += blockDim.x) sm.act[i] = 0;
    __syncthreads();
    if (P || scan) phase_begin(ctl, 1);
    const uint32_t spill_cur = LD<ro>(&ctl->spill_cur);
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    CommitWarp& cw = sm.cw[threadIdx.x >> 5];
    uint64_t mwords = 0, ncol = 0, wgroups = 0;
    // One round: up to 32 reached vertices of this warp, one per lane (ok);
    // w, its stage row idx, its changed words m and in-row [rs, re).
    auto round = [&](bool ok, uint32_t w, uint64_t idx, uint64_t m, uint64_t rs, uint64_t re) {
        const uint32_t ni = __popcll(m);
        const uint32_t incl = warp_incl_scan(ni);
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        cw.m[lane] = m;
        cw.w[lane] = w;
        cw.row[lane] = (uint32_t)idx;
        cw.start[lane] = incl - ni;
        cw.occ_lo[lane] = 0;
        cw.occ_hi[lane] = 0;
        cw.bits[lane] = 0;
        cw.he[lane] = re > rs;
        __syncwarp();
        for (uint32_t t0 = 0; t0 < total; t0 += 32) {
            const uint32_t t = t0 + lane;
            uint64_t nx = 0;
            uint32_t i = 0, wv = 0;
            if (t < total) {
                uint32_t o = 0;  // the vertex owning item t: largest o with start[o] <= t
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1)
                    if (cw.start[o + step] <= t) o += step;
                i = nth_bit64(cw.m[o], t - cw.start[o]);
                wv = cw.w[o];
                const uint64_t rowi = (uint64_t)wv * E.WB + i;
                // both loads go out before the word is cleared, and the clearing
                // store waits for the loaded value (a changed word is never zero):
                // a store queued behind an outstanding load of the same word held
                // up the level's loads and atomics by ~15 us
                const uint64_t nraw = L2(&E.next[rowi]);
                const uint64_t vis = L2(&E.visited[rowi]);
                if (nraw) E.next[rowi] = 0;
                nx = nraw & ~vis;
                if (nx) {
                    E.visited[rowi] = vis | nx;
                    E.stage[(uint64_t)cw.row[o] * E.WB + i] = nx;
                    if (i < 32) atomicOr(&cw.occ_lo[o], 1u << i);
                    else atomicOr(&cw.occ_hi[o], 1u << (i - 32));
                    atomicAdd(&cw.bits[o], (uint32_t)__popcll(nx));
                    if (cw.he[o]) {
                        if ((uint32_t)nx) atomicOr(&sm.act[2 * i], (uint32_t)nx);
                        if (nx >> 32) atomicOr(&sm.act[2 * i + 1], (uint32_t)(nx >> 32));
                    }
                }
            }
            // one entry per (item, new colour) in the lane's RR list; the
            // warp takes them 32 at a time, and equal lanes share one atomic
            const uint32_t nb = __popcll(nx);
            const uint32_t einc = warp_incl_scan(nb);
            const uint32_t etot = __shfl_sync(0xffffffffu, einc, 31);
            cw.ex[lane] = nx;
            cw.el[lane] = i << 6;
            cw.ev[lane] = wv;
            cw.es[lane] = einc - nb;
            __syncwarp();
            for (uint32_t e0 = 0; e0 < etot; e0 += 32) {
                const uint32_t e = e0 + lane;
                const bool ok = e < etot;
                uint32_t l = 0xFFFFFFFFu, v = 0;
                if (ok) {
                    uint32_t q = 0;
#pragma unroll
                    for (uint32_t step = 16; step > 0; step >>= 1)
                        if (cw.es[q + step] <= e) q += step;
                    l = cw.el[q] + nth_bit64(cw.ex[q], e - cw.es[q]);
                    v = cw.ev[q];
                }
                const uint32_t peers = __match_any_sync(0xffffffffu, l);
                const uint32_t leader = __ffs(peers) - 1;
                uint32_t pos = 0;
                if (ok && lane == leader) pos = atomicAdd(&ctl->lane_cnt[l], (uint32_t)__popc(peers));
                pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & lanemask_lt());
                const bool spill = ok && pos >= E.seg_cap;
                if (ok && !spill) E.seg[(uint64_t)l * E.seg_cap + pos] = v;
                if (!__any_sync(0xffffffffu, spill)) continue;
                const uint64_t sp = warp_alloc<unsigned long long>(&ctl->spill_len[spill_cur], spill ? 1ull : 0ull);
                if (spill) {
                    if (sp < E.spill_cap)
                        E.spill[(uint64_t)spill_cur * E.spill_cap + sp] =
                            ((uint64_t)l << (2 * kSpillPosBits)) | ((uint64_t)pos << kSpillPosBits) | v;
                    else
                        atomicOr(&ctl->error, (unsigned)kErrSpillOverflow);
                }
            }
            __syncwarp();
        }
        __syncwarp();
        const uint64_t occ = ((uint64_t)cw.occ_hi[lane] << 32) | cw.occ_lo[lane];
        const uint32_t bits = cw.bits[lane];
        __syncwarp();
        const uint64_t ng = occ ? row_groups(rs, re) : 0;
        const uint64_t units = ng ? (E.unfused ? bits : 1u) : 0u;
        // IC units of at least kWideMin groups are wide (own chunks, a record
        // each; unfused: one per colour); the rest are packed into the narrow
        // group space
        const bool wide = units && E.model == FBPT_MODEL_IC && ng >= kWideMin;
        const uint64_t nun = wide ? 0 : units;
        if (E.frontd && units) {  // frontier row by vertex, for a pull level
            for (uint32_t i = 0; i < E.WB; ++i)
                E.frontd[(uint64_t)w * E.WB + i] = ((occ >> i) & 1ull) ? L2(&E.stage[idx * E.WB + i]) : 0ull;
            E.fstamp[w] = (uint32_t)LD<ro>(&ctl->tick) + 1u;
        }
        mwords += units ? (E.unfused ? units : (uint64_t)__popcll(occ)) : 0;
        ncol += units ? bits : 0;
        // narrow units: (units | groups << 26); wide: a record and chunks of
        // their own per unit (64-group blocks times colour blocks; one colour
        // per unfused unit), (units | chunks << 26).  Both counters are bumped
        // by one lane before either result is awaited.
        const unsigned long long req = (unsigned long long)((nun * ng) << kUnitBits) | nun;
        const uint64_t wun = wide ? units : 0;
        const uint64_t ncb = E.unfused ? 1 : (bits + kColourBlock - 1) / kColourBlock;
        const uint64_t wck = wide ? ((ng + kWideSpan - 1) / kWideSpan) * ncb : 0;
        const unsigned long long wreq = (unsigned long long)((wun * wck) << kUnitBits) | wun;
        unsigned long long got, wgot;
        warp_alloc2<unsigned long long>(&ctl->new_packed, req, got, &ctl->wide_packed, wreq, wgot);
        const uint64_t pos0 = got & kUnitMask;
        const uint64_t gbeg0 = got >> kUnitBits;
        const bool fits = nun && pos0 + nun <= E.list_cap;
        if (nun && !fits) atomicOr(&ctl->error, (unsigned)kErrListOverflow);
        const uint64_t wpos = wgot & kUnitMask, wc0 = wgot >> kUnitBits;
        const bool wfits = wide && wpos + wun <= E.list_cap && wc0 + wun * wck <= E.wide_chunk_cap;
        if (wide && !wfits) {
            if (wpos + wun <= E.list_cap) {
                atomicOr(&ctl->error, (unsigned)kErrWideOverflow);
                atomicMax(&ctl->wide_need, (unsigned long long)(wc0 + wun * wck));
            } else {
                atomicOr(&ctl->error, (unsigned)kErrListOverflow);
            }
        }
        if (wfits) {
            const uint64_t q0 = rs >> 2;
            const uint32_t masks = ((0xFu << (uint32_t)(rs & 3)) & 0xFu) | ((0xFu >> (3u - (uint32_t)((re - 1) & 3))) << 4);
            if (!E.unfused) {
                E.wide_rec[2 * wpos] = make_uint4((uint32_t)q0, (uint32_t)(q0 >> 32), (uint32_t)occ, (uint32_t)(occ >> 32));
                E.wide_rec[2 * wpos + 1] = make_uint4((uint32_t)ng, (uint32_t)wc0, (uint32_t)idx, masks);
            } else {  // one unit per colour; bits 8.. of the masks hold its lane + 1
                uint64_t k = 0, ws = occ;
                while (ws) {
                    const uint32_t i = __ffsll((long long)ws) - 1;
                    ws &= ws - 1;
                    uint64_t x = E.stage[idx * E.WB + i];
                    while (x) {
                        const uint32_t c = __ffsll((long long)x) - 1;
                        x &= x - 1;
                        const uint64_t u = wpos + k;
                        E.wide_rec[2 * u] = make_uint4((uint32_t)q0, (uint32_t)(q0 >> 32), i < 32 ? 1u << i : 0u,
                                                       i < 32 ? 0u : 1u << (i - 32));
                        E.wide_rec[2 * u + 1] = make_uint4((uint32_t)ng, (uint32_t)(wc0 + k * wck), (uint32_t)idx,
                                                           masks | ((i * 64u + c + 1u) << 8));
                        ++k;
                    }
                }
            }
        }
        wgroups += wide ? wun * ng : 0;
        if (fits && !E.unfused) {
            write_unit(E, pos0, w, (uint32_t)idx, occ, 0u, rs, re, gbeg0, ng, false);
        } else if (fits) {
            uint64_t pos = pos0, gbeg = gbeg0;
            uint64_t ws = occ;
            while (ws) {
                const uint32_t i = __ffsll((long long)ws) - 1;
                ws &= ws - 1;
                uint64_t x = E.stage[idx * E.WB + i];
                while (x) {
                    const uint32_t c = __ffsll((long long)x) - 1;
                    x &= x - 1;
                    write_unit(E, pos++, w, (uint32_t)idx, 1ull << i, i * 64u + c + 1u, rs, re, gbeg, ng, true);
                    gbeg += ng;
                }
            }
        }
        // chunk map of the fused units: every chunk whose first group lies in a
        // unit points at it; the writes of the warp's units are spread over its lanes
        uint32_t c0 = 0, nck = 0;
        if (fits && !E.unfused) {
            c0 = (uint32_t)((gbeg0 + kChunk - 1) / kChunk);
            nck = (uint32_t)((gbeg0 + ng + kChunk - 1) / kChunk) - c0;
        }
        // wide chunk map first: chunk wc0 + r -> unit wpos + r / wck
        {
            const uint32_t wn = wfits ? (uint32_t)(wun * wck) : 0u;
            const uint32_t wincl = warp_incl_scan(wn);
            const uint32_t wtot = __shfl_sync(0xffffffffu, wincl, 31);
            cw.start[lane] = wincl - wn;
            cw.w[lane] = (uint32_t)wpos;
            cw.occ_lo[lane] = (uint32_t)wc0;
            cw.bits[lane] = (uint32_t)wck;
            __syncwarp();
            for (uint32_t t = lane; t < wtot; t += 32) {
                uint32_t o = 0;
#pragma unroll
                for (uint32_t step = 16; step > 0; step >>= 1)
                    if (cw.start[o + step] <= t) o += step;
                const uint32_t r = t - cw.start[o];
                E.wide_chunk[(uint64_t)cw.occ_lo[o] + r] = cw.w[o] + r / cw.bits[o];
            }
            __syncwarp();
        }
        const uint32_t cincl = warp_incl_scan(nck);
        const uint32_t ctot = __shfl_sync(0xffffffffu, cincl, 31);
        cw.start[lane] = cincl - nck;
        cw.w[lane] = (uint32_t)pos0;
        cw.occ_lo[lane] = c0;
        __syncwarp();
        for (uint32_t t = lane; t < ctot; t += 32) {
            uint32_t o = 0;
#pragma unroll
            for (uint32_t step = 16; step > 0; step >>= 1)
                if (cw.start[o + step] <= t) o += step;
            const uint64_t c = (uint64_t)cw.occ_lo[o] + (t - cw.start[o]);
            if (c < E.chunk_cap) E.chunk_u0[c] = cw.w[o];
            else atomicOr(&ctl->error, (unsigned)kErrChunkOverflow);
        }
        __syncwarp();
    };
    if (!scan) {
        for (uint64_t r0 = 0; r0 < P; r0 += nwarp * vpw) {
            const uint64_t C = min((uint64_t)P - r0, nwarp * vpw);  // vertices of this round
            const uint64_t nused = (C + vpw - 1) / vpw;
            if (wid >= nused) break;  // only the last round leaves warps out
            const uint64_t idx = r0 + wid + (uint64_t)lane * nused;
            const bool ok = lane < vpw && idx < r0 + C;
            uint32_t w = 0;
            uint64_t m = 0, rs = 0, re = 0;
            if (ok) {
                w = L2(&E.pend_v[idx]);
                m = L2(&E.nocc[w]);
                if (m) E.nocc[w] = 0;  // after the load has returned (a pending vertex's mask is non-zero)
                rs = __ldg(&E.rstart[w]);
                re = __ldg(&E.rend[w]);
            }
            round(ok, w, idx, m, rs, re);
        }
    } else {
        // the next warp-sized block's masks are loaded before this one is handled
        uint64_t base = wid * 32;
        uint64_t m = base + lane < E.n ? L2(&E.nocc[base + lane]) : 0ull;
        for (; base < E.n; base += nwarp * 32) {
            const uint64_t v = base + lane, nb = base + nwarp * 32;
            const uint64_t mnext = nb + lane < E.n ? L2(&E.nocc[nb + lane]) : 0ull;
            bool ok = m != 0;
            if (__any_sync(0xffffffffu, ok)) {
                if (ok) E.nocc[v] = 0;
                uint64_t idx = warp_alloc<unsigned int>(&ctl->scan_rows, ok ? 1u : 0u);
                if (ok && idx >= E.pend_cap) {
                    atomicOr(&ctl->error, (unsigned)kErrPendOverflow);
                    ok = false;
                }
                uint64_t rs = 0, re = 0;
                if (ok) {
                    rs = __ldg(&E.rstart[v]);
                    re = __ldg(&E.rend[v]);
                }
                round(ok, (uint32_t)v, idx, ok ? m : 0ull, rs, re);
            }
            m = mnext;
        }
    }
    // one reduction per CTA for the statistics and colour / group totals
    mwords = warp_sum(mwords);
    ncol = warp_sum(ncol);
    wgroups = warp_sum(wgroups);
    if (lane == 0) {
        sm.mscan[threadIdx.x >> 5][0] = mwords;
        sm.mscan[threadIdx.x >> 5][1] = ncol;
        sm.mscan[threadIdx.x >> 5][2] = wgroups;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0, c = 0;
        for (uint32_t k = 0; k < (blockDim.x >> 5); ++k) {
            a += sm.mscan[k][0];
            b += sm.mscan[k][1];
            c += sm.mscan[k][2];
        }
        if (a) atomicAdd(&ctl->st_mask_words, a);
        if (b) atomicAdd(&ctl->new_colours, b);
        if (c) atomicAdd(&ctl->wide_gnew, c);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < E.WB; i += blockDim.x) {
        const unsigned long long a = ((unsigned long long)sm.act[2 * i + 1] << 32) | sm.act[2 * i];
        if (a) atomicOr(&ctl->act_w[i], a);
    }
    if (P || scan) phase_end(ctl, 1);
}

// ---- level direction: degree-ratio heuristic and the policy network ----------------------

// Features of the coming level (also what the trace rows let a trainer rebuild):
// log2 of 1 + units, groups, colours and frontier lanes, the frontier's share of
// the edges (log2 of 4 * groups / m) and log2 of colours per unit.
// Feature k of a level (FP64 arithmetic, rounded to FP32).
__device__ __forceinline__ float level_feature(uint32_t k, double U, double G, double C, double L, double m) {
    switch (k) {
        case 0: return (float)log2(1.0 + U);
        case 1: return (float)log2(1.0 + G);
        case 2: return (float)log2(1.0 + C);
        case 3: return (float)log2(1.0 + L);
        case 4: return (float)(log2(1.0 + 4.0 * G) - log2(1.0 + m));
        default: return (float)log2(1.0 + C / (U > 1.0 ? U : 1.0));
    }
}

// The policy's level actions: outputs 0..4 of the network are the predicted
// log2 time of the level under each.
constexpr uint32_t kActPush = 0, kActFiltered = 1, kActPull = 2, kActPushScan = 3, kActFilteredScan = 4;
constexpr uint32_t kActions = 5;
__device__ __forceinline__ uint32_t action_dir(uint32_t a) {
    return a == kActPull ? kDirPull : (a == kActFiltered || a == kActFilteredScan) ? kDirFiltered : kDirPush;
}
__device__ __forceinline__ uint32_t action_mode(uint32_t a) {
    return a >= kActPushScan ? FBPT_COMPACT_SCAN : FBPT_COMPACT_QUEUE;
}

// Push draws about G * (colours per unit) times; a pull level reads every
// vertex's row and, at most, every edge.  Pull when the push would draw for more
// colour-edges than twice the edge count; filter pushes whose units carry many
// colours (their targets are likelier to have seen them already).
__device__ __forceinline__ uint32_t heuristic_dir(double U, double G, double C, double m, bool pull_ok) {
    const double cbar = C / (U > 1.0 ? U : 1.0);
    if (pull_ok && G * cbar > 2.0 * m) return kDirPull;
    if (cbar >= 8.0) return kDirFiltered;
    return kDirPush;
}

// 6 -> 32 -> 32 -> 8 ReLU network on the features in sm.rawf; outputs 0..2
// are the predicted log2 device time of the level under push, filtered push
// and pull.  P holds the input mean and scale (6 + 6), then W1 (32x6), b1,
// W2 (32x32), b2, W3 (8x32), b3.  All threads of the CTA call it.
__device__ void policy_forward(Smem& sm) {
    const int t = threadIdx.x;
    const float* P = sm.pol;
    const float* mu = P;
    const float* sd = P + kPolicyIn;
    const float* W1 = P + 2 * kPolicyIn;
    const float* b1 = W1 + kPolicyIn * kPolicyHidden;
    const float* W2 = b1 + kPolicyHidden;
    const float* b2 = W2 + kPolicyHidden * kPolicyHidden;
    const float* W3 = b2 + kPolicyHidden;
    const float* b3 = W3 + kPolicyHidden * kPolicyOut;
    if (t < kPolicyIn) sm.feat[t] = (sm.rawf[t] - mu[t]) / sd[t];
    __syncthreads();
    if (t < kPolicyHidden) {
        float h = b1[t];
        for (int k = 0; k < kPolicyIn; ++k) h += W1[t * kPolicyIn + k] * sm.feat[k];
        sm.h1[t] = h > 0.f ? h : 0.f;
    }
    __syncthreads();
    if (t < kPolicyHidden) {
        float h = b2[t];
        for (int k = 0; k < kPolicyHidden; ++k) h += W2[t * kPolicyHidden + k] * sm.h1[k];
        sm.h2[t] = h > 0.f ? h : 0.f;
    }
    __syncthreads();
    if (t < kPolicyOut) {
        float o = b3[t];
        for (int k = 0; k < kPolicyHidden; ++k) o += W3[t * kPolicyHidden + k] * sm.h2[k];
        sm.out[t] = o;
    }
    __syncthreads();
}

// ---- schedule (one CTA) ---------------------------------------------------------------

constexpr uint32_t kSchedThreads = 1024;  // threads of the per-level scheduler CTA
constexpr uint32_t kScanVals = 6;

// Exclusive prefixes of kScanVals values over the CTA's threads in one pass (all
// threads call): v[c] becomes its prefix, tot[c] the sum.  scratch has 33 rows.
__device__ __forceinline__ void block_scan_multi(unsigned long long (&v)[kScanVals],
                                                 unsigned long long (*scratch)[kScanVals],
                                                 unsigned long long (&tot)[kScanVals]) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long incl[kScanVals];
#pragma unroll
    for (uint32_t c = 0; c < kScanVals; ++c) incl[c] = warp_incl_scan(v[c]);
    if (lane == 31) {
#pragma unroll
        for (uint32_t c = 0; c < kScanVals; ++c) scratch[warp][c] = incl[c];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (uint32_t c = 0; c < kScanVals; ++c) {
            const unsigned long long x = lane < nw ? scratch[lane][c] : 0ull;
            const unsigned long long xi = warp_incl_scan(x);
            if (lane < nw) scratch[lane][c] = xi - x;
            if (lane == 31) scratch[32][c] = xi;
        }
    }
    __syncthreads();
#pragma unroll
    for (uint32_t c = 0; c < kScanVals; ++c) {
        tot[c] = scratch[32][c];
        v[c] = scratch[warp][c] + incl[c] - v[c];
    }
    __syncthreads();
}

// Lanes that held a sample but are absent from the new frontier have finished
// (the next sweep emits them).  Free lanes take the next sample ids, right away
// (lane refill) or once no lane is still traversing (batch mode).  The new
// frontier list becomes the expand's input; the loop continues while any
// lane holds a sample.  Every thread owns a run of consecutive lanes (inside
// one word; at most kPer of them), so lane-order prefixes are block scans.
// The start vertices of the lanes given a sample are placed by the next
// level's first kernel (dev_init, from init_w).
template <uint32_t kPer>
__device__ void dev_schedule(const Eng& E, Smem& sm) {
    Ctl* ctl = E.ctl;
    const uint32_t t = threadIdx.x;
    const uint32_t WB = E.WB, L = 64u * WB;
    SchedHead& h = sm.h;
    // 1. everything the step reads, in one round of loads: the control fields,
    // the lane masks of each word and the counts and sample ids of this
    // thread's lanes.  per: the smallest power of two with per * blockDim >= L
    // (per <= kPer by the launch shape), so that a run never straddles two words.
    // (one lane in each of four warps, its loads issued back to back before
    // any is stored: a switch over the lanes of one warp ran its cases one
    // after another, each waiting for its load, ~6 us per level)
    if ((t & 31u) == 0u && (t >> 5) < 4u) {
        switch (t >> 5) {
            case 0: {
                const uint32_t err = L2(&ctl->error), refill = L2(&ctl->refill), sched = L2(&ctl->sched);
                const unsigned long long nj = L2(&ctl->next_j), pc = L2(&ctl->pair_cursor);
                const unsigned long long np = L2(&ctl->new_packed), nc = L2(&ctl->new_colours), tk = L2(&ctl->tick);
                h.err = err; h.refill = refill; h.sched = sched;
                h.next_j = nj; h.pair_cursor = pc; h.new_packed = np; h.new_colours = nc; h.tick = tk;
                break;
            }
            case 1: {
                const unsigned long long lg = L2(&ctl->list_groups), lc = L2(&ctl->list_count);
                const unsigned long long lcol = L2(&ctl->list_colours), tl = L2(&ctl->tick_limit);
                const uint32_t pend = L2(&ctl->pend_count), dir = L2(&ctl->dir), fl = L2(&ctl->frontier_lanes);
                const uint32_t sc = L2(&ctl->spill_cur);
                h.list_groups = lg; h.list_count = lc; h.list_colours = lcol; h.tick_limit = tl;
                h.pend_count = pend; h.dir = dir; h.frontier_lanes = fl; h.spill_cur = sc;
                break;
            }
            case 2: {
                unsigned long long a[3], b[3];
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    a[p] = L2(&ctl->ph_t0[p]);
                    b[p] = L2(&ctl->ph_t1[p]);
                }
                const uint32_t md = L2(&ctl->mode), sr = L2(&ctl->scan_rows);
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    h.ph_t0[p] = a[p];
                    h.ph_t1[p] = b[p];
                }
                h.mode = md; h.scan_rows = sr;
                break;
            }
            default: {
                const unsigned long long wp = L2(&ctl->wide_packed), wg = L2(&ctl->wide_gnew);
                const unsigned long long wu = L2(&ctl->wide_units), wgr = L2(&ctl->wide_groups);
                const unsigned long long s0 = L2(&ctl->spill_len[0]), s1 = L2(&ctl->spill_len[1]);
                h.wide_packed = wp; h.wide_gnew = wg; h.wide_units = wu; h.wide_groups = wgr;
                h.spill_len[0] = s0; h.spill_len[1] = s1;
                break;
            }
        }
    }
    uint32_t per = 1;
    while (per * blockDim.x < L) per <<= 1;
    const uint32_t a0 = min(t * per, L), a1 = min(a0 + per, L);
    const uint32_t wi = a0 >> 6;
    unsigned long long run = 0, act = 0;
    if (a0 < a1) {
        run = L2(&ctl->run_w[wi]);
        act = L2(&ctl->act_w[wi]);
    }
    uint32_t cnt[kPer], jj[kPer];
    if (kPer % 4 == 0 && (per & 3u) == 0) {
        // runs of four lanes: one 16-byte load per array and four lanes
#pragma unroll
        for (uint32_t q = 0; q < kPer / 4; ++q) {
            uint4 c4 = make_uint4(0u, 0u, 0u, 0u), j4 = c4;
            if (4 * q < per && a0 < a1) {
                c4 = __ldcg(reinterpret_cast<const uint4*>(&ctl->lane_cnt[a0 + 4 * q]));
                j4 = __ldcg(reinterpret_cast<const uint4*>(&ctl->lane_j[a0 + 4 * q]));
            }
            cnt[4 * q] = c4.x; cnt[4 * q + 1] = c4.y; cnt[4 * q + 2] = c4.z; cnt[4 * q + 3] = c4.w;
            jj[4 * q] = j4.x; jj[4 * q + 1] = j4.y; jj[4 * q + 2] = j4.z; jj[4 * q + 3] = j4.w;
        }
    } else {
#pragma unroll
        for (uint32_t c = 0; c < kPer; ++c) {
            const bool in = a0 + c < a1;
            cnt[c] = in ? L2(&ctl->lane_cnt[a0 + c]) : 0u;
            jj[c] = in ? L2(&ctl->lane_j[a0 + c]) : 0u;
        }
    }
    // the schedule network's parameters (learned schedule only) into shared
    // memory, loaded together with the fields above (blockDim >= kThreads)
    if (E.policy) {
        constexpr uint32_t kN = 2 * kPolicyIn + kPolicyParams, kPP = (kN + kThreads - 1) / kThreads;
        float pv[kPP];
#pragma unroll
        for (uint32_t k = 0; k < kPP; ++k) {
            const uint32_t i = t + k * blockDim.x;
            pv[k] = i < kN ? __ldg(&E.policy[i]) : 0.f;
        }
#pragma unroll
        for (uint32_t k = 0; k < kPP; ++k) {
            const uint32_t i = t + k * blockDim.x;
            if (i < kN) sm.pol[i] = pv[k];
        }
    }
    if (t < WB) sm.init[t] = 0;
    if (a0 < a1 && (a0 & 63) == 0) {  // the first thread of each word keeps its masks
        sm.still[wi] = run & act;
        sm.sfin[wi] = run & ~act;
    }
    const unsigned long long runmask = a0 < a1 ? ((per >= 64 ? ~0ull : ((1ull << per) - 1ull))) : 0ull;
    const unsigned long long myfin = ((run & ~act) >> (a0 & 63)) & runmask;
    const unsigned long long mystill = ((run & act) >> (a0 & 63)) & runmask;
    const unsigned long long freem = ~mystill & runmask;
    __syncthreads();
    // 2. per thread: finished lanes, their entries, segment entries, spilled
    // lanes; free and traversing lanes.  One scan gives every prefix.
    unsigned long long sv[kScanVals] = {(unsigned long long)__popcll(myfin), 0ull, 0ull,
                                        (unsigned long long)__popcll(freem), (unsigned long long)__popcll(mystill),
                                        0ull};
#pragma unroll
    for (uint32_t c = 0; c < kPer; ++c) {
        if ((myfin >> c) & 1ull) {
            sv[1] += cnt[c];
            sv[2] += min(cnt[c], E.seg_cap);
            sv[5] += cnt[c] > E.seg_cap ? 1u : 0u;
        }
    }
    unsigned long long tot[kScanVals];
    block_scan_multi(sv, sm.mscan, tot);
    const uint32_t F = (uint32_t)tot[0];
    const unsigned long long R64 = tot[1], S64 = tot[2];
    const uint32_t nstill = (uint32_t)tot[4];
    const bool any_spill = tot[5] != 0;
    // 3. each finished lane's row: staging range, sample index, entry of the fin
    // list and its segment-entry prefix (the sweep's input)
    {
        unsigned long long rb = h.pair_cursor + sv[1], seg = sv[2];
        uint32_t k = (uint32_t)sv[0];
#pragma unroll
        for (uint32_t c = 0; c < kPer; ++c) {
            if ((myfin >> c) & 1ull) {
                const uint32_t l = a0 + c, rc = cnt[c], j = jj[c];
                ctl->retired_j[l] = j;
                ctl->lane_base[l] = rb;
                E.row_start[j] = rb;
                E.row_len[j] = rc;
                rb += rc;
                ctl->lane_cnt[l] = 0;
                ctl->fin_lane[k] = l;
                ctl->fin_pre[k] = (uint32_t)seg;
                seg += min(rc, E.seg_cap);
                ++k;
            }
        }
    }
    if (t < WB) ctl->fin_mask[t] = sm.sfin[t];
    // 4. refill: lanes without a sample take the next ids in lane order
    const bool may_refill = h.err == 0 && (h.refill == kRefillLane || nstill == 0);
    const unsigned long long avail = E.S > h.next_j ? E.S - h.next_j : 0ull;
    const unsigned long long N64 = may_refill ? tot[3] : 0ull;
    const unsigned long long assigned = N64 < avail ? N64 : avail;
    if (may_refill) {
        // the sample indices of this thread's refills are loaded together, then
        // stored (a store per load in one loop waited for each load in turn)
        unsigned long long r = sv[3], got = 0;
        uint32_t jv[kPer];
#pragma unroll
        for (uint32_t c = 0; c < kPer; ++c) {
            jv[c] = 0;
            if ((freem >> c) & 1ull) {
                if (r < avail) {
                    jv[c] = E.order ? __ldg(&E.order[h.next_j + r]) : (uint32_t)(h.next_j + r);
                    got |= 1ull << c;
                }
                ++r;
            }
        }
#pragma unroll
        for (uint32_t c = 0; c < kPer; ++c)
            if ((got >> c) & 1ull) ctl->lane_j[a0 + c] = jv[c];
        if (got) atomicOr(&sm.init[wi], got << (a0 & 63));
    }
    __syncthreads();
    if (t < WB) {
        ctl->init_w[t] = sm.init[t];
        ctl->run_w[t] = sm.still[t] | sm.init[t];
        ctl->still_w[t] = sm.still[t];
        ctl->act_w[t] = 0;
    }
    const bool any_run = nstill != 0 || assigned != 0;
    // 5. direction of the coming level
    {
        const unsigned long long np = h.new_packed, wp = h.wide_packed;
        const double U = (double)((np & kUnitMask) + (wp & kUnitMask)), G = (double)((np >> kUnitBits) + h.wide_gnew);
        const double C = (double)h.new_colours;
        const uint32_t sched = h.sched;
        const bool pull_ok = E.frontd != nullptr;
        // one feature per warp (lane 0 of warps 1..6): FP64 is slow on this
        // part, and the six logarithms overlap only in different warps
        if (((sched == FBPT_SCHED_LEARNED && E.policy) || E.trace) && (t & 31u) == 0 && t >= 32 &&
            t <= 32u * kPolicyIn && t < blockDim.x)
            sm.rawf[(t >> 5) - 1] = level_feature((t >> 5) - 1, U, G, C, (double)nstill, (double)E.m);
        if (t == 0) {
            uint32_t d = kDirPush;
            if (sched == FBPT_SCHED_PULL && pull_ok) d = kDirPull;
            else if (sched == FBPT_SCHED_FILTERED) d = kDirFiltered;
            else if (sched == FBPT_SCHED_HEURISTIC || sched == FBPT_SCHED_LEARNED)
                d = heuristic_dir(U, G, C, (double)E.m, pull_ok);
            // compaction: the option for fixed schedules; the heuristic scans when
            // the level just done reached more than n / 16 vertices
            const uint32_t reached = h.mode == FBPT_COMPACT_SCAN ? h.scan_rows : h.pend_count;
            uint32_t md = E.compaction;
            if (sched == FBPT_SCHED_HEURISTIC || sched == FBPT_SCHED_LEARNED)
                md = (uint64_t)reached * 16 > (uint64_t)E.n ? FBPT_COMPACT_SCAN : FBPT_COMPACT_QUEUE;
            if (d == kDirPull || E.model == FBPT_MODEL_LT) md = FBPT_COMPACT_QUEUE;
            sm.dir = d;
            sm.mode = md;
        }
        __syncthreads();
        if (sched == FBPT_SCHED_LEARNED && E.policy) {
            policy_forward(sm);
            if (t == 0) {
                // actions: push, filtered push, pull (queue compaction), then push
                // and filtered push with scan compaction; the smallest predicted time
                uint32_t best = kActPush;
                for (uint32_t a = 1; a < kActions; ++a) {
                    if (a == kActPull && !pull_ok) continue;
                    if (a >= kActPushScan && E.model == FBPT_MODEL_LT) continue;
                    if (sm.out[a] < sm.out[best]) best = a;
                }
                sm.dir = action_dir(best);
                sm.mode = action_mode(best);
            }
            __syncthreads();
        }
    }
    // 6. the level's bookkeeping (one thread, from the loaded fields)
    if (t == 0) {
        const uint32_t err = h.err;
        ctl->pair_cursor = h.pair_cursor + R64;
        ctl->fin_pre[F] = (uint32_t)S64;
        ctl->fin_count = F;
        // a lane whose segment overflowed has entries in the spill log: the next
        // sweep reads the log and writes the surviving entries to the other buffer
        if (any_spill) {
            const uint32_t dst = h.spill_cur ^ 1u;
            ctl->spill_cur = dst;
            ctl->spill_len[dst] = 0;
        }
        ctl->spill_sweep = any_spill ? 1u : 0u;
        // the sweep reads the log the commit just appended to (the buffer that
        // was current before the flip)
        ctl->sweep_work = max(S64, any_spill ? min(h.spill_len[h.spill_cur], (unsigned long long)E.spill_cap) : 0ull);
        const unsigned long long tick = h.tick;
        if (E.trace && tick < E.trace_cap) {
            fbpt_trace_row& row = E.trace[tick];
            row.level = tick;
            row.units = h.list_count + h.wide_units;
            row.groups = h.list_groups + h.wide_groups;
            row.compaction = h.mode;
            row.colours = h.list_colours;
            row.pending = h.mode == FBPT_COMPACT_SCAN ? h.scan_rows : h.pend_count;
            row.active_lanes = nstill;
            row.finished_lanes = F;
            row.started_lanes = assigned;
            uint64_t* pt[3] = {&row.expand_ns, &row.commit_ns, &row.sweep_ns};
            for (int p = 0; p < 3; ++p) *pt[p] = h.ph_t1[p] > h.ph_t0[p] ? h.ph_t1[p] - h.ph_t0[p] : 0;
            row.direction = h.dir;
            row.frontier_lanes = h.frontier_lanes;
        }
        // the features and network outputs the coming level's decision used
        if (E.trace && tick + 1 < E.trace_cap) {
            fbpt_trace_row& nx = E.trace[tick + 1];
            const bool net = h.sched == FBPT_SCHED_LEARNED && E.policy;
            for (int k = 0; k < kPolicyIn; ++k) nx.features[k] = sm.rawf[k];
            for (int k = 0; k < kPolicyOut; ++k) nx.outputs[k] = net ? sm.out[k] : 0.f;
        }
        ctl->list_colours = err ? 0 : h.new_colours;
        ctl->new_colours = 0;
        ctl->next_j = h.next_j + assigned;
        atomicAdd(&ctl->st_assigned, assigned);
        const unsigned long long np = h.new_packed, wp = h.wide_packed;
        ctl->list_count = err ? 0 : (np & kUnitMask);
        ctl->list_groups = err ? 0 : (np >> kUnitBits);
        ctl->wide_units = err ? 0 : (wp & kUnitMask);
        ctl->wide_chunks = err ? 0 : (wp >> kUnitBits);
        ctl->wide_groups = err ? 0 : h.wide_gnew;
        ctl->wide_packed = 0;
        ctl->wide_gnew = 0;
        ctl->wchunk_next = 0;
        atomicAdd(&ctl->st_units, (np & kUnitMask) + (wp & kUnitMask));
        const unsigned long long lg = h.list_groups + h.wide_groups;
        if (lg != 0) atomicAdd(h.dir == kDirPull ? &ctl->st_pull : &ctl->st_push, 1ull);
        if (h.dir != kDirPull) atomicAdd(&ctl->st_groups, lg);
        ctl->dir = sm.dir;
        ctl->mode = sm.mode;
        ctl->scan_rows = 0;
        ctl->frontier_lanes = nstill;
        for (int p = 0; p < 3; ++p) {
            if (h.ph_t1[p] > h.ph_t0[p]) atomicAdd(&ctl->st_phase_ns[p], h.ph_t1[p] - h.ph_t0[p]);
            ctl->ph_t0[p] = ~0ull;
            ctl->ph_t1[p] = 0;
        }
        ctl->new_packed = 0;
        ctl->chunk_next = 0;
        ctl->pend_count = 0;
        ctl->tick = tick + 1;
        uint32_t run = any_run ? 1u : 0u;
        if (tick + 1 > h.tick_limit) {
            atomicOr(&ctl->error, (unsigned)kErrTickLimit);
            run = 0;
        }
        if (err) run = 0;
        ctl->running = run;
        __threadfence();
        if (E.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)E.cond, run);
    }
    __syncthreads();
}

// ---- per-level kernels (host-driven or CUDA-graph loop) ------------------------------------

__global__ void __launch_bounds__(kThreads) k_sweep(const Eng E) {
    __shared__ uint32_t pre[kMaxLanes + 1];
    __shared__ uint64_t fin[kMaxWords];
    dev_sweep<true>(E, pre, fin);
}
// The level's first kernel: the start vertices of the lanes the last schedule
// refilled, this CTA's share of the sweep of the lanes that finished at the
// last level (the first CTAs take it, their shared memory reused for the lane
// table afterwards), then the push expand, whose chunk counter hands the other
// CTAs more chunks meanwhile.  No launch of its own for either.
__global__ void __launch_bounds__(kThreads, FBPT_EXPAND_MINB) k_expand(const Eng E) {
    __shared__ uint32_t lane_j[kMaxLanes + 1];
    __shared__ uint32_t pcnt[kThreads / 32], pbuf[kThreads / 32 * kPendBuf];
    __shared__ uint64_t fin[kMaxWords];
    extern __shared__ uint4 pstage[];  // kStageBytes, dynamic
    if (E.gated && !L2(&E.ctl->running)) return;
    dev_init(E);
    dev_sweep<true>(E, lane_j, fin);
    __syncthreads();
    dev_expand<kPartPush>(E, lane_j, pcnt, pbuf, pstage);
}
__global__ void __launch_bounds__(kThreads) k_expand_alt(const Eng E) {
    __shared__ uint32_t lane_j[kMaxLanes];
    __shared__ uint32_t pcnt[kThreads / 32], pbuf[kThreads / 32 * kPendBuf];
    extern __shared__ uint4 pstage[];  // kStageBytes, dynamic
    if (E.gated && !L2(&E.ctl->running)) return;
    dev_expand<kPartAlt>(E, lane_j, pcnt, pbuf, pstage);
}
__global__ void __launch_bounds__(kThreads) k_commit(const Eng E) {
    __shared__ Smem sm;
    if (E.gated && !L2(&E.ctl->running)) return;
    dev_commit<true>(E, sm);
}
__global__ void __launch_bounds__(kSchedThreads) k_schedule(const Eng E) {
    __shared__ Smem sm;
    if (E.gated && !L2(&E.ctl->running)) return;
    dev_schedule<kMaxLanes / kSchedThreads>(E, sm);
}

// ---- persistent form: the whole run in one cooperative launch -------------------------------

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier with a bounded wait.  The last CTA to arrive optionally
// runs the scheduler before releasing the others.  Returns false when a wait
// gave up (error bit set; the caller returns).
__device__ bool grid_barrier(const Eng& E, Smem& sm, unsigned& gen, bool schedule) {
    Ctl* ctl = E.ctl;
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.abort = 0;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        sm.last = arrived == gridDim.x;
    }
    __syncthreads();
    if (sm.last) {
        __threadfence();
        if (schedule) dev_schedule<kMaxLanes / kThreads>(E, sm);
        if (threadIdx.x == 0) {
            ctl->bar_count = 0;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        }
    } else if (threadIdx.x == 0) {
        unsigned long long spins = 0;
        while (ld_acquire_u32(&ctl->bar_gen) == gen) {
            if (++spins > E.spin_limit || (L2(&ctl->error) & kErrBarrierTimeout)) {
                atomicOr(&ctl->error, (unsigned)kErrBarrierTimeout);
                sm.abort = 1;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    ++gen;
    __syncthreads();
    return !sm.abort;
}

__global__ void __launch_bounds__(kThreads) k_run(const Eng E) {
    __shared__ Smem sm;
    extern __shared__ uint4 pstage[];  // kStageBytes, dynamic: the expand's per-warp slots
    Ctl* ctl = E.ctl;
    unsigned gen = 0;
    for (;;) {
        dev_sweep<false>(E, sm.lane, sm.fin);  // lanes finished at the previous level
        dev_init(E);       // lanes given a sample at the previous level
        dev_expand<kPartAll>(E, sm.lane, sm.pcnt, sm.pbuf, pstage);
        if (!grid_barrier(E, sm, gen, false)) return;
        dev_commit<false>(E, sm);
        if (!grid_barrier(E, sm, gen, true)) return;
        if (!L2(&ctl->running)) break;
    }
    dev_sweep<false>(E, sm.lane, sm.fin);
}

// ---- final CSR: each staged row sorted into its place -----------------------------------
//
// offsets[] is the exclusive scan of the row lengths in sample order; row j's
// vertices (distinct, in discovery order in the staging array) are written to
// verts[offsets[j] ..] ascending.  Rows of at most 32 vertices: one warp
// (bitonic network on registers); up to kMidRow: one CTA (bitonic network in
// shared memory); longer rows: one CTA marks a shared-memory bitmap of 2^20
// vertices at a time and writes the marked ids in order.

constexpr uint32_t kMidRow = 8192;
constexpr uint32_t kOrderThreads = 256;
constexpr uint32_t kBigThreads = 1024;
constexpr uint32_t kWinBits = 1u << 20;  // vertices per bitmap window (128 KB)

// Colour-edge visits of a run: every RR entry (sample, v) examines v's in-edges
// once, so the total is the sum over v of vcount[v] * indeg(v).
__global__ void k_cev(const uint64_t* row_ptr, const uint32_t* vcount, uint32_t n, unsigned long long* out) {
    unsigned long long acc = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)vcount[v] * (row_ptr[v + 1] - row_ptr[v]);
    acc = warp_sum(acc);
    if (lane_id() == 0 && acc) atomicAdd(out, acc);
}

__global__ void __launch_bounds__(kOrderThreads) k_order_tiny(const uint32_t* rows_v, const uint64_t* row_start,
                                                              const uint32_t* row_len, const uint64_t* offsets,
                                                              uint64_t S, uint32_t* verts) {
    const uint32_t lane = lane_id();
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < S; j += nwarp) {
        const uint32_t len = row_len[j];
        if (len > 32) continue;
        uint32_t v = lane < len ? rows_v[row_start[j] + lane] : 0xFFFFFFFFu;
#pragma unroll
        for (uint32_t k = 2; k <= 32; k <<= 1)
#pragma unroll
            for (uint32_t h = k >> 1; h > 0; h >>= 1) {
                const uint32_t o = __shfl_xor_sync(0xffffffffu, v, h);
                const bool up = (lane & k) == 0, low = (lane & h) == 0;
                v = (low == up) ? min(v, o) : max(v, o);
            }
        if (lane < len) verts[offsets[j] + lane] = v;
    }
}

__global__ void __launch_bounds__(kOrderThreads) k_order_mid(const uint32_t* rows_v, const uint64_t* row_start,
                                                             const uint32_t* row_len, const uint64_t* offsets,
                                                             uint64_t S, uint32_t* verts) {
    __shared__ uint32_t key[kMidRow];
    for (uint64_t j = blockIdx.x; j < S; j += gridDim.x) {
        const uint32_t len = row_len[j];
        if (len <= 32 || len > kMidRow) continue;
        uint32_t P = 64;
        while (P < len) P <<= 1;
        const uint64_t src = row_start[j];
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) key[i] = i < len ? rows_v[src + i] : 0xFFFFFFFFu;
        __syncthreads();
        for (uint32_t k = 2; k <= P; k <<= 1)
            for (uint32_t h = k >> 1; h > 0; h >>= 1) {
                for (uint32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                    const uint32_t a = 2 * t - (t & (h - 1)), b = a + h;
                    const uint32_t x = key[a], y = key[b];
                    if ((x > y) == ((a & k) == 0)) {
                        key[a] = y;
                        key[b] = x;
                    }
                }
                __syncthreads();
            }
        const uint64_t dst = offsets[j];
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) verts[dst + i] = key[i];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBigThreads) k_order_big(const uint32_t* rows_v, const uint64_t* row_start,
                                                           const uint32_t* row_len, const uint64_t* offsets,
                                                           uint64_t S, uint32_t n, uint32_t* verts) {
    extern __shared__ uint32_t bm[];  // kWinBits / 32 words
    __shared__ uint32_t wsum[kBigThreads / 32];
    __shared__ uint32_t wtot;
    constexpr uint32_t kWords = kWinBits / 32;
    constexpr uint32_t kPer = kWords / kBigThreads;  // bitmap words per thread
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    for (uint64_t j = blockIdx.x; j < S; j += gridDim.x) {
        const uint32_t len = row_len[j];
        if (len <= kMidRow) continue;
        const uint64_t src = row_start[j];
        uint64_t dst = offsets[j];
        for (uint32_t w0 = 0; w0 < n; w0 += kWinBits) {
            for (uint32_t q = t; q < kWords; q += kBigThreads) bm[q] = 0;
            __syncthreads();
            for (uint32_t i = t; i < len; i += kBigThreads) {
                const uint32_t v = rows_v[src + i] - w0;
                if (v < kWinBits) atomicOr(&bm[v >> 5], 1u << (v & 31));
            }
            __syncthreads();
            uint32_t c = 0;
#pragma unroll 4
            for (uint32_t q = 0; q < kPer; ++q) c += __popc(bm[t * kPer + q]);
            const uint32_t incl = warp_incl_scan(c);
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t x = wsum[lane];
                const uint32_t xi = warp_incl_scan(x);
                wsum[lane] = xi - x;
                if (lane == 31) wtot = xi;
            }
            __syncthreads();
            uint64_t pos = dst + wsum[warp] + incl - c;
            for (uint32_t q = 0; q < kPer; ++q) {
                uint32_t m = bm[t * kPer + q];
                while (m) {
                    const uint32_t b = __ffs(m) - 1;
                    m &= m - 1;
                    verts[pos++] = w0 + (t * kPer + q) * 32 + b;
                }
            }
            dst += wtot;
            __syncthreads();
        }
    }
}

struct LaunchShape {
    int level_blocks = 0, run_blocks = 0;
};

LaunchShape launch_shape() {
    static LaunchShape ls;
    static bool done = false;
    if (!done) {
        const int sms = device_sm_count();
        int per = 0;
        cudaFuncSetAttribute(k_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
        cudaFuncSetAttribute(k_expand_alt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
        cudaFuncSetAttribute(k_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStageBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_expand, kThreads, kStageBytes);
        ls.level_blocks = sms * std::max(per, 1);
        per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_run, kThreads, kStageBytes);
        ls.run_blocks = sms * std::max(per, 1);
        done = true;
    }
    return ls;
}

int order_rows(const uint32_t* rows_v, const uint64_t* row_start, const uint32_t* row_len, const uint64_t* offsets,
               uint64_t S, uint32_t n, uint32_t* verts, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        FBPT_CUDA_TRY(cudaFuncSetAttribute(k_order_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(kWinBits / 8)));
        attr = true;
    }
    const int sms = device_sm_count();
    const uint64_t grid = std::min<uint64_t>((S + 7) / 8, (uint64_t)sms * 8);
    k_order_tiny<<<(unsigned)std::max<uint64_t>(grid, 1), kOrderThreads, 0, st>>>(rows_v, row_start, row_len,
                                                                                    offsets, S, verts);
    k_order_mid<<<(unsigned)std::min<uint64_t>(S, (uint64_t)sms * 6), kOrderThreads, 0, st>>>(
        rows_v, row_start, row_len, offsets, S, verts);
    k_order_big<<<(unsigned)std::min<uint64_t>(S, (uint64_t)sms), kBigThreads, kWinBits / 8, st>>>(
        rows_v, row_start, row_len, offsets, S, n, verts);
    FBPT_CUDA_TRY(cudaGetLastError());
    return FBPT_OK;
}

// One level: expand (with the start vertices and the sweep of the last level's
// finished lanes), the filtered/pull expand when the level takes it, commit and
// schedule.  The sweep touches the finished lanes' segments, the spill log,
// visited[], the RR staging rows and the counts; the expand reads the frontier
// list, col/thr and the lanes' sample ids and writes next[], nocc[] and the
// pending list, so the two may share the kernel in any order across its CTAs;
// the commit, which reads visited[], follows the whole kernel.  ex0/ex1 bracket
// the expand launches.
int launch_level(const Eng& E, cudaStream_t st, int blocks, cudaEvent_t ex0 = nullptr, cudaEvent_t ex1 = nullptr) {
    if (ex0) FBPT_CUDA_TRY(cudaEventRecord(ex0, st));
    k_expand<<<blocks, kThreads, kStageBytes, st>>>(E);
    if (E.alt) k_expand_alt<<<blocks, kThreads, kStageBytes, st>>>(E);
    if (ex1) FBPT_CUDA_TRY(cudaEventRecord(ex1, st));
    k_commit<<<blocks, kThreads, 0, st>>>(E);
    k_schedule<<<1, kSchedThreads, 0, st>>>(E);
    FBPT_CUDA_TRY(cudaGetLastError());
    return FBPT_OK;
}

int launch_final_sweep(const Eng& E, cudaStream_t st, int blocks) {
    k_sweep<<<blocks, kThreads, 0, st>>>(E);
    FBPT_CUDA_TRY(cudaGetLastError());
    return FBPT_OK;
}

int run_persistent(const Eng& E, cudaStream_t st) {
    const LaunchShape ls = launch_shape();
    Eng e = E;
    void* args[] = {(void*)&e};
    cudaError_t err =
        cudaLaunchCooperativeKernel((const void*)k_run, dim3(ls.run_blocks), dim3(kThreads), args, kStageBytes, st);
    if (err != cudaSuccess) {
        cudaGetLastError();
        return fail(FBPT_ECUDA, std::string("cooperative launch: ") + cudaGetErrorString(err));
    }
    return FBPT_OK;
}

// Adds to `graph` a WHILE conditional node (after deps) whose body is one
// level of E's run; the scheduler kernel sets the condition.
int add_level_loop(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps, Eng E, int blocks,
                   cudaGraphNode_t* node) {
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
        return fail(FBPT_ECUDA, "cudaGraphConditionalHandleCreate failed");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    if (cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &p) != cudaSuccess)
        return fail(FBPT_ECUDA, "cudaGraphAddNode(conditional) failed");
    cudaGraph_t body = p.conditional.phGraph_out[0];
    cudaStream_t cs = nullptr;
    auto release = [&]() {
        if (cs) cudaStreamDestroy(cs);
    };
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(FBPT_ECUDA, "stream create failed");
    }
    E.cond = (unsigned long long)h;
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        release();
        return fail(FBPT_ECUDA, "cudaStreamBeginCaptureToGraph failed");
    }
    const int lrc = launch_level(E, cs, blocks);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    release();
    if (lrc != FBPT_OK) return lrc;
    if (ce != cudaSuccess) return fail(FBPT_ECUDA, std::string("capture failed: ") + cudaGetErrorString(ce));
    return FBPT_OK;
}

// The level loop of one run as one CUDA graph, then the last sweep.
int run_graph(const Eng& E, cudaStream_t st, int blocks) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FBPT_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphNode_t node;
    int rc = add_level_loop(graph, nullptr, 0, E, blocks, &node);
    if (rc == FBPT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        rc = fail(FBPT_ECUDA, "cudaGraphInstantiate failed");
    if (rc == FBPT_OK && cudaGraphLaunch(exec, st) != cudaSuccess) rc = fail(FBPT_ECUDA, "cudaGraphLaunch failed");
    if (rc == FBPT_OK) rc = launch_final_sweep(E, st, blocks);
    if (exec) {
        cudaStreamSynchronize(st);
        cudaGraphExecDestroy(exec);
    }
    cudaGraphDestroy(graph);
    return rc;
}

template <typename T>
int dalloc(T** p, uint64_t count, size_t& bytes) {
    const size_t b = sizeof(T) * std::max<uint64_t>(count, 1);
    cudaError_t e = cudaMalloc((void**)p, b);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? FBPT_ENOMEM : FBPT_ECUDA,
                    std::string("cudaMalloc(") + std::to_string(b) + "): " + cudaGetErrorString(e));
    }
    bytes += b;
    return FBPT_OK;
}

void ws_free(Workspace* w) {
    if (!w) return;
    cudaFree(w->visited); cudaFree(w->next); cudaFree(w->nocc); cudaFree(w->stage); cudaFree(w->pend_v);
    cudaFree(w->seg); cudaFree(w->spill); cudaFree(w->list_v); cudaFree(w->list_mrow); cudaFree(w->list_only); cudaFree(w->list_rs);
    cudaFree(w->list_re); cudaFree(w->list_g); cudaFree(w->list_occ); cudaFree(w->chunk_u0); cudaFree(w->ctl);
    cudaFree(w->wide_rec); cudaFree(w->wide_chunk);
    cudaFree(w->frontd); cudaFree(w->fstamp);
    if (w->ctl_host) cudaFreeHost(w->ctl_host);
    delete w;
}

int ws_zero(Workspace* w, cudaStream_t st) {
    const uint64_t rows = (uint64_t)w->n * w->WB;
    FBPT_CUDA_TRY(cudaMemsetAsync(w->visited, 0, rows * 8, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(w->next, 0, rows * 8, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(w->nocc, 0, (uint64_t)w->n * 8, st));
    w->clean = true;
    return FBPT_OK;
}

int ws_get(fbpt_graph* g, uint32_t WB, bool unfused, bool dense, cudaStream_t st, Workspace** out) {
    Workspace* w = g->ws;
    if (w && w->WB == WB && w->unfused == unfused && (w->frontd != nullptr) == dense) {
        if (!w->clean) FBPT_TRY(ws_zero(w, st));
        *out = w;
        return FBPT_OK;
    }
    if (w) {
        cudaStreamSynchronize(st);
        ws_free(w);
        g->ws = nullptr;
    }
    w = new Workspace();
    w->n = g->n;
    w->WB = WB;
    w->unfused = unfused;
    const uint64_t n = g->n;
    const uint64_t rows = n * WB;
    w->pend_cap = n;
    w->list_cap = unfused ? std::min<uint64_t>(n * 64ull * WB, std::max<uint64_t>(16 * n, 1 << 20)) : n;
    if (w->list_cap > kUnitMask) w->list_cap = kUnitMask;
    // groups of a row [rs, re) are at most (re - rs) / 4 + 2
    const uint64_t max_groups = (g->m / 4 + 2 * n + 1) * (unfused ? 64ull * WB : 1ull);
    w->chunk_cap = std::min<uint64_t>(max_groups / kChunk + 2, 0xFFFFFFFFull);
    // a wide unit's chunks are at most twice its groups / 32 (it has >= 32 groups)
    w->wide_chunk_cap = std::min<uint64_t>(2 * (max_groups / kChunk) + 2, 0xFFFFFFFFull);
    w->spill_cap = std::max<uint64_t>(1ull << 22, 4 * n);
    int rc = FBPT_OK;
    size_t& b = w->bytes;
    if (rc == FBPT_OK) rc = dalloc(&w->visited, rows, b);
    if (rc == FBPT_OK) rc = dalloc(&w->next, rows, b);
    if (rc == FBPT_OK) rc = dalloc(&w->nocc, n, b);
    if (rc == FBPT_OK) rc = dalloc(&w->stage, w->pend_cap * WB, b);
    if (rc == FBPT_OK) rc = dalloc(&w->pend_v, w->pend_cap, b);
    w->seg_cap = kSegMin;
    if (rc == FBPT_OK) rc = dalloc(&w->seg, 64ull * WB * w->seg_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->spill, 2 * w->spill_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_v, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_mrow, w->list_cap, b);
    if (rc == FBPT_OK && unfused) rc = dalloc(&w->list_only, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_rs, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_re, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_g, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_occ, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->chunk_u0, w->chunk_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->wide_rec, 2 * w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->wide_chunk, w->wide_chunk_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->ctl, 1, b);
    if (rc == FBPT_OK && dense) rc = dalloc(&w->frontd, rows, b);
    if (rc == FBPT_OK && dense) rc = dalloc(&w->fstamp, n, b);
    if (rc == FBPT_OK && cudaMallocHost((void**)&w->ctl_host, sizeof(Ctl)) != cudaSuccess)
        rc = fail(FBPT_ENOMEM, "cudaMallocHost(ctl) failed");
    if (rc == FBPT_OK) rc = ws_zero(w, st);
    if (rc != FBPT_OK) {
        ws_free(w);
        return rc;
    }
    g->ws = w;
    *out = w;
    return FBPT_OK;
}


}  // namespace


namespace {

// ---- one sampling run, in steps the batched path reuses -------------------------------

struct Run {
    fbpt_graph* g = nullptr;
    uint64_t seed = 0, first_id = 0, S = 0;
    fbpt_opts o = {};
    uint32_t WB = 0;
    int blocks = 0;
    bool dense = false;
    cudaStream_t st = nullptr;
    Workspace* ws = nullptr;
    fbpt_rrsets* out = nullptr;
    uint64_t cap = 0;               // staging entries
    uint32_t* rows_v = nullptr;     // staging: each finished sample's RR row, unsorted
    uint64_t* row_start = nullptr;  // S
    uint32_t* row_len = nullptr;    // S
    fbpt_trace_row* dtrace = nullptr;
    uint32_t* order = nullptr;      // S: sample index of each refill position (sorted starts), or NULL
    double expand_event_ms = 0.0;   // host-launched levels: CUDA-event time of the expand launches
    Ctl* H = nullptr;               // pinned: the initial control block in, the final one out
    Eng E = {};
};

void release_out(fbpt_rrsets* out) {
    if (!out) return;
    cudaStream_t st = (cudaStream_t)out->stream;
    if (out->offsets) cudaFreeAsync(out->offsets, st);
    if (out->verts) cudaFreeAsync(out->verts, st);
    if (out->starts) cudaFreeAsync(out->starts, st);
    if (out->vcount) cudaFreeAsync(out->vcount, st);
    std::memset(out, 0, sizeof(*out));
}

void run_release(Run& r, bool with_out) {
    if (r.rows_v) cudaFreeAsync(r.rows_v, r.st);
    if (r.row_start) cudaFreeAsync(r.row_start, r.st);
    if (r.row_len) cudaFreeAsync(r.row_len, r.st);
    if (r.dtrace) cudaFreeAsync(r.dtrace, r.st);
    if (r.order) cudaFreeAsync(r.order, r.st);
    r.rows_v = nullptr;
    r.row_start = nullptr;
    r.row_len = nullptr;
    r.dtrace = nullptr;
    r.order = nullptr;
    if (with_out) release_out(r.out);
}

// Replaces the spill log by an empty one of `cap` entries per buffer.
int grow_spill(Workspace* ws, uint64_t cap, cudaStream_t st) {
    cudaStreamSynchronize(st);
    cudaFree(ws->spill);
    ws->spill = nullptr;
    ws->spill_cap = cap;
    size_t unused = 0;
    const int rc = dalloc(&ws->spill, 2 * cap, unused);
    if (rc != FBPT_OK) ws->spill_cap = 0;  // the kernels then flag overflow instead of writing
    return rc;
}

constexpr uint64_t kSpillMax = 1ull << 31;
constexpr uint64_t kWideChunkMax = 0xFFFFFFFFull;

// Replaces the wide-chunk map by one of `cap` entries.
int grow_wide_chunks(Workspace* ws, uint64_t cap, cudaStream_t st) {
    cudaStreamSynchronize(st);
    cudaFree(ws->wide_chunk);
    ws->wide_chunk = nullptr;
    ws->wide_chunk_cap = cap;
    size_t unused = 0;
    const int rc = dalloc(&ws->wide_chunk, cap, unused);
    if (rc != FBPT_OK) ws->wide_chunk_cap = 0;
    return rc;
}

// Validates the arguments, gets the workspace and the output's fixed-size buffers.
// force_wb (when not 0) sets the row width in words instead of the options:
// tasks of a batch that share a graph use the widest of their widths.
int run_setup(Run& r, fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, const fbpt_opts* opts,
              fbpt_rrsets* out, uint32_t force_wb = 0) {
    if (!g || !out) return fail(FBPT_EINVAL, "fbpt_sample: null graph or output");
    std::memset(out, 0, sizeof(*out));
    if (S == 0 || S > 0xFFFFFFFFull) return fail(FBPT_EINVAL, "fbpt_sample: S must be in [1, 2^32)");
    if (first_id + S < first_id) return fail(FBPT_EINVAL, "fbpt_sample: sample ids overflow");
    fbpt_opts o = {};
    if (opts) o = *opts;
    const uint32_t W = o.words ? o.words : 8;
    if (W != 1 && W != 2 && W != 4 && W != 8) return fail(FBPT_EINVAL, "fbpt_sample: words must be 1, 2, 4 or 8");
    const uint32_t B = o.slots ? o.slots : kMaxWords / W;
    if (B < 1 || B * W > kMaxWords) return fail(FBPT_EINVAL, "fbpt_sample: words * slots must be <= 64");
    // never more lanes than samples (rounded up to whole words)
    const uint32_t WB = force_wb ? force_wb : (uint32_t)std::min<uint64_t>(W * B, (S + 63) / 64);
    if (WB > kMaxWords) return fail(FBPT_EINVAL, "fbpt_sample: row width above 64 words");
    if (o.schedule > FBPT_SCHED_FILTERED) return fail(FBPT_EINVAL, "fbpt_sample: bad schedule");
    if (o.model != FBPT_MODEL_IC && o.model != FBPT_MODEL_LT) return fail(FBPT_EINVAL, "fbpt_sample: bad model");
    if (o.model == FBPT_MODEL_LT) {
        // LT levels are push only: a choice among other directions does not apply
        if (o.schedule == FBPT_SCHED_PULL || o.schedule == FBPT_SCHED_FILTERED || o.unfused)
            return fail(FBPT_EUNSUPPORTED, "fbpt_sample: the LT model runs fused push levels only");
        o.schedule = FBPT_SCHED_PUSH;
    }
    // pull levels need dense frontier rows (WB <= 8 words), fused units, 32-bit
    // edge ids and the caller's vertex order
    const bool pull_ok = WB <= kPullMaxWords && !o.unfused && g->m < (1ull << 32) && !g->perm;
    if (o.schedule == FBPT_SCHED_PULL && !pull_ok)
        return fail(FBPT_EUNSUPPORTED,
                    "fbpt_sample: pull needs words * slots <= 8, fused units, m < 2^32 and no vertex order");
    if (o.schedule == FBPT_SCHED_LEARNED && o.policy && !o.policy->d_params)
        return fail(FBPT_EINVAL, "fbpt_sample: policy has no parameters");
    if (o.launch != FBPT_LAUNCH_HOST && o.launch != FBPT_LAUNCH_GRAPH && o.launch != FBPT_LAUNCH_PERSISTENT)
        return fail(FBPT_EINVAL, "fbpt_sample: bad launch mode");
    if (o.refill != FBPT_REFILL_LANE && o.refill != FBPT_REFILL_BATCH)
        return fail(FBPT_EINVAL, "fbpt_sample: bad refill mode");
    if (o.compaction != FBPT_COMPACT_QUEUE && o.compaction != FBPT_COMPACT_SCAN)
        return fail(FBPT_EINVAL, "fbpt_sample: bad compaction mode");
    r.g = g;
    r.seed = seed;
    r.first_id = first_id;
    r.S = S;
    r.o = o;
    r.WB = WB;
    r.dense = pull_ok && (o.schedule == FBPT_SCHED_PULL || o.schedule == FBPT_SCHED_HEURISTIC ||
                          o.schedule == FBPT_SCHED_LEARNED);
    r.st = o.stream ? (cudaStream_t)o.stream : g->stream;
    const int full = launch_shape().level_blocks;
    r.blocks = o.blocks ? std::max(1, std::min<int>((int)o.blocks, full)) : full;
    r.out = out;

    if (r.dense) FBPT_TRY(ensure_out_csr(g, r.st));
    if (o.model == FBPT_MODEL_LT) FBPT_TRY(ensure_lt_weights(g, r.st));
    FBPT_TRY(ws_get(g, WB, o.unfused != 0, r.dense, r.st, &r.ws));
    // per-lane segments sized to hold about twice the expected RR set, so that
    // few lanes fall back to the shared spill log (which the sweep compacts
    // every level); the rest of a longer set goes to the log
    {
        uint64_t want = kSegMin;
        while (want < 2.0 * g->rr_hint && 64ull * WB * (want * 2) * sizeof(uint32_t) <= kSegBytesMax) want *= 2;
        if (want > r.ws->seg_cap) {
            cudaStreamSynchronize(r.st);
            cudaFree(r.ws->seg);
            r.ws->seg = nullptr;
            r.ws->seg_cap = 0;
            size_t unused = 0;
            FBPT_TRY(dalloc(&r.ws->seg, 64ull * WB * want, unused));
            r.ws->seg_cap = (uint32_t)want;
        }
        const double over = g->rr_hint * 1.5 - (double)r.ws->seg_cap;
        const double spill_want = 64.0 * WB * over;
        if (over > 0 && spill_want > (double)r.ws->spill_cap && r.ws->spill_cap < kSpillMax)
            FBPT_TRY(grow_spill(r.ws, std::min<uint64_t>((uint64_t)spill_want, kSpillMax), r.st));
    }
    r.H = r.ws->ctl_host;

    out->S = S;
    out->n = g->n;
    out->stream = r.st;
    FBPT_CUDA_TRY(cudaMallocAsync(&out->starts, sizeof(uint32_t) * S, r.st));
    FBPT_CUDA_TRY(cudaMallocAsync(&out->vcount, sizeof(uint32_t) * g->n, r.st));
    FBPT_CUDA_TRY(cudaMallocAsync(&out->offsets, sizeof(uint64_t) * (S + 1), r.st));
    FBPT_CUDA_TRY(cudaMallocAsync(&r.row_start, sizeof(uint64_t) * S, r.st));
    FBPT_CUDA_TRY(cudaMallocAsync(&r.row_len, sizeof(uint32_t) * S, r.st));
    r.cap = (uint64_t)(g->rr_hint * 1.25 * (double)S) + 4096;
    if (o.trace && o.trace_cap)
        FBPT_CUDA_TRY(cudaMallocAsync(&r.dtrace, sizeof(fbpt_trace_row) * o.trace_cap, r.st));
    return FBPT_OK;
}

// Sizes the staging buffer and writes the initial control block (host side) and
// the kernel parameters of one attempt.
int run_arm(Run& r) {
    fbpt_graph* g = r.g;
    Workspace* ws = r.ws;
    if (g->sorted_starts && !r.order) FBPT_TRY(start_order(g, r.seed, r.first_id, r.S, r.st, &r.order));
    if (r.rows_v) cudaFreeAsync(r.rows_v, r.st);
    r.rows_v = nullptr;
    FBPT_CUDA_TRY(cudaMallocAsync(&r.rows_v, sizeof(uint32_t) * r.cap, r.st));
    if (r.dtrace) FBPT_CUDA_TRY(cudaMemsetAsync(r.dtrace, 0, sizeof(fbpt_trace_row) * r.o.trace_cap, r.st));
    Ctl* H = r.H;
    std::memset(H, 0, sizeof(Ctl));
    H->S = r.S;
    H->sched = r.o.schedule;
    H->dir = r.o.schedule == FBPT_SCHED_FILTERED ? kDirFiltered : kDirPush;
    H->mode = FBPT_COMPACT_QUEUE;  // the first levels carry only the start vertices
    H->refill = r.o.refill == FBPT_REFILL_BATCH ? kRefillBatch : kRefillLane;
    H->running = 1;  // the first level runs (the scheduler sets it from then on)
    H->pair_cap = r.cap;
    for (int p = 0; p < 3; ++p) H->ph_t0[p] = ~0ull;
    const uint64_t waves = r.S / (64ull * r.WB) + 2;
    H->tick_limit = std::min<uint64_t>(waves * ((uint64_t)g->n + 2) + 16, 1ull << 40);

    Eng& E = r.E;
    E = Eng{};
    E.n = g->n; E.WB = r.WB;
    E.row_ptr = g->row_ptr; E.col = g->col; E.thr = g->thr;
    E.rstart = g->rstart ? g->rstart : g->row_ptr;
    E.rend = g->rend ? g->rend : g->row_ptr + 1;
    E.perm = g->perm;
    E.inv = g->inv;
    E.order = r.order;
    E.seed = r.seed; E.first_id = r.first_id; E.S = r.S;
    {
        uint32_t a = (uint32_t)r.seed, b = (uint32_t)(r.seed >> 32);
        for (int k = 0; k < 10; ++k, a += kPhiloxW0, b += kPhiloxW1) {
            E.key0[k] = a;
            E.key1[k] = b;
        }
    }
    E.visited = ws->visited; E.next = ws->next; E.nocc = ws->nocc; E.stage = ws->stage;
    E.pend_v = ws->pend_v; E.seg = ws->seg; E.seg_cap = ws->seg_cap; E.spill = ws->spill;
    E.list_v = ws->list_v; E.list_mrow = ws->list_mrow; E.list_only = ws->list_only;
    E.list_rs = ws->list_rs; E.list_re = ws->list_re; E.list_g = ws->list_g; E.list_occ = ws->list_occ;
    E.chunk_u0 = ws->chunk_u0;
    E.wide_rec = ws->wide_rec; E.wide_chunk = ws->wide_chunk; E.wide_chunk_cap = ws->wide_chunk_cap;
    E.orow = g->orow; E.odst = g->odst; E.oeid = g->oeid;
    E.frontd = ws->frontd; E.fstamp = ws->fstamp;
    E.policy = (r.o.schedule == FBPT_SCHED_LEARNED && r.o.policy) ? r.o.policy->d_params : nullptr;
    E.alt = r.o.schedule == FBPT_SCHED_PUSH ? 0u : 1u;
    E.model = r.o.model;
    E.compaction = r.o.compaction == FBPT_COMPACT_SCAN && r.o.schedule != FBPT_SCHED_PULL ? FBPT_COMPACT_SCAN
                                                                                       : FBPT_COMPACT_QUEUE;
    E.wpre = g->wpre;
    E.m = g->m;
    E.pend_cap = ws->pend_cap; E.list_cap = ws->list_cap; E.chunk_cap = ws->chunk_cap;
    E.spill_cap = ws->spill_cap;
    E.unfused = r.o.unfused ? 1u : 0u;
    E.ctl = ws->ctl;
    E.starts = r.out->starts; E.vcount = r.out->vcount;
    E.rows_v = r.rows_v; E.row_start = r.row_start; E.row_len = r.row_len;
    E.cond = 0;
    E.spin_limit = r.o.spin_limit ? r.o.spin_limit : (1ull << 26);
    E.trace = r.dtrace;
    E.trace_cap = r.dtrace ? r.o.trace_cap : 0;
    ws->clean = false;
    return FBPT_OK;
}

// Enqueues one attempt on the run's stream and reads the final control block
// back into r.H (the caller synchronises).
int run_enqueue(Run& r) {
    Workspace* ws = r.ws;
    const cudaStream_t st = r.st;
    FBPT_CUDA_TRY(cudaMemcpyAsync(ws->ctl, r.H, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(r.out->vcount, 0, sizeof(uint32_t) * r.g->n, st));
    if (ws->fstamp) FBPT_CUDA_TRY(cudaMemsetAsync(ws->fstamp, 0xFF, sizeof(uint32_t) * r.g->n, st));
    int rc = FBPT_OK;
    if (r.o.launch == FBPT_LAUNCH_GRAPH) {
        rc = run_graph(r.E, st, r.blocks);
    } else if (r.o.launch == FBPT_LAUNCH_PERSISTENT) {
        rc = run_persistent(r.E, st);
    } else {
        // host-driven levels, one level queued ahead of the one the host waits
        // for: level L + 1 is enqueued before the host reads level L's loop
        // condition, and its kernels return at once (gated) if level L ended
        // the run.  So the stream is busy when a level is enqueued, and the
        // CUDA events around each level's expand launches bracket the kernels
        // rather than the host's launch latency; their times are summed into
        // ms_expand_events for the levels that ran.
        Eng eg = r.E;
        eg.gated = 1;
        cudaEvent_t ex[4] = {}, done[2] = {};
        bool ev_ok = true;
        for (auto& e : ex) ev_ok = ev_ok && cudaEventCreate(&e) == cudaSuccess;
        for (auto& e : done) ev_ok = ev_ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
        auto destroy = [&]() {
            for (auto& e : ex) if (e) cudaEventDestroy(e);
            for (auto& e : done) if (e) cudaEventDestroy(e);
        };
        if (!ev_ok) {
            destroy();
            cudaGetLastError();
            return fail(FBPT_ECUDA, "level loop: event create failed");
        }
        r.expand_event_ms = 0.0;
        auto enqueue = [&](uint64_t L) -> int {
            const int b = (int)(L & 1);
            FBPT_TRY(launch_level(eg, st, r.blocks, ex[2 * b], ex[2 * b + 1]));
            FBPT_CUDA_TRY(cudaMemcpyAsync(&r.H->host_flag[b], &ws->ctl->running, sizeof(unsigned),
                                          cudaMemcpyDeviceToHost, st));
            FBPT_CUDA_TRY(cudaEventRecord(done[b], st));
            return FBPT_OK;
        };
        rc = enqueue(0);
        for (uint64_t L = 0; rc == FBPT_OK; ++L) {
            rc = enqueue(L + 1);
            if (rc != FBPT_OK) break;
            const int b = (int)(L & 1);
            if (cudaEventSynchronize(done[b]) != cudaSuccess) {
                rc = fail(FBPT_ECUDA, std::string("level loop: ") + cudaGetErrorString(cudaGetLastError()));
                break;
            }
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ex[2 * b], ex[2 * b + 1]) == cudaSuccess) r.expand_event_ms += ms;
            if (!r.H->host_flag[b]) break;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == FBPT_OK)
            rc = fail(FBPT_ECUDA, std::string("level loop: ") + cudaGetErrorString(cudaGetLastError()));
        destroy();
        if (rc == FBPT_OK) rc = launch_final_sweep(r.E, st, r.blocks);
    }
    if (rc != FBPT_OK) return rc;
    FBPT_CUDA_TRY(cudaMemcpyAsync(r.H, ws->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    return FBPT_OK;
}

// Reads the outcome of an attempt from r.H.  Sets again when the run must be
// repeated: the spill log was too small (grown here; the workspace is reset)
// or the staging buffer was (its exact size is now known).
int run_check(Run& r, fbpt_stats* stats, bool& again) {
    again = false;
    const Ctl* H = r.H;
    Workspace* ws = r.ws;
    if (H->error & kErrBarrierTimeout) return fail(FBPT_ETIMEOUT, "sampling run: a grid barrier wait gave up");
    const unsigned growable = kErrSpillOverflow | kErrWideOverflow;
    if (H->error && (H->error & ~growable) == 0 &&
        (!(H->error & kErrSpillOverflow) || ws->spill_cap < kSpillMax) &&
        (!(H->error & kErrWideOverflow) || ws->wide_chunk_cap < kWideChunkMax)) {
        // long RR sets outgrew the spill log, or many-colour units the wide-chunk
        // map: grow what overflowed and run again from a clean state
        if (H->error & kErrSpillOverflow)
            FBPT_TRY(grow_spill(ws, std::min<uint64_t>(ws->spill_cap * 8, kSpillMax), r.st));
        if (H->error & kErrWideOverflow)
            FBPT_TRY(grow_wide_chunks(ws, std::min<uint64_t>(std::max<uint64_t>(2 * H->wide_need, 2 * ws->wide_chunk_cap),
                                                             kWideChunkMax), r.st));
        FBPT_TRY(ws_zero(ws, r.st));
        if (stats) stats->overflow_reruns += 1;
        again = true;
        return FBPT_OK;
    }
    if (H->error)
        return fail(FBPT_EDEVICE, "sampling run: device check failed (error bits " + std::to_string(H->error) + ")");
    ws->clean = true;  // every lane finished and was swept: the kernels restored the zero state
    if (H->pair_cursor > r.cap) {
        r.cap = H->pair_cursor + 1024;
        if (stats) stats->overflow_reruns += 1;
        again = true;
    }
    return FBPT_OK;
}

// Runs attempts until one fits (at most 8).
int run_attempts(Run& r, fbpt_stats* stats) {
    for (int attempt = 0; attempt < 8; ++attempt) {
        FBPT_TRY(run_arm(r));
        FBPT_TRY(run_enqueue(r));
        if (cudaStreamSynchronize(r.st) != cudaSuccess)
            return fail(FBPT_ECUDA, std::string("sampling run: ") + cudaGetErrorString(cudaGetLastError()));
        bool again = false;
        FBPT_TRY(run_check(r, stats, again));
        if (!again) return FBPT_OK;
    }
    return fail(FBPT_ENOMEM, "fbpt_sample: output did not fit after re-runs");
}

// Trace copy, the CSR (offsets by a scan of the row lengths, each row sorted
// into place), statistics.
int run_finish(Run& r, fbpt_stats* stats) {
    const Ctl* H = r.H;
    const cudaStream_t st = r.st;
    fbpt_rrsets* out = r.out;
    if (r.dtrace) {
        const uint64_t rows = std::min<uint64_t>(H->tick, r.o.trace_cap);
        if (cudaMemcpyAsync(r.o.trace, r.dtrace, sizeof(fbpt_trace_row) * rows, cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return fail(FBPT_ECUDA, "fbpt_sample: trace copy failed");
        if (stats) stats->trace_rows = rows;
    }
    const uint64_t total = H->pair_cursor;
    r.g->rr_hint = std::max(1.0, (double)total / (double)r.S);
    FBPT_TRY(exclusive_scan_u32(r.row_len, out->offsets, r.S, st));
    if (cudaMallocAsync(&out->verts, sizeof(uint32_t) * std::max<uint64_t>(total, 1), st) != cudaSuccess)
        return fail(FBPT_ENOMEM, "fbpt_sample: verts");
    FBPT_TRY(order_rows(r.rows_v, r.row_start, r.row_len, out->offsets, r.S, r.g->n, out->verts, st));
    unsigned long long cev = 0;
    if (stats) {
        FBPT_CUDA_TRY(cudaMemsetAsync(&r.ws->ctl->st_cev, 0, sizeof(unsigned long long), st));
        k_cev<<<device_sm_count() * 4, 256, 0, st>>>(r.g->row_ptr, out->vcount, r.g->n, &r.ws->ctl->st_cev);
        FBPT_CUDA_TRY(cudaGetLastError());
        FBPT_CUDA_TRY(cudaMemcpyAsync(&r.H->st_cev, &r.ws->ctl->st_cev, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, st));
        FBPT_CUDA_TRY(cudaStreamSynchronize(st));
        cev = r.H->st_cev;
    }
    cudaFreeAsync(r.rows_v, st);
    cudaFreeAsync(r.row_start, st);
    cudaFreeAsync(r.row_len, st);
    if (r.order) cudaFreeAsync(r.order, st);
    r.rows_v = nullptr;
    r.row_start = nullptr;
    r.row_len = nullptr;
    r.order = nullptr;
    out->total = total;
    if (stats) {
        stats->levels += H->tick;
        stats->batches += (r.S + 64ull * r.WB - 1) / (64ull * r.WB);
        stats->push_levels += H->st_push;
        stats->pull_levels += H->st_pull;
        stats->units_expanded += H->st_units;
        stats->edge_accesses += H->st_edges;
        stats->philox_calls += H->st_calls;
        stats->colour_edge_visits += cev;
        stats->rr_total += total;
        stats->mask_words += H->st_mask_words;
        stats->groups_expanded += H->st_groups;
        stats->ms_expand += 1e-6 * (double)H->st_phase_ns[0];
        stats->ms_commit += 1e-6 * (double)H->st_phase_ns[1];
        stats->ms_sweep += 1e-6 * (double)H->st_phase_ns[2];
        stats->ms_expand_events += r.expand_event_ms;
    }
    return FBPT_OK;
}

// Device time between two events recorded on the same stream; 0 if unavailable.
float elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    Events() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~Events() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// Adds one task's branch to the batched graph: control block in, vcount (and
// pull stamps) cleared, the level loop, the last sweep, control block out.
int add_task(cudaGraph_t graph, const cudaGraphNode_t* dep, Run& r, cudaGraphNode_t* tail) {
    cudaGraphNode_t a, b;
    FBPT_CUDA_TRY(cudaGraphAddMemcpyNode1D(&a, graph, dep, dep ? 1 : 0, r.ws->ctl, r.H, sizeof(Ctl),
                                           cudaMemcpyHostToDevice));
    cudaMemsetParams mp = {};
    mp.dst = r.out->vcount;
    mp.elementSize = 4;
    mp.width = r.g->n;
    mp.height = 1;
    mp.value = 0;
    FBPT_CUDA_TRY(cudaGraphAddMemsetNode(&b, graph, &a, 1, &mp));
    if (r.ws->fstamp) {
        mp.dst = r.ws->fstamp;
        mp.value = 0xFFFFFFFFu;
        FBPT_CUDA_TRY(cudaGraphAddMemsetNode(&a, graph, &b, 1, &mp));
        b = a;
    }
    FBPT_TRY(add_level_loop(graph, &b, 1, r.E, r.blocks, &a));
    Eng Ef = r.E;
    Ef.cond = 0;
    void* args[] = {(void*)&Ef};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_sweep;
    kp.gridDim = dim3(r.blocks);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    FBPT_CUDA_TRY(cudaGraphAddKernelNode(&b, graph, &a, 1, &kp));
    FBPT_CUDA_TRY(cudaGraphAddMemcpyNode1D(tail, graph, &b, 1, r.H, r.ws->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    return FBPT_OK;
}

}  // namespace

int workspace_release(fbpt_graph* g) {
    if (g && g->ws) {
        ws_free(g->ws);
        g->ws = nullptr;
    }
    return FBPT_OK;
}

// One sampling run (rows first_id .. first_id+S-1) into out.
int sample_impl(fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, const fbpt_opts* opts, fbpt_rrsets* out,
                fbpt_stats* stats) {
    Run r;
    int rc = run_setup(r, g, seed, first_id, S, opts, out);
    Events ev;
    if (rc == FBPT_OK) {
        cudaEventRecord(ev.a, r.st);
        rc = run_attempts(r, stats);
    }
    if (rc == FBPT_OK) rc = run_finish(r, stats);
    if (rc != FBPT_OK) {
        run_release(r, true);
        return rc;
    }
    cudaEventRecord(ev.b, r.st);
    const float ms = elapsed_ms(ev.a, ev.b);
    if (stats) stats->ms_total += ms;
    return FBPT_OK;
}

int sample_batched_impl(uint32_t G, fbpt_graph* const* gs, const uint64_t* seeds, const uint64_t* first_ids,
                        const uint64_t* Ss, const fbpt_opts* opts, fbpt_rrsets* outs, fbpt_stats* stats) {
    if (G == 0 || !gs || !seeds || !first_ids || !Ss || !outs)
        return fail(FBPT_EINVAL, "fbpt_sample_batched: null argument");
    for (uint32_t i = 0; i < G; ++i) std::memset(&outs[i], 0, sizeof(outs[i]));
    fbpt_opts base = {};
    if (opts) base = *opts;
    base.trace = nullptr;
    base.trace_cap = 0;
    std::vector<fbpt_opts> oi(G, base);
    for (uint32_t i = 0; i < G; ++i) {
        if (!gs[i]) return fail(FBPT_EINVAL, "fbpt_sample_batched: null graph");
        if (base.words == 0 && gs[i]->tuned_valid) {
            oi[i].words = gs[i]->tuned.words;
            oi[i].slots = gs[i]->tuned.slots;
            oi[i].refill = gs[i]->tuned.refill;
            oi[i].blocks = gs[i]->tuned.blocks;
            oi[i].schedule = gs[i]->tuned.schedule;
        }
    }
    if (base.launch == FBPT_LAUNCH_HOST) {
        // the plain form: one run after another
        for (uint32_t i = 0; i < G; ++i) {
            const int rc = sample_impl(gs[i], seeds[i], first_ids[i], Ss[i], &oi[i], &outs[i], stats);
            if (rc != FBPT_OK) {
                for (uint32_t j = 0; j < i; ++j) release_out(&outs[j]);
                return rc;
            }
        }
        return FBPT_OK;
    }
    for (uint32_t i = 0; i < G; ++i) oi[i].launch = FBPT_LAUNCH_GRAPH;
    Ctl* Hs = nullptr;
    if (cudaMallocHost((void**)&Hs, sizeof(Ctl) * G) != cudaSuccess) {
        cudaGetLastError();
        return fail(FBPT_ENOMEM, "fbpt_sample_batched: pinned control blocks");
    }
    std::vector<Run> runs(G);
    cudaStream_t st = base.stream ? (cudaStream_t)base.stream : gs[0]->stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    Events ev;
    int rc = FBPT_OK;
    // tasks on one graph share its workspace, so they share one row width: the
    // widest any of them would get alone (a lane without a sample stays idle)
    std::vector<uint32_t> wb(G, 0);
    for (uint32_t i = 0; i < G; ++i) {
        const uint32_t W = oi[i].words ? oi[i].words : 8;
        const uint32_t B = oi[i].slots ? oi[i].slots : kMaxWords / std::max<uint32_t>(W, 1);
        wb[i] = (uint32_t)std::min<uint64_t>((uint64_t)W * B, (Ss[i] + 63) / 64);
    }
    for (uint32_t i = 0; i < G; ++i)
        for (uint32_t j = 0; j < G; ++j)
            if (gs[j] == gs[i]) wb[i] = std::max(wb[i], wb[j]);
    for (uint32_t i = 0; i < G && rc == FBPT_OK; ++i) {
        oi[i].stream = st;
        rc = run_setup(runs[i], gs[i], seeds[i], first_ids[i], Ss[i], &oi[i], &outs[i], wb[i]);
        runs[i].H = &Hs[i];
        for (uint32_t j = 0; j < i && rc == FBPT_OK; ++j)
            if (gs[j] == gs[i] && (runs[j].WB != runs[i].WB || runs[j].dense != runs[i].dense))
                rc = fail(FBPT_EINVAL, "fbpt_sample_batched: tasks on one graph need one workspace shape");
    }
    if (rc == FBPT_OK) cudaEventRecord(ev.a, st);
    for (uint32_t i = 0; i < G && rc == FBPT_OK; ++i) rc = run_arm(runs[i]);
    // one graph: a branch per task; tasks on one graph chained in order
    if (rc == FBPT_OK && cudaGraphCreate(&graph, 0) != cudaSuccess) rc = fail(FBPT_ECUDA, "cudaGraphCreate failed");
    std::vector<cudaGraphNode_t> tails(G);
    for (uint32_t i = 0; i < G && rc == FBPT_OK; ++i) {
        const cudaGraphNode_t* dep = nullptr;
        for (uint32_t j = i; j-- > 0;)
            if (gs[j] == gs[i]) {
                dep = &tails[j];
                break;
            }
        rc = add_task(graph, dep, runs[i], &tails[i]);
    }
    if (rc == FBPT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess)
        rc = fail(FBPT_ECUDA, "cudaGraphInstantiate failed");
    if (rc == FBPT_OK && cudaGraphLaunch(exec, st) != cudaSuccess) rc = fail(FBPT_ECUDA, "cudaGraphLaunch failed");
    if (rc == FBPT_OK && cudaStreamSynchronize(st) != cudaSuccess)
        rc = fail(FBPT_ECUDA, std::string("batched run: ") + cudaGetErrorString(cudaGetLastError()));
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    // outcomes in task order; a task that failed on the device leaves its
    // graph's workspace dirty, so later tasks on that graph run again too
    std::vector<fbpt_graph*> dirty;
    for (uint32_t i = 0; i < G && rc == FBPT_OK; ++i) {
        Run& r = runs[i];
        bool again = false;
        if (std::find(dirty.begin(), dirty.end(), gs[i]) != dirty.end()) {
            again = true;
        } else {
            rc = run_check(r, stats, again);
            if (rc == FBPT_OK && again && r.H->error) dirty.push_back(gs[i]);
        }
        if (rc == FBPT_OK && again) rc = run_attempts(r, stats);
    }
    for (uint32_t i = 0; i < G && rc == FBPT_OK; ++i) rc = run_finish(runs[i], stats);
    if (rc != FBPT_OK) {
        for (uint32_t i = 0; i < G; ++i) {
            runs[i].out = &outs[i];
            run_release(runs[i], true);
        }
        cudaStreamSynchronize(st);
        cudaFreeHost(Hs);
        return rc;
    }
    cudaEventRecord(ev.b, st);
    const float ms = elapsed_ms(ev.a, ev.b);
    if (stats) stats->ms_total += ms;
    cudaFreeHost(Hs);
    return FBPT_OK;
}

// The policy network's row-width choice: one probe at the reference shape
// (8 words x 1 slot, lane refill, the learned schedule) records the network's
// outputs 5..7 on every level (predicted log2 ns per sample at row widths of
// 4, 16 and 64 words); their means over the probe's levels rank the widths.
int policy_width_impl(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, uint32_t* row_words,
                      float* scores) {
    if (!g || !base || !row_words) return fail(FBPT_EINVAL, "fbpt_policy_width: null argument");
    if (!base->policy) return fail(FBPT_EINVAL, "fbpt_policy_width: needs a policy");
    if (S == 0) return fail(FBPT_EINVAL, "fbpt_policy_width: S must be >= 1");
    fbpt_opts q = *base;
    q.schedule = FBPT_SCHED_LEARNED;
    q.words = 8;
    q.slots = 1;
    q.refill = FBPT_REFILL_LANE;
    q.unfused = 0;
    q.blocks = 0;
    if (q.launch == FBPT_LAUNCH_PERSISTENT) q.launch = FBPT_LAUNCH_GRAPH;
    const uint64_t P = std::min<uint64_t>(S, 8192);
    std::vector<fbpt_trace_row> rows(1u << 16);
    q.trace = rows.data();
    q.trace_cap = rows.size();
    fbpt_rrsets rr;
    fbpt_stats st = {};
    FBPT_TRY(sample_impl(g, seed, 0, P, &q, &rr, &st));
    release_out(&rr);
    double sum[kPolicyWidthCount] = {};
    uint64_t cnt = 0;
    for (uint64_t r = 1; r < st.trace_rows; ++r) {
        if (rows[r].units == 0) continue;
        for (uint32_t k = 0; k < kPolicyWidthCount; ++k) sum[k] += rows[r].outputs[kPolicyWidthOut + k];
        ++cnt;
    }
    uint32_t best = kPolicyWidthCount - 1;  // no level with a frontier: the widest row
    if (cnt) {
        best = 0;
        for (uint32_t k = 1; k < kPolicyWidthCount; ++k)
            if (sum[k] < sum[best]) best = k;
    }
    *row_words = kPolicyWidths[best];
    if (scores)
        for (uint32_t k = 0; k < kPolicyWidthCount; ++k) scores[k] = cnt ? (float)(sum[k] / (double)cnt) : 0.f;
    return FBPT_OK;
}

int autotune_impl(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, fbpt_tuning* out) {
    if (!g) return fail(FBPT_EINVAL, "fbpt_autotune: null graph");
    if (S == 0) return fail(FBPT_EINVAL, "fbpt_autotune: S must be >= 1");
    fbpt_opts o = {};
    if (base) o = *base;
    o.trace = nullptr;
    o.trace_cap = 0;
    o.unfused = 0;
    if (o.launch == FBPT_LAUNCH_PERSISTENT) o.launch = FBPT_LAUNCH_GRAPH;
    // probe size: about kProbeMs of sampling per probe, measured on a first
    // run of 4,096 samples, within [4,096, 65,536] samples (and at most S)
    constexpr double kProbeMs = 50.0;
    const uint64_t P0 = std::min<uint64_t>(S, 4096);
    uint64_t P = P0;
    {
        fbpt_opts q = o;
        q.words = 8;
        q.slots = 1;
        q.refill = FBPT_REFILL_LANE;
        q.blocks = 0;
        if (q.schedule == FBPT_SCHED_PULL) q.schedule = FBPT_SCHED_HEURISTIC;
        fbpt_rrsets rr;
        fbpt_stats s0 = {};
        for (int rep = 0; rep < 2; ++rep) {
            s0 = fbpt_stats{};
            FBPT_TRY(sample_impl(g, seed, 0, P0, &q, &rr, &s0));
            release_out(&rr);
        }
        if (s0.ms_total > 0)
            P = std::max<uint64_t>(P0, std::min<uint64_t>(std::min<uint64_t>(S, 65536),
                                                          (uint64_t)((double)P0 * kProbeMs / s0.ms_total)));
    }
    const uint64_t warm = std::max<uint64_t>(P / 8, std::min<uint64_t>(P, 64));
    fbpt_tuning t = {};
    t.probe_samples = P;
    double rr_sum = 0;
    uint64_t rr_n = 0;
    // samples per second of one shape (a warm-up run on `warm` samples first)
    auto probe = [&](uint32_t WB, uint32_t blocks, double& rate, uint32_t sched) -> int {
        fbpt_opts q = o;
        q.schedule = sched;
        q.words = std::min<uint32_t>(WB, 8);
        q.slots = WB / q.words;
        q.refill = FBPT_REFILL_LANE;
        q.blocks = blocks;
        if (q.schedule == FBPT_SCHED_PULL && WB > kPullMaxWords) q.schedule = FBPT_SCHED_HEURISTIC;
        fbpt_rrsets rr;
        fbpt_stats s0 = {}, s1 = {};
        FBPT_TRY(sample_impl(g, seed, 0, warm, &q, &rr, &s0));
        release_out(&rr);
        FBPT_TRY(sample_impl(g, seed, 0, P, &q, &rr, &s1));
        release_out(&rr);
        rate = s1.ms_total > 0 ? (double)P / (1e-3 * s1.ms_total) : 0.0;
        rr_sum += (double)s1.rr_total;
        rr_n += P;
        t.candidates += 1;
        return FBPT_OK;
    };
    // a row width given in base (words * slots) caps the widths tried
    const uint32_t max_wb = (base && base->words) ? base->words * (base->slots ? base->slots : 1) : kMaxWords;
    uint32_t best_wb = 1;
    double best = -1;
    for (uint32_t WB = 1; WB <= std::min(max_wb, kMaxWords); WB *= 2) {
        if (WB > 1 && 64ull * WB > P) break;
        double rate = 0;
        FBPT_TRY(probe(WB, 0, rate, o.schedule));
        if (rate > best) {
            best = rate;
            best_wb = WB;
        }
    }
    // a smaller grid is kept only if it is more than 3% faster than the best so
    // far: the probe runs few samples, whose small frontiers favour small grids
    // more than a full-size run's do
    const int full = launch_shape().level_blocks;
    uint32_t best_blocks = (uint32_t)full;
    double best_rate = best;
    for (int div = 2; div <= 8; div *= 2) {
        const uint32_t blocks = (uint32_t)std::max(1, full / div);
        double rate = 0;
        FBPT_TRY(probe(best_wb, blocks, rate, o.schedule));
        if (rate > 1.03 * best_rate) {
            best_blocks = blocks;
            best_rate = rate;
        }
    }
    // the learned schedule is judged against the degree-ratio heuristic and
    // plain push on this graph: another one is kept only if it is at least 3%
    // faster at the chosen shape
    uint32_t best_sched = o.schedule;
    if (o.schedule == FBPT_SCHED_LEARNED || o.schedule == FBPT_SCHED_HEURISTIC) {
        const uint32_t other = o.schedule == FBPT_SCHED_LEARNED ? (uint32_t)FBPT_SCHED_HEURISTIC
                                                                : (uint32_t)FBPT_SCHED_LEARNED;
        if (other != FBPT_SCHED_LEARNED || o.policy) {
            double rate = 0;
            FBPT_TRY(probe(best_wb, best_blocks, rate, other));
            if (rate > 1.03 * best_rate) {
                best_rate = rate;
                best_sched = other;
            }
        }
        // plain push (no second expand kernel per level) is kept whenever it is
        // within 3% of the best
        double rate = 0;
        FBPT_TRY(probe(best_wb, best_blocks, rate, FBPT_SCHED_PUSH));
        if (rate >= 0.97 * best_rate) {
            best_rate = std::max(best_rate, rate);
            best_sched = FBPT_SCHED_PUSH;
        }
    }
    t.words = std::min<uint32_t>(best_wb, 8);
    t.slots = best_wb / t.words;
    t.refill = FBPT_REFILL_LANE;
    t.blocks = best_blocks;
    t.schedule = best_sched;
    t.probe_rate = best_rate;
    t.rr_per_sample = rr_n ? rr_sum / (double)rr_n : 0.0;
    g->tuned = t;
    g->tuned_valid = true;
    if (t.rr_per_sample > 0) g->rr_hint = t.rr_per_sample;
    if (out) *out = t;
    return FBPT_OK;
}

}  // namespace fbpt
