// The fused-BPT sampling engine (Section 3, Listing 1; Section 9 future-work
// items (a) and (b)).
//
// Colours.  A vertex row holds WB = B * W 64-bit words.  Word i belongs to
// slot k = i / W; a slot traverses one batch of 64*W consecutive samples, and
// colour c of the slot is sample slot_base[k] + c.  All slots share one
// frontier: a frontier unit is a vertex with the non-zero words of its new
// colour mask, so the in-edges of a vertex are read once per level for every
// colour of every slot that reached it (Listing 1's "fusing" line, widened
// across batches).  When a slot's colours are all finished, its RR sets are
// dumped and the slot takes the next batch without stopping the others
// (mid-traversal refill).
//
// One level ("tick") is five kernels, all launched with fixed grids so that a
// CUDA graph can loop them on the device:
//   expand   frontier units x 4-edge groups -> next masks, pending vertices
//   commit   pending vertices -> visited, new frontier list, touched lists
//   schedule (1 CTA) finished slots, refills, loop condition
//   dump     RR pairs (sample, vertex) of finished slots; clears their state
//   init     start vertices of newly assigned batches
//
// Liveness never reads visited[]: the expand draws for every colour of the
// frontier mask and the commit removes colours a vertex has already seen.
// The result is the same closure (each colour reaches each vertex once), and
// the hot loop streams col/thr with 128-bit loads instead of gathering masks.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace fbpt {
namespace {

constexpr int kExpThreads = 256;
constexpr int kComThreads = 256;
constexpr int kAuxThreads = 256;

__device__ __forceinline__ uint64_t row_groups(uint64_t rs, uint64_t re) {
    return re > rs ? ((re - 1) >> 2) - (rs >> 2) + 1 : 0;
}

// Bit k set iff slot k has a non-zero word in occ (words k*W .. k*W+W-1).
__device__ __forceinline__ uint64_t slots_of(uint64_t occ, uint32_t W) {
    if (W == 1) return occ;
    const uint64_t wm = (1ull << W) - 1;
    uint64_t s = 0;
    for (uint32_t k = 0; occ; ++k, occ >>= W)
        if (occ & wm) s |= 1ull << k;
    return s;
}

__device__ __forceinline__ void mark_dirty(const Eng& E, uint32_t w) {
    const unsigned long long bit = 1ull << (w & 63);
    const unsigned long long old = atomicOr((unsigned long long*)&E.dirty[w >> 6], bit);
    if (!(old & bit)) {
        const uint32_t p = atomicAdd(&E.ctl->pend_count, 1u);
        if (p < E.pend_cap)
            E.pend_v[p] = w;
        else
            atomicOr(&E.ctl->error, (unsigned)kErrPendOverflow);
    }
}

// ---- expand (push over in-edges) -----------------------------------------------------

// One 4-edge group of frontier unit u: edges 4q .. 4q+3 of the in-row of v,
// with q = rs/4 + j.  For each colour of the unit one Philox call decides all
// four edges (Listing 1's per-colour liveness draw); live colours are ORed
// into next[w] (Listing 1's fusing update).
__device__ __forceinline__ void expand_group(const Eng& E, uint32_t u, uint64_t j, const uint64_t* s_wbase,
                                             uint64_t& n_edges, uint64_t& n_calls) {
    const uint32_t v = E.list_v[u];
    const uint64_t occ = E.list_occ[u];
    const uint32_t mrow = E.list_mrow[u];
    const uint32_t only = E.unfused ? E.list_only[u] : 0u;
    const uint64_t rs = E.row_ptr[v], re = E.row_ptr[v + 1];
    const uint64_t q = (rs >> 2) + j;
    const uint64_t e0 = q << 2;
    const uint4 c4 = __ldg(reinterpret_cast<const uint4*>(E.col) + q);
    uint4 t4 = __ldg(reinterpret_cast<const uint4*>(E.thr) + q);
    if (e0 + 0 < rs || e0 + 0 >= re) t4.x = 0;
    if (e0 + 1 < rs || e0 + 1 >= re) t4.y = 0;
    if (e0 + 2 < rs || e0 + 2 >= re) t4.z = 0;
    if (e0 + 3 < rs || e0 + 3 >= re) t4.w = 0;
    n_edges += (uint64_t)min(re, e0 + 4) - (uint64_t)max(rs, e0);
    if ((t4.x | t4.y | t4.z | t4.w) == 0) return;
    // A draw is needed only for edges with 0 < thr < 0xFFFFFFFF.
    const bool need = (t4.x - 1u < 0xFFFFFFFEu) || (t4.y - 1u < 0xFFFFFFFEu) || (t4.z - 1u < 0xFFFFFFFEu) ||
                      (t4.w - 1u < 0xFFFFFFFEu);
    bool a0 = false, a1 = false, a2 = false, a3 = false;
    uint64_t words = occ;
    while (words) {
        const uint32_t i = __ffsll((long long)words) - 1;
        words &= words - 1;
        const uint64_t x = only ? (1ull << ((only - 1u) & 63u)) : E.stage[(uint64_t)mrow * E.WB + i];
        uint64_t y0, y1, y2, y3;
        if (need) {
            y0 = y1 = y2 = y3 = 0;
            const uint64_t sb = s_wbase[i];
            uint64_t xx = x;
            while (xx) {
                const uint32_t c = __ffsll((long long)xx) - 1;
                xx &= xx - 1;
                const uint4 r = edge_draws4(E.seed, sb + c, q);
                ++n_calls;
                const uint64_t bit = 1ull << c;
                if (live(r.x, t4.x)) y0 |= bit;
                if (live(r.y, t4.y)) y1 |= bit;
                if (live(r.z, t4.z)) y2 |= bit;
                if (live(r.w, t4.w)) y3 |= bit;
            }
        } else {
            y0 = t4.x ? x : 0;
            y1 = t4.y ? x : 0;
            y2 = t4.z ? x : 0;
            y3 = t4.w ? x : 0;
        }
        if (y0) { atomicOr((unsigned long long*)&E.next[(uint64_t)c4.x * E.WB + i], y0); a0 = true; }
        if (y1) { atomicOr((unsigned long long*)&E.next[(uint64_t)c4.y * E.WB + i], y1); a1 = true; }
        if (y2) { atomicOr((unsigned long long*)&E.next[(uint64_t)c4.z * E.WB + i], y2); a2 = true; }
        if (y3) { atomicOr((unsigned long long*)&E.next[(uint64_t)c4.w * E.WB + i], y3); a3 = true; }
    }
    if (a0) mark_dirty(E, c4.x);
    if (a1) mark_dirty(E, c4.y);
    if (a2) mark_dirty(E, c4.z);
    if (a3) mark_dirty(E, c4.w);
}

// Persistent, edge-balanced: CTAs take tiles of kTileGroups consecutive groups
// of the frontier's group space from an atomic counter; the unit of each group
// is found by binary search over the units' group offsets staged in shared
// memory.
__global__ void __launch_bounds__(kExpThreads) k_expand(const Eng E) {
    __shared__ uint64_t s_gb[kTileGroups + 1];
    __shared__ uint64_t s_wbase[kMaxWords];
    __shared__ uint32_t s_tile;
    Ctl* ctl = E.ctl;
    const uint64_t G = ctl->list_groups;
    if (G == 0) return;
    if (threadIdx.x == 0) atomicMin(&ctl->exp_t0, globaltimer_ns());
    const uint64_t U = ctl->list_count;
    for (uint32_t i = threadIdx.x; i < E.WB; i += blockDim.x)
        s_wbase[i] = ctl->slot_base[i / E.W] + 64ull * (i % E.W);
    const uint64_t ntiles = (G + kTileGroups - 1) / kTileGroups;
    if (ntiles > E.tile_cap || U > E.list_cap) return;  // overflow already flagged by commit
    uint64_t n_edges = 0, n_calls = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->tile_next, 1u);
        __syncthreads();
        const uint64_t t = s_tile;
        if (t >= ntiles) break;
        const uint64_t g0 = t * kTileGroups;
        const uint64_t g1 = min(g0 + kTileGroups, G);
        const uint32_t u0 = E.tile_u0[t];
        const uint32_t u1 = (t + 1 < ntiles) ? E.tile_u0[t + 1] : (uint32_t)(U - 1);
        const uint32_t nu = u1 - u0 + 1;
        for (uint32_t i = threadIdx.x; i < nu; i += blockDim.x) s_gb[i] = E.list_g[u0 + i];
        __syncthreads();
        for (uint64_t g = g0 + threadIdx.x; g < g1; g += blockDim.x) {
            uint32_t lo = 0, hi = nu;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_gb[mid] <= g) lo = mid; else hi = mid;
            }
            expand_group(E, u0 + lo, g - s_gb[lo], s_wbase, n_edges, n_calls);
        }
    }
    n_edges = warp_sum(n_edges);
    n_calls = warp_sum(n_calls);
    if (lane_id() == 0) {
        if (n_edges) atomicAdd(&ctl->st_edges, (unsigned long long)n_edges);
        if (n_calls) atomicAdd(&ctl->st_calls, (unsigned long long)n_calls);
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicMax(&ctl->exp_t1, globaltimer_ns());
}

// ---- commit -------------------------------------------------------------------------

__device__ __forceinline__ void write_unit(const Eng& E, uint64_t pos, uint32_t w, uint32_t mrow, uint64_t occ,
                                           uint32_t only, uint64_t gbeg, uint64_t ng) {
    E.list_v[pos] = w;
    E.list_mrow[pos] = mrow;
    E.list_occ[pos] = occ;
    E.list_g[pos] = gbeg;
    if (E.unfused) E.list_only[pos] = only;
    // tiles whose first group falls inside this unit start their search here
    const uint64_t end = gbeg + ng;
    for (uint64_t t = (gbeg + kTileGroups - 1) / kTileGroups; t * kTileGroups < end; ++t) {
        if (t < E.tile_cap) E.tile_u0[t] = (uint32_t)pos;
        else atomicOr(&E.ctl->error, (unsigned)kErrTileOverflow);
    }
}

// For every pending vertex w: nx = next[w] & ~visited[w]; next[w] = 0;
// visited[w] |= nx.  Non-empty nx becomes a frontier unit (if w has in-edges);
// the first colour of a slot to reach w appends w to that slot's touched list.
__global__ void __launch_bounds__(kComThreads) k_commit(const Eng E) {
    Ctl* ctl = E.ctl;
    const uint32_t P = (uint32_t)min((uint64_t)ctl->pend_count, E.pend_cap);
    const uint32_t lane = lane_id();
    uint64_t mwords = 0;
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    uint64_t active = 0;
    for (uint64_t base = wid * 32; base < P; base += nwarp * 32) {
        const uint64_t idx = base + lane;
        const bool ok = idx < P;
        uint32_t w = 0, bits = 0;
        uint64_t occ = 0, rs = 0, re = 0;
        if (ok) {
            w = E.pend_v[idx];
            E.dirty[w >> 6] = 0ull;  // every dirty bit of this word belongs to a pending vertex
            const uint64_t rowb = (uint64_t)w * E.WB;
            for (uint32_t i = 0; i < E.WB; ++i) {
                uint64_t nx = E.next[rowb + i];
                if (!nx) continue;
                E.next[rowb + i] = 0;
                const uint64_t vis = E.visited[rowb + i];
                nx &= ~vis;
                if (!nx) continue;
                E.visited[rowb + i] = vis | nx;
                E.stage[idx * E.WB + i] = nx;
                occ |= 1ull << i;
                bits += __popcll(nx);
            }
            uint64_t so = slots_of(occ, E.W);
            const uint64_t bit = 1ull << (w & 63);
            while (so) {
                const uint32_t k = __ffsll((long long)so) - 1;
                so &= so - 1;
                const unsigned long long old = atomicOr((unsigned long long*)&E.touched[k * E.nw + (w >> 6)], bit);
                if (!(old & bit)) {
                    const uint32_t t = atomicAdd(&ctl->tcount[k], 1u);
                    E.tlist[(uint64_t)k * E.n + t] = w;
                }
            }
            if (occ) {
                rs = E.row_ptr[w];
                re = E.row_ptr[w + 1];
            }
        }
        const uint64_t ng = row_groups(rs, re);
        const uint64_t units = ng ? (E.unfused ? bits : 1u) : 0u;
        if (units) active |= slots_of(occ, E.W);
        mwords += units ? (E.unfused ? units : (uint64_t)__popcll(occ)) : 0;
        const unsigned long long req = (unsigned long long)((units * ng) << kUnitBits) | units;
        const unsigned long long got = warp_alloc<unsigned long long>(&ctl->new_packed, req);
        if (units) {
            uint64_t pos = got & kUnitMask;
            uint64_t gbeg = got >> kUnitBits;
            if (pos + units > E.list_cap) {
                atomicOr(&ctl->error, (unsigned)kErrListOverflow);
            } else if (!E.unfused) {
                write_unit(E, pos, w, (uint32_t)idx, occ, 0u, gbeg, ng);
            } else {
                uint64_t ws = occ;
                while (ws) {
                    const uint32_t i = __ffsll((long long)ws) - 1;
                    ws &= ws - 1;
                    uint64_t x = E.stage[idx * E.WB + i];
                    while (x) {
                        const uint32_t c = __ffsll((long long)x) - 1;
                        x &= x - 1;
                        write_unit(E, pos++, w, (uint32_t)idx, 1ull << i, i * 64u + c + 1u, gbeg, ng);
                        gbeg += ng;
                    }
                }
            }
        }
    }
    active = warp_or64(active);
    mwords = warp_sum(mwords);
    if (lane == 0 && active) atomicOr(&ctl->active_mask, (unsigned long long)active);
    if (lane == 0 && mwords) atomicAdd(&ctl->st_mask_words, (unsigned long long)mwords);
}

// ---- schedule (one CTA of kMaxSlots threads) ---------------------------------------------

__global__ void k_schedule(const Eng E) {
    Ctl* ctl = E.ctl;
    __shared__ uint32_t s_fin, s_init, s_run;
    if (threadIdx.x == 0) { s_fin = 0; s_init = 0; s_run = 0; }
    __syncthreads();
    const uint64_t act = ctl->active_mask;
    const uint32_t k = threadIdx.x;
    if (k < E.B) {
        uint32_t st = ctl->slot_state[k];
        if (st == kSlotRunning && !((act >> k) & 1ull)) {
            const uint32_t f = atomicAdd(&s_fin, 1u);
            ctl->fin_slot[f] = k;
            ctl->fin_base[f] = ctl->slot_base[k];
            ctl->fin_ncol[f] = ctl->slot_ncol[k];
            st = kSlotIdle;
        }
        if (st == kSlotIdle && ctl->error == 0) {
            const unsigned long long b = atomicAdd(&ctl->next_batch, 1ull);
            if (b < ctl->nbatches) {
                const uint64_t colours = 64ull * E.W;
                const uint64_t s0 = b * colours;
                ctl->slot_base[k] = E.first_id + s0;
                ctl->slot_ncol[k] = (uint32_t)min(colours, E.S - s0);
                ctl->init_slot[atomicAdd(&s_init, 1u)] = k;
                st = kSlotRunning;
            }
        }
        ctl->slot_state[k] = st;
        if (st == kSlotRunning) atomicOr(&s_run, 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ctl->fin_count = s_fin;
        ctl->init_count = s_init;
        ctl->st_batches += s_init;
        const unsigned long long np = ctl->new_packed;
        ctl->list_count = np & kUnitMask;
        ctl->list_groups = np >> kUnitBits;
        if (ctl->error) {  // a capacity check tripped: expand nothing more
            ctl->list_count = 0;
            ctl->list_groups = 0;
        }
        ctl->st_units += np & kUnitMask;
        if ((np >> kUnitBits) != 0) ctl->st_push += 1;
        if (ctl->exp_t1 > ctl->exp_t0) ctl->st_expand_ns += ctl->exp_t1 - ctl->exp_t0;
        ctl->exp_t0 = ~0ull;
        ctl->exp_t1 = 0;
        ctl->new_packed = 0;
        ctl->tile_next = 0;
        ctl->pend_count = 0;
        ctl->active_mask = 0;
        ctl->tick += 1;
        uint32_t run = s_run;
        if (ctl->tick > ctl->tick_limit) {
            ctl->error |= kErrTickLimit;
        }
        if (ctl->error) run = 0;
        ctl->running = run;
        if (E.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)E.cond, run);
    }
}

// ---- dump: RR pairs of finished slots (Listing 1's RRR-set construction) -------------------

__global__ void __launch_bounds__(kAuxThreads) k_dump(const Eng E) {
    Ctl* ctl = E.ctl;
    const uint32_t F = ctl->fin_count;
    if (F == 0) return;
    __shared__ uint64_t s_pre[kMaxSlots + 1];
    __shared__ uint32_t s_slot[kMaxSlots];
    __shared__ uint64_t s_base[kMaxSlots];
    if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (uint32_t f = 0; f < F; ++f) {
            s_slot[f] = ctl->fin_slot[f];
            s_base[f] = ctl->fin_base[f] - E.first_id;
            s_pre[f + 1] = s_pre[f] + ctl->tcount[s_slot[f]];
        }
    }
    __syncthreads();
    const uint64_t total = s_pre[F];
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t cap = ctl->pair_cap;
    uint64_t cev = 0;
    for (uint64_t base = wid * 32; base < total; base += nwarp * 32) {
        const uint64_t idx = base + lane;
        const bool ok = idx < total;
        uint64_t x[8];
        uint32_t cnt = 0, v = 0, f = 0;
        if (ok) {
            while (s_pre[f + 1] <= idx) ++f;
            const uint32_t k = s_slot[f];
            v = E.tlist[(uint64_t)k * E.n + (idx - s_pre[f])];
            const uint64_t rowb = (uint64_t)v * E.WB + (uint64_t)k * E.W;
#pragma unroll
            for (uint32_t w = 0; w < 8; ++w) {
                x[w] = 0;
                if (w < E.W) {
                    x[w] = E.visited[rowb + w];
                    E.visited[rowb + w] = 0;
                    cnt += __popcll(x[w]);
                }
            }
            E.touched[(uint64_t)k * E.nw + (v >> 6)] = 0ull;  // all its bits are in this dump
            atomicAdd(&E.vcount[v], cnt);
            cev += (uint64_t)cnt * (E.row_ptr[v + 1] - E.row_ptr[v]);
        }
        uint64_t pos = warp_alloc<unsigned long long>(&ctl->pair_cursor, (unsigned long long)cnt);
        if (ok && pos + cnt <= cap) {
            const uint64_t jb = s_base[f];
#pragma unroll
            for (uint32_t w = 0; w < 8; ++w) {
                uint64_t xx = x[w];
                while (xx) {
                    const uint32_t c = __ffsll((long long)xx) - 1;
                    xx &= xx - 1;
                    E.pairs[pos++] = ((jb + 64ull * w + c) << E.vbits) | v;
                }
            }
        }
    }
    cev = warp_sum(cev);
    if (lane == 0 && cev) atomicAdd(&ctl->st_cev, (unsigned long long)cev);
}

// ---- init: start vertices of newly assigned batches (Listing 1's frontier initialization) --------

__global__ void __launch_bounds__(kAuxThreads) k_init(const Eng E) {
    Ctl* ctl = E.ctl;
    const uint32_t I = ctl->init_count;
    const uint32_t F = ctl->fin_count;
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (gt < F) ctl->tcount[ctl->fin_slot[gt]] = 0;
    const uint64_t colours = 64ull * E.W;
    const uint64_t total = (uint64_t)I * colours;
    for (uint64_t idx = gt; idx < total; idx += stride) {
        const uint32_t k = ctl->init_slot[idx / colours];
        const uint32_t c = (uint32_t)(idx % colours);
        if (c >= ctl->slot_ncol[k]) continue;
        const uint64_t s = ctl->slot_base[k] + c;
        const uint32_t v = start_vertex(E.seed, s, E.n);
        E.starts[s - E.first_id] = v;
        atomicOr((unsigned long long*)&E.next[(uint64_t)v * E.WB + (uint64_t)k * E.W + (c >> 6)], 1ull << (c & 63));
        mark_dirty(E, v);
    }
}

// ---- finalize: sorted pairs -> CSR --------------------------------------------------------

__global__ void k_finalize(const uint64_t* keys, uint64_t total, uint32_t vbits, uint64_t S, uint64_t* offsets,
                           uint32_t* verts) {
    const uint64_t vmask = (1ull << vbits) - 1;
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
        const uint64_t j = key >> vbits;
        verts[p] = (uint32_t)(key & vmask);
        if (p == 0 || (keys[p - 1] >> vbits) != j) offsets[j] = p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) offsets[S] = total;
}

struct LaunchShape {
    int expand_blocks = 0, commit_blocks = 0, aux_blocks = 0;
};

LaunchShape launch_shape() {
    static LaunchShape ls;
    static bool done = false;
    if (!done) {
        const int sms = device_sm_count();
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_expand, kExpThreads, 0);
        ls.expand_blocks = sms * std::max(per, 1);
        ls.commit_blocks = sms * 4;
        ls.aux_blocks = sms * 2;
        done = true;
    }
    return ls;
}

int launch_tick(const Eng& E, cudaStream_t st) {
    const LaunchShape ls = launch_shape();
    k_expand<<<ls.expand_blocks, kExpThreads, 0, st>>>(E);
    k_commit<<<ls.commit_blocks, kComThreads, 0, st>>>(E);
    k_schedule<<<1, kMaxSlots, 0, st>>>(E);
    k_dump<<<ls.aux_blocks, kAuxThreads, 0, st>>>(E);
    k_init<<<ls.aux_blocks, kAuxThreads, 0, st>>>(E);
    FBPT_CUDA_TRY(cudaGetLastError());
    return FBPT_OK;
}

// The whole run as one CUDA graph: a WHILE conditional node whose body is one
// tick; k_schedule sets the condition.
int run_graph(Eng E, cudaStream_t st) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    FBPT_CUDA_TRY(cudaGraphCreate(&graph, 0));
    int rc = FBPT_OK;
    do {
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, "cudaGraphConditionalHandleCreate failed");
            break;
        }
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, "cudaGraphAddNode(conditional) failed");
            break;
        }
        cudaGraph_t body = p.conditional.phGraph_out[0];
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, "stream create failed");
            break;
        }
        E.cond = (unsigned long long)h;
        if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) !=
            cudaSuccess) {
            cudaStreamDestroy(cs);
            rc = fail(FBPT_ECUDA, "cudaStreamBeginCaptureToGraph failed");
            break;
        }
        int lrc = launch_tick(E, cs);
        cudaGraph_t captured = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cs, &captured);
        cudaStreamDestroy(cs);
        if (lrc != FBPT_OK) { rc = lrc; break; }
        if (ce != cudaSuccess) { rc = fail(FBPT_ECUDA, std::string("capture failed: ") + cudaGetErrorString(ce)); break; }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, "cudaGraphInstantiate failed");
            break;
        }
        if (cudaGraphLaunch(exec, st) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, "cudaGraphLaunch failed");
            break;
        }
    } while (0);
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
    cudaFree(w->visited); cudaFree(w->next); cudaFree(w->stage); cudaFree(w->dirty); cudaFree(w->touched);
    cudaFree(w->tlist); cudaFree(w->pend_v); cudaFree(w->list_v); cudaFree(w->list_mrow); cudaFree(w->list_only);
    cudaFree(w->list_g); cudaFree(w->list_occ); cudaFree(w->tile_u0); cudaFree(w->ctl);
    if (w->ctl_host) cudaFreeHost(w->ctl_host);
    delete w;
}

int ws_get(fbpt_graph* g, uint32_t W, uint32_t B, bool unfused, cudaStream_t st, Workspace** out) {
    Workspace* w = g->ws;
    if (w && w->W == W && w->B == B && w->unfused == unfused) {
        if (!w->clean) {
            const uint64_t rows = (uint64_t)g->n * w->WB;
            FBPT_CUDA_TRY(cudaMemsetAsync(w->visited, 0, rows * 8, st));
            FBPT_CUDA_TRY(cudaMemsetAsync(w->next, 0, rows * 8, st));
            FBPT_CUDA_TRY(cudaMemsetAsync(w->dirty, 0, w->nw * 8, st));
            FBPT_CUDA_TRY(cudaMemsetAsync(w->touched, 0, (uint64_t)B * w->nw * 8, st));
            w->clean = true;
        }
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
    w->W = W;
    w->B = B;
    w->WB = W * B;
    w->unfused = unfused;
    w->nw = (g->n + 63) / 64;
    const uint64_t n = g->n;
    const uint64_t rows = n * w->WB;
    w->pend_cap = n;
    w->list_cap = unfused ? std::min<uint64_t>(n * (uint64_t)w->WB * 64, std::max<uint64_t>(16 * n, 1 << 20)) : n;
    if (w->list_cap > kUnitMask) w->list_cap = kUnitMask;
    // groups of a row [rs, re) are at most (re - rs) / 4 + 2
    const uint64_t max_groups = (g->m / 4 + 2 * n + 1) * (unfused ? 64ull * w->WB : 1ull);
    w->tile_cap = std::min<uint64_t>(max_groups / kTileGroups + 2, (uint64_t)1 << 32);
    int rc = FBPT_OK;
    size_t& b = w->bytes;
    if (rc == FBPT_OK) rc = dalloc(&w->visited, rows, b);
    if (rc == FBPT_OK) rc = dalloc(&w->next, rows, b);
    if (rc == FBPT_OK) rc = dalloc(&w->stage, w->pend_cap * w->WB, b);
    if (rc == FBPT_OK) rc = dalloc(&w->dirty, w->nw, b);
    if (rc == FBPT_OK) rc = dalloc(&w->touched, (uint64_t)B * w->nw, b);
    if (rc == FBPT_OK) rc = dalloc(&w->tlist, (uint64_t)B * n, b);
    if (rc == FBPT_OK) rc = dalloc(&w->pend_v, w->pend_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_v, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_mrow, w->list_cap, b);
    if (rc == FBPT_OK && unfused) rc = dalloc(&w->list_only, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_g, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->list_occ, w->list_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->tile_u0, w->tile_cap, b);
    if (rc == FBPT_OK) rc = dalloc(&w->ctl, 1, b);
    if (rc == FBPT_OK && cudaMallocHost((void**)&w->ctl_host, sizeof(Ctl)) != cudaSuccess)
        rc = fail(FBPT_ENOMEM, "cudaMallocHost(ctl) failed");
    if (rc != FBPT_OK) {
        ws_free(w);
        return rc;
    }
    FBPT_CUDA_TRY(cudaMemsetAsync(w->visited, 0, rows * 8, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(w->next, 0, rows * 8, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(w->dirty, 0, w->nw * 8, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(w->touched, 0, (uint64_t)B * w->nw * 8, st));
    w->clean = true;
    g->ws = w;
    *out = w;
    return FBPT_OK;
}

uint32_t bits_for(uint64_t x) {  // bits to hold values 0 .. x
    uint32_t b = 1;
    while (b < 64 && (x >> b) != 0) ++b;
    return b;
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
    if (!g || !out) return fail(FBPT_EINVAL, "fbpt_sample: null graph or output");
    if (S == 0 || S > 0xFFFFFFFFull) return fail(FBPT_EINVAL, "fbpt_sample: S must be in [1, 2^32)");
    if (first_id + S < first_id) return fail(FBPT_EINVAL, "fbpt_sample: sample ids overflow");
    fbpt_opts o = {};
    if (opts) o = *opts;
    uint32_t W = o.words ? o.words : 8;
    if (W != 1 && W != 2 && W != 4 && W != 8) return fail(FBPT_EINVAL, "fbpt_sample: words must be 1, 2, 4 or 8");
    uint32_t B = o.slots ? o.slots : kMaxWords / W;
    if (B < 1 || B * W > kMaxWords) return fail(FBPT_EINVAL, "fbpt_sample: words * slots must be <= 64");
    const uint64_t nbatches = (S + 64ull * W - 1) / (64ull * W);
    if (B > nbatches) B = (uint32_t)nbatches;
    if (o.schedule != FBPT_SCHED_PUSH && o.schedule != FBPT_SCHED_HEURISTIC && o.schedule != FBPT_SCHED_LEARNED)
        return fail(FBPT_EUNSUPPORTED, "fbpt_sample: schedule not available");
    if (o.launch != FBPT_LAUNCH_HOST && o.launch != FBPT_LAUNCH_GRAPH)
        return fail(FBPT_EINVAL, "fbpt_sample: bad launch mode");
    cudaStream_t st = o.stream ? (cudaStream_t)o.stream : g->stream;
    const uint32_t vbits = bits_for(g->n - 1);
    const uint32_t sbits = bits_for(S - 1);
    if (vbits + sbits > 64) return fail(FBPT_EUNSUPPORTED, "fbpt_sample: sample x vertex keys exceed 64 bits");

    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, st);

    Workspace* ws = nullptr;
    FBPT_TRY(ws_get(g, W, B, o.unfused != 0, st, &ws));

    std::memset(out, 0, sizeof(*out));
    out->S = S;
    out->n = g->n;
    out->stream = st;
    FBPT_CUDA_TRY(cudaMallocAsync(&out->starts, sizeof(uint32_t) * S, st));
    FBPT_CUDA_TRY(cudaMallocAsync(&out->vcount, sizeof(uint32_t) * g->n, st));
    FBPT_CUDA_TRY(cudaMallocAsync(&out->offsets, sizeof(uint64_t) * (S + 1), st));

    uint64_t cap = (uint64_t)(g->rr_hint * 1.25 * (double)S) + 4096;
    uint64_t* pairs = nullptr;
    Ctl* H = ws->ctl_host;
    int rc = FBPT_OK;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if (pairs) cudaFreeAsync(pairs, st);
        FBPT_CUDA_TRY(cudaMallocAsync(&pairs, sizeof(uint64_t) * cap, st));
        FBPT_CUDA_TRY(cudaMemsetAsync(out->vcount, 0, sizeof(uint32_t) * g->n, st));
        std::memset(H, 0, sizeof(Ctl));
        H->nbatches = nbatches;
        H->pair_cap = cap;
        H->exp_t0 = ~0ull;
        const uint64_t rounds = nbatches / B + 2;
        H->tick_limit = std::min<uint64_t>(rounds * ((uint64_t)g->n + 2), 1ull << 40);
        FBPT_CUDA_TRY(cudaMemcpyAsync(ws->ctl, H, sizeof(Ctl), cudaMemcpyHostToDevice, st));

        Eng E = {};
        E.n = g->n; E.W = W; E.B = B; E.WB = W * B; E.nw = ws->nw;
        E.row_ptr = g->row_ptr; E.col = g->col; E.thr = g->thr;
        E.seed = seed; E.first_id = first_id; E.S = S;
        E.visited = ws->visited; E.next = ws->next; E.stage = ws->stage; E.dirty = ws->dirty;
        E.touched = ws->touched; E.tlist = ws->tlist; E.pend_v = ws->pend_v;
        E.list_v = ws->list_v; E.list_mrow = ws->list_mrow; E.list_only = ws->list_only;
        E.list_g = ws->list_g; E.list_occ = ws->list_occ; E.tile_u0 = ws->tile_u0;
        E.pend_cap = ws->pend_cap; E.list_cap = ws->list_cap; E.tile_cap = ws->tile_cap;
        E.unfused = o.unfused ? 1u : 0u;
        E.vbits = vbits;
        E.ctl = ws->ctl;
        E.starts = out->starts; E.vcount = out->vcount; E.pairs = pairs;
        E.cond = 0;
        ws->clean = false;
        if (o.launch == FBPT_LAUNCH_GRAPH) {
            rc = run_graph(E, st);
        } else {
            for (;;) {
                rc = launch_tick(E, st);
                if (rc != FBPT_OK) break;
                if (cudaMemcpyAsync(&H->running, &ws->ctl->running, sizeof(unsigned), cudaMemcpyDeviceToHost, st) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = fail(FBPT_ECUDA, std::string("level loop: ") + cudaGetErrorString(cudaGetLastError()));
                    break;
                }
                if (!H->running) break;
            }
        }
        if (rc != FBPT_OK) break;
        if (cudaMemcpyAsync(H, ws->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = fail(FBPT_ECUDA, std::string("sampling run: ") + cudaGetErrorString(cudaGetLastError()));
            break;
        }
        if (H->error) {
            rc = fail(FBPT_EDEVICE, "sampling run: device check failed (error bits " + std::to_string(H->error) + ")");
            break;
        }
        ws->clean = true;  // every slot finished: kernels restored the zero state
        if (H->pair_cursor <= cap) break;
        cap = H->pair_cursor + 1024;  // exact size is now known; run again
        if (stats) stats->overflow_reruns += nbatches;
    }
    if (rc != FBPT_OK) {
        if (pairs) cudaFreeAsync(pairs, st);
        return rc;
    }
    const uint64_t total = H->pair_cursor;
    if (total > cap) {
        cudaFreeAsync(pairs, st);
        return fail(FBPT_ENOMEM, "fbpt_sample: output did not fit after re-runs");
    }
    g->rr_hint = std::max(1.0, (double)total / (double)S);
    uint64_t* tmp = nullptr;
    rc = FBPT_OK;
    if (cudaMallocAsync(&tmp, sizeof(uint64_t) * std::max<uint64_t>(total, 1), st) != cudaSuccess)
        rc = fail(FBPT_ENOMEM, "fbpt_sample: sort buffer");
    if (rc == FBPT_OK) rc = radix_sort_u64(pairs, tmp, total, vbits + sbits, st);
    if (rc == FBPT_OK && cudaMallocAsync(&out->verts, sizeof(uint32_t) * std::max<uint64_t>(total, 1), st) != cudaSuccess)
        rc = fail(FBPT_ENOMEM, "fbpt_sample: verts");
    if (rc == FBPT_OK) {
        const int blocks = (int)std::min<uint64_t>((total + 255) / 256 + 1, (uint64_t)device_sm_count() * 8);
        k_finalize<<<blocks, 256, 0, st>>>(pairs, total, vbits, S, out->offsets, out->verts);
        if (cudaGetLastError() != cudaSuccess) rc = fail(FBPT_ECUDA, "finalize launch failed");
    }
    if (tmp) cudaFreeAsync(tmp, st);
    cudaFreeAsync(pairs, st);
    if (rc != FBPT_OK) return rc;
    out->total = total;
    cudaEventRecord(ev1, st);
    if (cudaEventSynchronize(ev1) != cudaSuccess)
        return fail(FBPT_ECUDA, std::string("fbpt_sample: ") + cudaGetErrorString(cudaGetLastError()));
    float ms = 0;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (stats) {
        stats->levels += H->tick;
        stats->batches += H->st_batches;
        stats->push_levels += H->st_push;
        stats->units_expanded += H->st_units;
        stats->edge_accesses += H->st_edges;
        stats->philox_calls += H->st_calls;
        stats->colour_edge_visits += H->st_cev;
        stats->rr_total += total;
        stats->mask_words += H->st_mask_words;
        stats->ms_total += ms;
        stats->ms_expand += 1e-6 * (double)H->st_expand_ns;
    }
    return FBPT_OK;
}

}  // namespace fbpt
