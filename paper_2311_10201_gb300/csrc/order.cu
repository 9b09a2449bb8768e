// Vertex orders (Section 5: relabelling the vertices so that vertices reached
// together lie together, and a sorted list of start vertices): reverse
// Cuthill-McKee, degree, random and Louvain clustering orders computed on the host, their
// application to a graph's device state, and the sorted start list of a
// sampling call.
//
// An order relabels what the sampler indexes by vertex (visited / next rows,
// the pending list, frontier units); the in-edges stay at their in-CSR
// positions, so the (sample id, edge index) counter of every liveness draw is
// unchanged and so is every result.  Only col is rewritten (to perm[col0]);
// each new label w reads its in-row [rstart[w], rend[w]) of the caller's CSR.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

namespace fbpt {
namespace {

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): the random order's stream.
uint64_t splitmix64(uint64_t& x) {
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

bool csr_ok(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col) {
    if (row_ptr[0] != 0 || row_ptr[n] != m) return false;
    for (uint32_t v = 0; v < n; ++v)
        if (row_ptr[v + 1] < row_ptr[v]) return false;
    for (uint64_t e = 0; e < m; ++e)
        if (col[e] >= n) return false;
    return true;
}

// Undirected simple graph of the CSR: u - v for every edge u -> v, u != v;
// each neighbour list sorted and without repeats.
void undirected(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, std::vector<uint64_t>& off,
                std::vector<uint32_t>& adj) {
    off.assign((size_t)n + 1, 0);
    for (uint32_t v = 0; v < n; ++v)
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (col[e] != v) {
                ++off[col[e] + 1];
                ++off[v + 1];
            }
    for (uint32_t v = 0; v < n; ++v) off[v + 1] += off[v];
    adj.resize(off[n]);
    std::vector<uint64_t> cur(off.begin(), off.end() - 1);
    for (uint32_t v = 0; v < n; ++v)
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            const uint32_t u = col[e];
            if (u == v) continue;
            adj[cur[u]++] = v;
            adj[cur[v]++] = u;
        }
    // sort and drop repeats, compacting the lists in place
    uint64_t w = 0;
    for (uint32_t v = 0; v < n; ++v) {
        const uint64_t a = off[v], b = off[v + 1];
        std::sort(adj.begin() + a, adj.begin() + b);
        const uint64_t start = w;
        for (uint64_t i = a; i < b; ++i)
            if (i == a || adj[i] != adj[i - 1]) adj[w++] = adj[i];
        off[v] = start;
    }
    off[n] = w;
    adj.resize(w);
}

// Reverse Cuthill-McKee: per component, breadth-first from the unvisited
// vertex of least degree (ties: least id), each vertex's unvisited neighbours
// appended by increasing (degree, id); perm = the reversed visit order.
void rcm(uint32_t n, const std::vector<uint64_t>& off, const std::vector<uint32_t>& adj, uint32_t* perm) {
    std::vector<uint32_t> deg(n);
    uint32_t dmax = 0;
    for (uint32_t v = 0; v < n; ++v) {
        deg[v] = (uint32_t)(off[v + 1] - off[v]);
        dmax = std::max(dmax, deg[v]);
    }
    // vertices by (degree, id): a counting sort, stable in id
    std::vector<uint32_t> by_deg(n), cnt((size_t)dmax + 2, 0);
    for (uint32_t v = 0; v < n; ++v) ++cnt[deg[v] + 1];
    for (uint32_t d = 0; d <= dmax; ++d) cnt[d + 1] += cnt[d];
    for (uint32_t v = 0; v < n; ++v) by_deg[cnt[deg[v]]++] = v;
    std::vector<char> seen(n, 0);
    std::vector<uint32_t> cm;
    cm.reserve(n);
    std::vector<uint32_t> nb;
    uint32_t next_start = 0;
    while (cm.size() < n) {
        while (seen[by_deg[next_start]]) ++next_start;
        const uint32_t s = by_deg[next_start];
        seen[s] = 1;
        cm.push_back(s);
        for (size_t head = cm.size() - 1; head < cm.size(); ++head) {
            const uint32_t x = cm[head];
            nb.clear();
            for (uint64_t i = off[x]; i < off[x + 1]; ++i) {
                const uint32_t y = adj[i];
                if (!seen[y]) {
                    seen[y] = 1;
                    nb.push_back(y);
                }
            }
            std::sort(nb.begin(), nb.end(), [&](uint32_t a, uint32_t b) {
                return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
            });
            cm.insert(cm.end(), nb.begin(), nb.end());
        }
    }
    for (uint32_t i = 0; i < n; ++i) perm[cm[i]] = n - 1 - i;
}

// By decreasing total degree (in + out over edges u -> v with u != v), ties by id.
void degree_order(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, uint32_t* perm) {
    std::vector<uint64_t> deg(n, 0);
    for (uint32_t v = 0; v < n; ++v)
        for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
            if (col[e] != v) {
                ++deg[v];
                ++deg[col[e]];
            }
    std::vector<uint32_t> ids(n);
    for (uint32_t v = 0; v < n; ++v) ids[v] = v;
    std::stable_sort(ids.begin(), ids.end(), [&](uint32_t a, uint32_t b) { return deg[a] > deg[b]; });
    for (uint32_t i = 0; i < n; ++i) perm[ids[i]] = i;
}

// A uniform permutation: Fisher-Yates over splitmix64(seed), each index drawn
// as the high 64 bits of a 64 x 64-bit product (Lemire's bounded draw, without
// the rejection step: bias below 2^-32 for n <= 2^32).
void random_order(uint32_t n, uint64_t seed, uint32_t* perm) {
    for (uint32_t v = 0; v < n; ++v) perm[v] = v;
    uint64_t x = seed;
    for (uint32_t i = n - 1; i > 0; --i) {
        const uint64_t r = splitmix64(x);
        const uint32_t j = (uint32_t)(((unsigned __int128)r * (uint64_t)(i + 1)) >> 64);
        std::swap(perm[i], perm[j]);
    }
}

// ---- clustering order: Louvain (Blondel, Guillaume, Lambiotte and Lefebvre,
// J. Stat. Mech. 2008), the sequential form of Section 5's Grappolo ----

// One level's graph: symmetric weighted adjacency (integer weights), each
// node's self-loop weight (internal edges of its community, counted from both
// ends) and its degree k = incident weights + self-loop weight.
struct LevelGraph {
    uint32_t n = 0;
    std::vector<uint64_t> off;
    std::vector<uint32_t> adj;
    std::vector<uint64_t> wt;
    std::vector<uint64_t> self_w;
    std::vector<uint64_t> k;
};

// Local moving: nodes in id order, each to the neighbouring community of the
// largest modularity gain k_i,c - tot_c * k_i / 2m (compared exactly, scaled by
// 2m); a node stays unless another community's gain is larger, ties between
// other communities go to the lower id.  Passes repeat until at most 0.1 % of
// the nodes move (at most 16).  Returns whether any node moved.
bool local_moving(const LevelGraph& G, uint64_t two_m, std::vector<uint32_t>& comm) {
    const uint32_t n = G.n;
    comm.resize(n);
    std::vector<uint64_t> tot(n);
    for (uint32_t i = 0; i < n; ++i) {
        comm[i] = i;
        tot[i] = G.k[i];
    }
    std::vector<uint64_t> nw(n, 0);
    std::vector<uint32_t> touched;
    bool moved_any = false;
    for (int pass = 0; pass < 16; ++pass) {
        uint64_t moves = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t ci = comm[i];
            touched.clear();
            for (uint64_t a = G.off[i]; a < G.off[i + 1]; ++a) {
                const uint32_t j = G.adj[a];
                if (j == i) continue;
                const uint32_t c = comm[j];
                if (nw[c] == 0) touched.push_back(c);
                nw[c] += G.wt[a];
            }
            tot[ci] -= G.k[i];
            auto gain = [&](uint32_t c) {
                return (__int128)nw[c] * (__int128)two_m - (__int128)tot[c] * (__int128)G.k[i];
            };
            uint32_t best = ci;
            __int128 best_gain = gain(ci);
            for (uint32_t c : touched) {
                if (c == ci) continue;
                const __int128 g = gain(c);
                if (g > best_gain || (g == best_gain && best != ci && c < best)) {
                    best = c;
                    best_gain = g;
                }
            }
            tot[best] += G.k[i];
            if (best != ci) {
                comm[i] = best;
                ++moves;
            }
            for (uint32_t c : touched) nw[c] = 0;
        }
        if (moves) moved_any = true;
        if (moves * 1000 <= n) break;  // fewer than 0.1 % of the nodes moved: the level has settled
    }
    return moved_any;
}

// Renumbers the communities 0 .. C-1 by first appearance in node order (ids
// written back into comm) and builds the community graph.
LevelGraph aggregate(const LevelGraph& G, std::vector<uint32_t>& comm) {
    const uint32_t n = G.n;
    std::vector<uint32_t> id(n, 0xFFFFFFFFu);
    uint32_t C = 0;
    for (uint32_t i = 0; i < n; ++i) {
        if (id[comm[i]] == 0xFFFFFFFFu) id[comm[i]] = C++;
        comm[i] = id[comm[i]];
    }
    // members of each community, in node order
    std::vector<uint64_t> moff((size_t)C + 1, 0);
    for (uint32_t i = 0; i < n; ++i) ++moff[comm[i] + 1];
    for (uint32_t c = 0; c < C; ++c) moff[c + 1] += moff[c];
    std::vector<uint32_t> mem(n);
    {
        std::vector<uint64_t> cur(moff.begin(), moff.end() - 1);
        for (uint32_t i = 0; i < n; ++i) mem[cur[comm[i]]++] = i;
    }
    LevelGraph H;
    H.n = C;
    H.off.assign((size_t)C + 1, 0);
    H.self_w.assign(C, 0);
    H.k.assign(C, 0);
    std::vector<uint64_t> nw(C, 0);
    std::vector<uint32_t> touched;
    for (uint32_t c = 0; c < C; ++c) {
        touched.clear();
        for (uint64_t a = moff[c]; a < moff[c + 1]; ++a) {
            const uint32_t i = mem[a];
            H.self_w[c] += G.self_w[i];
            H.k[c] += G.k[i];
            for (uint64_t e = G.off[i]; e < G.off[i + 1]; ++e) {
                const uint32_t d = comm[G.adj[e]];
                if (d == c) {
                    H.self_w[c] += G.wt[e];
                    continue;
                }
                if (nw[d] == 0) touched.push_back(d);
                nw[d] += G.wt[e];
            }
        }
        std::sort(touched.begin(), touched.end());
        for (uint32_t d : touched) {
            H.adj.push_back(d);
            H.wt.push_back(nw[d]);
            nw[d] = 0;
        }
        H.off[c + 1] = H.adj.size();
    }
    return H;
}

void cluster_order(uint32_t n, const std::vector<uint64_t>& off, const std::vector<uint32_t>& adj, uint32_t* perm) {
    LevelGraph G;
    G.n = n;
    G.off = off;
    G.adj = adj;
    G.wt.assign(adj.size(), 1);
    G.self_w.assign(n, 0);
    G.k.resize(n);
    for (uint32_t v = 0; v < n; ++v) G.k[v] = off[v + 1] - off[v];
    const uint64_t two_m = adj.size();
    // node of each vertex at every level; total degree and least member id of each node
    std::vector<std::vector<uint32_t>> node_of;   // [level][vertex]
    std::vector<std::vector<uint64_t>> tot_of;    // [level][node]
    std::vector<std::vector<uint32_t>> minid_of;  // [level][node]
    std::vector<uint32_t> cur(n);
    for (uint32_t v = 0; v < n; ++v) cur[v] = v;
    node_of.push_back(cur);
    tot_of.push_back(G.k);
    {
        std::vector<uint32_t> ids(n);
        for (uint32_t v = 0; v < n; ++v) ids[v] = v;
        minid_of.push_back(ids);
    }
    std::vector<uint32_t> comm;
    for (int level = 0; level < 8 && two_m > 0; ++level) {
        if (!local_moving(G, two_m, comm)) break;
        LevelGraph H = aggregate(G, comm);
        for (uint32_t v = 0; v < n; ++v) cur[v] = comm[cur[v]];
        std::vector<uint32_t> minid(H.n, 0xFFFFFFFFu);
        for (uint32_t v = 0; v < n; ++v) minid[cur[v]] = std::min(minid[cur[v]], v);
        node_of.push_back(cur);
        tot_of.push_back(H.k);
        minid_of.push_back(minid);
        G = std::move(H);
    }
    const int L = (int)node_of.size();
    std::vector<uint32_t> ids(n);
    for (uint32_t v = 0; v < n; ++v) ids[v] = v;
    std::sort(ids.begin(), ids.end(), [&](uint32_t a, uint32_t b) {
        for (int l = L - 1; l >= 0; --l) {
            const uint32_t x = node_of[l][a], y = node_of[l][b];
            if (x == y) continue;
            if (tot_of[l][x] != tot_of[l][y]) return tot_of[l][x] > tot_of[l][y];
            return minid_of[l][x] < minid_of[l][y];
        }
        return false;
    });
    for (uint32_t i = 0; i < n; ++i) perm[ids[i]] = i;
}

__global__ void k_relabel(const uint32_t* perm, const uint64_t* row_ptr, const uint32_t* col0, uint32_t n,
                          uint64_t m, uint32_t* col, uint32_t* inv, uint64_t* rstart, uint64_t* rend) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t e = t; e < m; e += stride) col[e] = perm[col0[e]];
    for (uint64_t v = t; v < n; v += stride) {
        const uint32_t w = perm[v];
        inv[w] = (uint32_t)v;
        rstart[w] = row_ptr[v];
        rend[w] = row_ptr[v + 1];
    }
}

// key = (sample index << 32) | label of its start vertex
__global__ void k_start_keys(uint64_t seed, uint64_t first_id, uint64_t S, uint32_t n, const uint32_t* perm,
                             uint64_t* keys) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t v = start_vertex(seed, first_id + j, n);
        keys[j] = (j << 32) | (perm ? perm[v] : v);
    }
}

__global__ void k_key_index(const uint64_t* keys, uint64_t S, uint32_t* order) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < S; k += (uint64_t)gridDim.x * blockDim.x)
        order[k] = (uint32_t)(keys[k] >> 32);
}

void drop_order(fbpt_graph* g) {
    cudaFree(g->perm);
    cudaFree(g->inv);
    cudaFree(g->col0);
    cudaFree(g->rstart);
    cudaFree(g->rend);
    g->perm = g->inv = g->col0 = nullptr;
    g->rstart = g->rend = nullptr;
}

}  // namespace

int start_order(const fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, cudaStream_t st,
                uint32_t** order) {
    *order = nullptr;
    uint64_t* keys = nullptr;
    uint64_t* tmp = nullptr;
    uint32_t* out = nullptr;
    auto release = [&](bool with_out) {
        if (keys) cudaFreeAsync(keys, st);
        if (tmp) cudaFreeAsync(tmp, st);
        if (with_out && out) cudaFreeAsync(out, st);
    };
    if (cudaMallocAsync(&keys, sizeof(uint64_t) * S, st) != cudaSuccess ||
        cudaMallocAsync(&tmp, sizeof(uint64_t) * S, st) != cudaSuccess ||
        cudaMallocAsync(&out, sizeof(uint32_t) * S, st) != cudaSuccess) {
        release(true);
        cudaGetLastError();
        return fail(FBPT_ENOMEM, "sorted starts: allocation failed");
    }
    const unsigned blocks = (unsigned)std::min<uint64_t>((S + 255) / 256, (uint64_t)device_sm_count() * 8);
    k_start_keys<<<blocks, 256, 0, st>>>(seed, first_id, S, g->n, g->perm, keys);
    // the label occupies the low bits (whole bytes), the sample index the high
    // 32: a stable sort on the label keeps equal labels in index order
    uint32_t bits = 8;
    while (bits < 32 && (1ull << bits) < (uint64_t)g->n) bits += 8;
    int rc = radix_sort_u64(keys, tmp, S, bits, st);
    if (rc == FBPT_OK) {
        k_key_index<<<blocks, 256, 0, st>>>(keys, S, out);
        if (cudaGetLastError() != cudaSuccess) rc = fail(FBPT_ECUDA, "sorted starts: launch failed");
    }
    release(rc != FBPT_OK);
    if (rc == FBPT_OK) *order = out;
    return rc;
}

}  // namespace fbpt

using namespace fbpt;

extern "C" int fbpt_order_compute(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                                  uint32_t method, uint64_t seed, uint32_t* perm) {
    if (n == 0 || !row_ptr || !perm || (m && !col)) return fail(FBPT_EINVAL, "fbpt_order_compute: null array or n = 0");
    if (method > FBPT_ORDER_CLUSTER) return fail(FBPT_EINVAL, "fbpt_order_compute: unknown method");
    if (!csr_ok(n, m, row_ptr, col)) return fail(FBPT_EINVAL, "fbpt_order_compute: malformed CSR");
    try {
        switch (method) {
            case FBPT_ORDER_IDENTITY:
                for (uint32_t v = 0; v < n; ++v) perm[v] = v;
                break;
            case FBPT_ORDER_RCM: {
                std::vector<uint64_t> off;
                std::vector<uint32_t> adj;
                undirected(n, row_ptr, col, off, adj);
                rcm(n, off, adj, perm);
                break;
            }
            case FBPT_ORDER_DEGREE:
                degree_order(n, row_ptr, col, perm);
                break;
            case FBPT_ORDER_CLUSTER: {
                std::vector<uint64_t> off;
                std::vector<uint32_t> adj;
                undirected(n, row_ptr, col, off, adj);
                cluster_order(n, off, adj, perm);
                break;
            }
            default:
                random_order(n, seed, perm);
                break;
        }
    } catch (const std::bad_alloc&) {
        return fail(FBPT_ENOMEM, "fbpt_order_compute: host allocation failed");
    }
    return FBPT_OK;
}

extern "C" int fbpt_graph_set_order(fbpt_graph* g, const uint32_t* perm, uint32_t sorted_starts) {
    if (!g) return fail(FBPT_EINVAL, "fbpt_graph_set_order: null graph");
    if (sorted_starts > 1) return fail(FBPT_EINVAL, "fbpt_graph_set_order: sorted_starts must be 0 or 1");
    bool identity = true;
    if (perm) {
        std::vector<char> seen(g->n, 0);
        for (uint32_t v = 0; v < g->n; ++v) {
            if (perm[v] >= g->n || seen[perm[v]])
                return fail(FBPT_EINVAL, "fbpt_graph_set_order: perm is not a permutation of 0 .. n-1");
            seen[perm[v]] = 1;
            identity = identity && perm[v] == v;
        }
    }
    const cudaStream_t st = g->stream;
    FBPT_CUDA_TRY(cudaStreamSynchronize(st));
    // the pull direction's out-edge CSR is built from col: drop it (rebuilt on demand)
    cudaFree(g->orow);
    cudaFree(g->odst);
    cudaFree(g->oeid);
    g->orow = nullptr;
    g->odst = nullptr;
    g->oeid = nullptr;
    if (identity) {
        if (g->col0 && g->m)
            FBPT_CUDA_TRY(cudaMemcpyAsync(g->col, g->col0, sizeof(uint32_t) * g->m, cudaMemcpyDeviceToDevice, st));
        FBPT_CUDA_TRY(cudaStreamSynchronize(st));
        drop_order(g);
        g->sorted_starts = sorted_starts;
        return FBPT_OK;
    }
    const uint64_t n = g->n;
    if (!g->col0) {
        if (cudaMalloc(&g->col0, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1)) != cudaSuccess) {
            g->col0 = nullptr;
            cudaGetLastError();
            return fail(FBPT_ENOMEM, "fbpt_graph_set_order: device allocation failed");
        }
        if (g->m && (cudaMemcpyAsync(g->col0, g->col, sizeof(uint32_t) * g->m, cudaMemcpyDeviceToDevice, st) !=
                         cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess)) {
            cudaFree(g->col0);
            g->col0 = nullptr;
            return fail(FBPT_ECUDA, std::string("fbpt_graph_set_order: ") + cudaGetErrorString(cudaGetLastError()));
        }
    }
    if ((!g->perm && cudaMalloc(&g->perm, sizeof(uint32_t) * n) != cudaSuccess) ||
        (!g->inv && cudaMalloc(&g->inv, sizeof(uint32_t) * n) != cudaSuccess) ||
        (!g->rstart && cudaMalloc(&g->rstart, sizeof(uint64_t) * n) != cudaSuccess) ||
        (!g->rend && cudaMalloc(&g->rend, sizeof(uint64_t) * n) != cudaSuccess)) {
        cudaGetLastError();
        if (g->m) cudaMemcpy(g->col, g->col0, sizeof(uint32_t) * g->m, cudaMemcpyDeviceToDevice);
        drop_order(g);
        return fail(FBPT_ENOMEM, "fbpt_graph_set_order: device allocation failed");
    }
    FBPT_CUDA_TRY(cudaMemcpyAsync(g->perm, perm, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st));
    const unsigned blocks = (unsigned)std::min<uint64_t>((std::max<uint64_t>(g->m, n) + 255) / 256,
                                                         (uint64_t)device_sm_count() * 8);
    k_relabel<<<std::max(blocks, 1u), 256, 0, st>>>(g->perm, g->row_ptr, g->col0, g->n, g->m, g->col, g->inv,
                                                     g->rstart, g->rend);
    FBPT_CUDA_TRY(cudaGetLastError());
    FBPT_CUDA_TRY(cudaStreamSynchronize(st));
    g->sorted_starts = sorted_starts;
    return FBPT_OK;
}

extern "C" int fbpt_graph_get_order(const fbpt_graph* g, uint32_t* perm, uint32_t* sorted_starts) {
    if (!g) return fail(FBPT_EINVAL, "fbpt_graph_get_order: null graph");
    if (perm) {
        if (g->perm) {
            FBPT_CUDA_TRY(cudaMemcpy(perm, g->perm, sizeof(uint32_t) * g->n, cudaMemcpyDeviceToHost));
        } else {
            for (uint32_t v = 0; v < g->n; ++v) perm[v] = v;
        }
    }
    if (sorted_starts) *sorted_starts = g->sorted_starts;
    return FBPT_OK;
}
