// Greedy max-k-cover seed selection over RR sets (Section 2: selecting the k
// seeds reduces to a maximum k-cover over the RRR sets; greedy gives 1-1/e).
//
// Initial gains are the per-vertex RR-row counts, i.e. the popcounts of the
// visited masks accumulated when the rows were emitted.  An inverted index
// (vertex -> rows containing it) turns each pick into a walk over the newly
// covered rows, decrementing the gain of every vertex in them.
#include <algorithm>
#include <string>

#include "internal.cuh"

namespace fbpt {
namespace {

__global__ void k_inv_fill(const uint64_t* offsets, const uint32_t* verts, uint64_t S, const uint64_t* inv_off,
                           uint32_t* cursor, uint32_t* inv) {
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t j = wid; j < S; j += nwarp) {
        const uint64_t a = offsets[j], b = offsets[j + 1];
        for (uint64_t p = a + lane; p < b; p += 32) {
            const uint32_t v = verts[p];
            const uint32_t pos = atomicAdd(&cursor[v], 1u);
            inv[inv_off[v] + pos] = (uint32_t)j;
        }
    }
}

// key(v) = gain << 32 | (2^32-1 - v): the maximum is the largest gain, the
// smallest id among equals; selected vertices get key 0 (never the maximum,
// since an unselected vertex always has key >= 1).
__global__ void k_argmax(const uint32_t* gain, const uint8_t* selected, uint32_t n, unsigned long long* best) {
    unsigned long long m = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x) {
        if (selected[v]) continue;
        const unsigned long long key = ((unsigned long long)gain[v] << 32) | (0xFFFFFFFFull - v);
        m = key > m ? key : m;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    __shared__ unsigned long long s_m[32];
    if (lane_id() == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? s_m[threadIdx.x] : 0ull;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, d);
            m = o > m ? o : m;
        }
        if (threadIdx.x == 0 && m) atomicMax(best, m);
    }
}

__global__ void k_cover(const unsigned long long* best, uint32_t r, uint32_t n, const uint64_t* offsets, const uint32_t* verts,
                        const uint64_t* inv_off, const uint32_t* inv, uint8_t* covered, uint32_t* gain,
                        uint8_t* selected, uint32_t* seeds, uint64_t* gains) {
    const unsigned long long key = best[r];
    const uint32_t u = (uint32_t)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
    if (key == 0 || u >= n) return;  // cannot happen for k <= n; never index with it
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        selected[u] = 1;
        seeds[r] = u;
        gains[r] = key >> 32;
    }
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t a = inv_off[u], cnt = inv_off[u + 1] - a;
    for (uint64_t i = wid; i < cnt; i += nwarp) {
        const uint32_t j = inv[a + i];
        if (covered[j]) continue;  // warp-uniform
        __syncwarp();
        if (lane == 0) covered[j] = 1;
        for (uint64_t p = offsets[j] + lane; p < offsets[j + 1]; p += 32) atomicSub(&gain[verts[p]], 1u);
    }
}

}  // namespace
}  // namespace fbpt

using namespace fbpt;

extern "C" int fbpt_select_seeds(const fbpt_rrsets* rr, uint32_t k, uint32_t* seeds_host, uint64_t* gains_host) {
    if (!rr || !rr->offsets || !rr->vcount) return fail(FBPT_EINVAL, "fbpt_select_seeds: null rrsets");
    if (k > rr->n) return fail(FBPT_EINVAL, "fbpt_select_seeds: k > n");
    if (k == 0) return FBPT_OK;
    if (!seeds_host) return fail(FBPT_EINVAL, "fbpt_select_seeds: null seeds");
    cudaStream_t st = (cudaStream_t)rr->stream;
    const uint32_t n = rr->n;
    const uint64_t S = rr->S;
    uint64_t* inv_off = nullptr;
    uint32_t *inv = nullptr, *cursor = nullptr, *gain = nullptr, *seeds = nullptr;
    uint8_t *covered = nullptr, *selected = nullptr;
    unsigned long long* best = nullptr;
    uint64_t* gains = nullptr;
    int rc = FBPT_OK;
    auto A = [&](void** p, size_t b) {
        if (rc == FBPT_OK && cudaMallocAsync(p, std::max<size_t>(b, 8), st) != cudaSuccess)
            rc = fail(FBPT_ENOMEM, "fbpt_select_seeds: allocation failed");
    };
    A((void**)&inv_off, sizeof(uint64_t) * ((size_t)n + 1));
    A((void**)&inv, sizeof(uint32_t) * rr->total);
    A((void**)&cursor, sizeof(uint32_t) * n);
    A((void**)&gain, sizeof(uint32_t) * n);
    A((void**)&covered, S);
    A((void**)&selected, n);
    A((void**)&best, sizeof(unsigned long long) * k);
    A((void**)&seeds, sizeof(uint32_t) * k);
    A((void**)&gains, sizeof(uint64_t) * k);
    if (rc == FBPT_OK) {
        cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * n, st);
        cudaMemsetAsync(covered, 0, S, st);
        cudaMemsetAsync(selected, 0, n, st);
        cudaMemsetAsync(best, 0, sizeof(unsigned long long) * k, st);
        cudaMemcpyAsync(gain, rr->vcount, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        rc = exclusive_scan_u32(rr->vcount, inv_off, n, st);
    }
    if (rc == FBPT_OK) {
        const int sms = device_sm_count();
        k_inv_fill<<<sms * 8, 256, 0, st>>>(rr->offsets, rr->verts, S, inv_off, cursor, inv);
        const int ablocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
        for (uint32_t r = 0; r < k; ++r) {
            k_argmax<<<ablocks, 256, 0, st>>>(gain, selected, n, best + r);
            k_cover<<<sms * 4, 256, 0, st>>>(best, r, n, rr->offsets, rr->verts, inv_off, inv, covered, gain, selected,
                                               seeds, gains);
        }
        if (cudaGetLastError() != cudaSuccess) rc = fail(FBPT_ECUDA, "fbpt_select_seeds: launch failed");
    }
    if (rc == FBPT_OK) {
        cudaMemcpyAsync(seeds_host, seeds, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st);
        if (gains_host) cudaMemcpyAsync(gains_host, gains, sizeof(uint64_t) * k, cudaMemcpyDeviceToHost, st);
    }
    cudaFreeAsync(inv_off, st); cudaFreeAsync(inv, st); cudaFreeAsync(cursor, st); cudaFreeAsync(gain, st);
    cudaFreeAsync(covered, st); cudaFreeAsync(selected, st); cudaFreeAsync(best, st); cudaFreeAsync(seeds, st);
    cudaFreeAsync(gains, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == FBPT_OK)
        rc = fail(FBPT_ECUDA, std::string("fbpt_select_seeds: ") + cudaGetErrorString(cudaGetLastError()));
    return rc;
}

// ---- seed selection that allocates nothing ------------------------------------------------
//
// Some callers cannot allocate device memory at the point where they pick
// seeds: a serving process that hands all free device memory to its own pool
// at start-up (a cudaMalloc would fail or fragment that pool), or a host
// thread on a latency-critical path that must not take the allocator's locks.
// fbpt_select_seeds_noalloc gives them the same greedy picks as
// fbpt_select_seeds with its working memory in the file-scope array below:
// every GPU that loads libfbpt holds these 64 MiB until the process exits.
// CUDA places a module's device arrays when the module is loaded on a device,
// and by default it loads modules lazily, on first use; so graph creation
// (noalloc_preload) touches the array, which loads this file's module while
// the caller can still allocate, and the later call needs nothing new.
// Instead of an inverted index it finds, each round, the uncovered rows that
// contain the pick by a binary search in every row (rows are ascending).

namespace fbpt {
namespace {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Each thread takes uncovered rows; a row containing the pick is covered and
// the gain of each of its vertices drops by one.
__global__ void k_cover_rows(const unsigned long long* best, uint32_t r, uint32_t n, const uint64_t* offsets,
                             const uint32_t* verts, uint64_t S, uint8_t* covered, uint32_t* gain, uint8_t* selected,
                             uint32_t* seeds, uint64_t* gains) {
    const unsigned long long key = best[r];
    const uint32_t u = (uint32_t)(0xFFFFFFFFull - (key & 0xFFFFFFFFull));
    if (key == 0 || u >= n) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        selected[u] = 1;
        seeds[r] = u;
        gains[r] = key >> 32;
    }
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x) {
        if (covered[j]) continue;
        uint64_t lo = offsets[j], hi = offsets[j + 1];
        const uint64_t a = lo, b = hi;
        while (lo < hi) {  // first position with verts[p] >= u
            const uint64_t mid = (lo + hi) >> 1;
            if (verts[mid] < u) lo = mid + 1; else hi = mid;
        }
        if (lo == b || verts[lo] != u) continue;
        covered[j] = 1;
        for (uint64_t p = a; p < b; ++p) atomicSub(&gain[verts[p]], 1u);
    }
}

// Device address of the scratch array on the current device, looked up on
// every call (a host-side cache could outlive the context that it came from,
// e.g. across a cudaDeviceReset; the lookup costs next to nothing).
int noalloc_base(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(FBPT_ECUDA, std::string("fbpt_select_seeds_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return FBPT_OK;
}

}  // namespace

// Loads this file's module (and so places the scratch array) on the current
// device; called when a graph is created there.
int noalloc_preload() {
    void* p = nullptr;
    return noalloc_base(&p);
}

}  // namespace fbpt

extern "C" int fbpt_select_seeds_noalloc(const fbpt_rrsets* rr, uint32_t k, uint32_t* seeds_host,
                                         uint64_t* gains_host) {
    if (!rr || !rr->offsets || !rr->vcount) return fail(FBPT_EINVAL, "fbpt_select_seeds_noalloc: null rrsets");
    if (k > rr->n) return fail(FBPT_EINVAL, "fbpt_select_seeds_noalloc: k > n");
    if (k == 0) return FBPT_OK;
    if (!seeds_host) return fail(FBPT_EINVAL, "fbpt_select_seeds_noalloc: null seeds");
    const uint32_t n = rr->n;
    const uint64_t S = rr->S;
    const size_t o_gain = 0;
    const size_t o_sel = o_gain + align256(sizeof(uint32_t) * (size_t)n);
    const size_t o_cov = o_sel + align256((size_t)n);
    const size_t o_best = o_cov + align256((size_t)S);
    const size_t o_seeds = o_best + align256(sizeof(unsigned long long) * k);
    const size_t o_gains = o_seeds + align256(sizeof(uint32_t) * k);
    const size_t need = o_gains + align256(sizeof(uint64_t) * k);
    if (need > kNoAllocScratchBytes)
        return fail(FBPT_EINVAL, "fbpt_select_seeds_noalloc: needs " + std::to_string(need) +
                                     " bytes of scratch (5 bytes per vertex + 1 per RR set + 20 per seed), more "
                                     "than its fixed " + std::to_string(kNoAllocScratchBytes) + " bytes");
    void* basev = nullptr;
    FBPT_TRY(noalloc_base(&basev));
    unsigned char* base = static_cast<unsigned char*>(basev);
    uint32_t* gain = reinterpret_cast<uint32_t*>(base + o_gain);
    uint8_t* selected = base + o_sel;
    uint8_t* covered = base + o_cov;
    unsigned long long* best = reinterpret_cast<unsigned long long*>(base + o_best);
    uint32_t* seeds = reinterpret_cast<uint32_t*>(base + o_seeds);
    uint64_t* gains = reinterpret_cast<uint64_t*>(base + o_gains);
    cudaStream_t st = (cudaStream_t)rr->stream;
    // the array keeps the previous call's contents: start from zero
    FBPT_CUDA_TRY(cudaMemsetAsync(selected, 0, n, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(covered, 0, S, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(best, 0, sizeof(unsigned long long) * k, st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(gain, rr->vcount, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
    const int sms = device_sm_count();
    const int ablocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
    const int cblocks = (int)std::min<uint64_t>((S + 255) / 256, (uint64_t)sms * 8);
    for (uint32_t r = 0; r < k; ++r) {
        k_argmax<<<ablocks, 256, 0, st>>>(gain, selected, n, best + r);
        k_cover_rows<<<cblocks, 256, 0, st>>>(best, r, n, rr->offsets, rr->verts, S, covered, gain, selected, seeds,
                                              gains);
    }
    // from here on, work that uses the shared array is queued: on any error, wait
    // for it before returning so that a following call cannot overlap it
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(seeds_host, seeds, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && gains_host)
        e = cudaMemcpyAsync(gains_host, gains, sizeof(uint64_t) * k, cudaMemcpyDeviceToHost, st);
    const cudaError_t es = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess)
        return fail(FBPT_ECUDA, std::string("fbpt_select_seeds_noalloc: ") + cudaGetErrorString(e));
    return FBPT_OK;
}
