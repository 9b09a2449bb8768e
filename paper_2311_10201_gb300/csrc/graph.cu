// Graph upload and validation (the input of Definition 2: G with per-edge
// probabilities, here as integer thresholds floor(p * 2^32)).
#include <algorithm>

#include "internal.cuh"

namespace fbpt {
namespace {

// Error bits: 1 row_ptr[0] != 0, 2 row_ptr decreases, 4 row_ptr[n] != m, 8 col >= n.
__global__ void k_validate(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m, unsigned* err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t0 == 0) {
        if (row_ptr[0] != 0) atomicOr(err, 1u);
        if (row_ptr[n] != m) atomicOr(err, 4u);
    }
    for (uint64_t v = t0; v < n; v += stride)
        if (row_ptr[v + 1] < row_ptr[v]) atomicOr(err, 2u);
    for (uint64_t e = t0; e < m; e += stride)
        if (col[e] >= n) atomicOr(err, 8u);
}

__global__ void k_outdeg(const uint32_t* col, uint64_t m, uint32_t* deg) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[col[e]], 1u);
}

// One warp per in-row v: each in-edge e = (w -> v) goes to out-row w as (v, e).
__global__ void k_outfill(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, const uint64_t* orow,
                          uint32_t* cursor, uint32_t* odst, uint32_t* oeid) {
    const uint32_t lane = lane_id();
    const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarp = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = wid; v < n; v += nwarp)
        for (uint64_t e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) {
            const uint32_t w = col[e];
            const uint64_t p = orow[w] + atomicAdd(&cursor[w], 1u);
            odst[p] = (uint32_t)v;
            oeid[p] = (uint32_t)e;
        }
}

// LT weights in units of 2^-32 (0xFFFFFFFF is the always-kept marker: 2^32).
__global__ void k_lt_weights(const uint32_t* thr, uint64_t m, uint64_t* w) {
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
        w[e] = thr[e] == 0xFFFFFFFFu ? (1ull << 32) : (uint64_t)thr[e];
}

__global__ void k_lt_rows(const uint64_t* row_ptr, const uint64_t* wpre, uint32_t n, unsigned* bad) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (uint64_t)gridDim.x * blockDim.x)
        if (wpre[row_ptr[v + 1]] - wpre[row_ptr[v]] > (1ull << 32)) atomicOr(bad, 1u);
}

}  // namespace

int ensure_lt_weights(fbpt_graph* g, cudaStream_t st) {
    if (g->lt_rows < 0) return fail(FBPT_EINVAL, "LT model: some row's in-edge weights sum to more than 1");
    if (g->wpre) return FBPT_OK;
    uint64_t* w = nullptr;
    unsigned* bad = nullptr;
    unsigned hbad = 0;
    FBPT_CUDA_TRY(cudaMalloc(&g->wpre, sizeof(uint64_t) * (g->m + 1)));
    int rc = FBPT_OK;
    if (cudaMallocAsync(&w, sizeof(uint64_t) * std::max<uint64_t>(g->m, 1), st) != cudaSuccess ||
        cudaMallocAsync(&bad, sizeof(unsigned), st) != cudaSuccess)
        rc = fail(FBPT_ENOMEM, "LT model: weight prefix scratch");
    if (rc == FBPT_OK) {
        const int sms = device_sm_count();
        k_lt_weights<<<sms * 8, 256, 0, st>>>(g->thr, g->m, w);
        rc = exclusive_scan_u64(w, g->wpre, g->m, st);
    }
    if (rc == FBPT_OK) {
        cudaMemsetAsync(bad, 0, sizeof(unsigned), st);
        k_lt_rows<<<device_sm_count() * 8, 256, 0, st>>>(g->row_ptr, g->wpre, g->n, bad);
        if (cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = fail(FBPT_ECUDA, "LT model: weight check failed");
    }
    if (w) cudaFreeAsync(w, st);
    if (bad) cudaFreeAsync(bad, st);
    if (rc == FBPT_OK && hbad) {
        g->lt_rows = -1;
        rc = fail(FBPT_EINVAL, "LT model: some row's in-edge weights sum to more than 1");
    }
    if (rc != FBPT_OK) {
        cudaStreamSynchronize(st);
        cudaFree(g->wpre);
        g->wpre = nullptr;
        return rc;
    }
    g->lt_rows = 1;
    return FBPT_OK;
}

int ensure_out_csr(fbpt_graph* g, cudaStream_t st) {
    if (g->orow) return FBPT_OK;
    if (g->m >= (1ull << 32)) return fail(FBPT_EUNSUPPORTED, "pull levels need fewer than 2^32 edges");
    uint32_t* cnt = nullptr;
    FBPT_CUDA_TRY(cudaMalloc(&g->orow, sizeof(uint64_t) * ((uint64_t)g->n + 1)));
    FBPT_CUDA_TRY(cudaMalloc(&g->odst, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1)));
    FBPT_CUDA_TRY(cudaMalloc(&g->oeid, sizeof(uint32_t) * std::max<uint64_t>(g->m, 1)));
    FBPT_CUDA_TRY(cudaMallocAsync(&cnt, sizeof(uint32_t) * g->n, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * g->n, st));
    const int sms = device_sm_count();
    k_outdeg<<<sms * 8, 256, 0, st>>>(g->col, g->m, cnt);
    int rc = exclusive_scan_u32(cnt, g->orow, g->n, st);
    if (rc == FBPT_OK) {
        FBPT_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * g->n, st));
        k_outfill<<<sms * 8, 256, 0, st>>>(g->row_ptr, g->col, g->n, g->orow, cnt, g->odst, g->oeid);
        FBPT_CUDA_TRY(cudaGetLastError());
    }
    cudaFreeAsync(cnt, st);
    if (rc != FBPT_OK) {
        cudaFree(g->orow); cudaFree(g->odst); cudaFree(g->oeid);
        g->orow = nullptr; g->odst = nullptr; g->oeid = nullptr;
    }
    return rc;
}

}  // namespace fbpt

using namespace fbpt;

extern "C" int fbpt_graph_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                                 const uint32_t* thr, int mem_kind, void* stream, fbpt_graph** out) {
    if (!out) return fail(FBPT_EINVAL, "fbpt_graph_create: out is NULL");
    *out = nullptr;
    if (n == 0) return fail(FBPT_EINVAL, "fbpt_graph_create: n must be >= 1");
    if (n > (1u << kUnitBits)) return fail(FBPT_EINVAL, "fbpt_graph_create: n must be <= 2^26");
    if (m >= (1ull << 40)) return fail(FBPT_EINVAL, "fbpt_graph_create: m must be < 2^40");
    if (!row_ptr || (m && (!col || !thr))) return fail(FBPT_EINVAL, "fbpt_graph_create: null array");
    if (mem_kind != FBPT_MEM_HOST && mem_kind != FBPT_MEM_DEVICE)
        return fail(FBPT_EINVAL, "fbpt_graph_create: bad mem_kind");
    cudaStream_t st = (cudaStream_t)stream;
    FBPT_TRY(noalloc_preload());
    fbpt_graph* g = new fbpt_graph();
    g->n = n;
    g->m = m;
    g->stream = st;
    cudaGetDevice(&g->device);
    const uint64_t mpad = ((m + 3) / 4) * 4 + 4;
    auto cleanup = [&](int code, const char* what) {
        cudaFree(g->row_ptr);
        cudaFree(g->col);
        cudaFree(g->thr);
        delete g;
        cudaGetLastError();
        return fail(code, std::string("fbpt_graph_create: ") + what);
    };
    if (cudaMalloc(&g->row_ptr, sizeof(uint64_t) * ((uint64_t)n + 1)) != cudaSuccess ||
        cudaMalloc(&g->col, sizeof(uint32_t) * mpad) != cudaSuccess ||
        cudaMalloc(&g->thr, sizeof(uint32_t) * mpad) != cudaSuccess)
        return cleanup(FBPT_ENOMEM, "device allocation failed");
    const cudaMemcpyKind kind = mem_kind == FBPT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (cudaMemsetAsync(g->col, 0, sizeof(uint32_t) * mpad, st) != cudaSuccess ||
        cudaMemsetAsync(g->thr, 0, sizeof(uint32_t) * mpad, st) != cudaSuccess ||
        cudaMemcpyAsync(g->row_ptr, row_ptr, sizeof(uint64_t) * ((uint64_t)n + 1), kind, st) != cudaSuccess ||
        (m && cudaMemcpyAsync(g->col, col, sizeof(uint32_t) * m, kind, st) != cudaSuccess) ||
        (m && cudaMemcpyAsync(g->thr, thr, sizeof(uint32_t) * m, kind, st) != cudaSuccess))
        return cleanup(FBPT_ECUDA, "copy failed");
    unsigned* derr = nullptr;
    unsigned herr = 0;
    if (cudaMallocAsync(&derr, sizeof(unsigned), st) != cudaSuccess) return cleanup(FBPT_ENOMEM, "scratch");
    cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
    const int blocks = (int)std::min<uint64_t>(((std::max<uint64_t>(m, n)) + 255) / 256 + 1,
                                               (uint64_t)device_sm_count() * 8);
    k_validate<<<blocks, 256, 0, st>>>(g->row_ptr, g->col, n, m, derr);
    cudaMemcpyAsync(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(derr, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return cleanup(FBPT_ECUDA, cudaGetErrorString(cudaGetLastError()));
    if (herr) {
        std::string why;
        if (herr & 1) why += " row_ptr[0] != 0;";
        if (herr & 2) why += " row_ptr decreases;";
        if (herr & 4) why += " row_ptr[n] != m;";
        if (herr & 8) why += " col[e] >= n;";
        return cleanup(FBPT_EINVAL, ("invalid CSR:" + why).c_str());
    }
    *out = g;
    return FBPT_OK;
}

extern "C" int fbpt_graph_destroy(fbpt_graph* g) {
    if (!g) return FBPT_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    cudaDeviceSynchronize();
    workspace_release(g);
    cudaFree(g->orow);
    cudaFree(g->odst);
    cudaFree(g->oeid);
    cudaFree(g->wpre);
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->thr);
    cudaFree(g->perm);
    cudaFree(g->inv);
    cudaFree(g->col0);
    cudaFree(g->rstart);
    cudaFree(g->rend);
    delete g;
    return FBPT_OK;
}

extern "C" int fbpt_graph_info(const fbpt_graph* g, uint32_t* n, uint64_t* m, const uint64_t** row_ptr,
                               const uint32_t** col, const uint32_t** thr) {
    if (!g) return fail(FBPT_EINVAL, "fbpt_graph_info: null graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (row_ptr) *row_ptr = g->row_ptr;
    if (col) *col = g->col;
    if (thr) *thr = g->thr;
    return FBPT_OK;
}
