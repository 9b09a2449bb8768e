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

}  // namespace
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
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->thr);
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
