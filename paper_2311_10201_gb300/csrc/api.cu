// C ABI glue: errors, version, RR-set buffers, sampling entry points and the
// verification building blocks (device results of the bit-level contract).
#include <algorithm>
#include <cstring>
#include <string>

#include "internal.cuh"

namespace fbpt {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
const char* last_error() { return g_last_error.c_str(); }

int device_sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

namespace {

__global__ void k_edge_draws(uint64_t seed, const uint64_t* s, const uint64_t* e, uint64_t count, uint32_t* out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 r = edge_draws4(seed, s[i], e[i] >> 2);
        const uint32_t k = (uint32_t)(e[i] & 3);
        out[i] = k == 0 ? r.x : k == 1 ? r.y : k == 2 ? r.z : r.w;
    }
}

__global__ void k_starts(uint64_t seed, const uint64_t* s, uint64_t count, uint32_t n, uint32_t* out) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = start_vertex(seed, s[i], n);
}

// Nothing but Philox4x32-10 evaluations with the round keys hoisted as in the
// expand: two independent counter chains per iteration, outputs folded into
// one word (stored only if it matches a value it never takes, so that the
// calls are not optimised away).
constexpr int kRateThreads = 256;
__global__ void __launch_bounds__(kRateThreads) k_philox_rate(uint64_t seed, uint32_t iters, uint32_t* sink) {
    const PhiloxKeys K = philox_keys(seed);
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint32_t k = 0; k < iters; ++k) {
        const uint4 a = philox4x32_10(make_uint4(t, k, 2u * k, 7u), K);
        const uint4 b = philox4x32_10(make_uint4(t, k, 2u * k + 1u, 7u), K);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w;
    }
    if (acc == 0x9E3779B9u && t == 0xFFFFFFFFu) sink[0] = acc;
}

}  // namespace
}  // namespace fbpt

using namespace fbpt;

extern "C" const char* fbpt_last_error(void) { return last_error(); }
extern "C" int fbpt_version(void) { return FBPT_VERSION; }

extern "C" int fbpt_abi_sizes(uint64_t* sizes, int count) {
    if (!sizes || count < 3) return fail(FBPT_EINVAL, "fbpt_abi_sizes: need at least 3 entries");
    const uint64_t all[6] = {sizeof(fbpt_opts), sizeof(fbpt_rrsets), sizeof(fbpt_stats), sizeof(fbpt_tuning),
                             sizeof(fbpt_imm_result), sizeof(fbpt_trace_row)};
    for (int i = 0; i < count && i < 6; ++i) sizes[i] = all[i];
    return FBPT_OK;
}

extern "C" int fbpt_sample(fbpt_graph* g, uint64_t seed, uint64_t first_id, uint64_t S, const fbpt_opts* opts,
                           fbpt_rrsets* out, fbpt_stats* stats) {
    try {
        return sample_impl(g, seed, first_id, S, opts, out, stats);
    } catch (const std::exception& e) {
        return fail(FBPT_ENOMEM, std::string("fbpt_sample: ") + e.what());
    }
}

extern "C" int fbpt_sample_batched(uint32_t G, fbpt_graph* const* gs, const uint64_t* seeds, const uint64_t* first_ids,
                                   const uint64_t* Ss, const fbpt_opts* opts, fbpt_rrsets* outs, fbpt_stats* stats) {
    try {
        return sample_batched_impl(G, gs, seeds, first_ids, Ss, opts, outs, stats);
    } catch (const std::exception& e) {
        return fail(FBPT_ENOMEM, std::string("fbpt_sample_batched: ") + e.what());
    }
}

extern "C" int fbpt_autotune(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base, fbpt_tuning* out) {
    try {
        return autotune_impl(g, seed, S, base, out);
    } catch (const std::exception& e) {
        return fail(FBPT_ENOMEM, std::string("fbpt_autotune: ") + e.what());
    }
}

extern "C" int fbpt_imm(fbpt_graph* g, uint32_t k, double epsilon, double ell, uint64_t seed, uint64_t max_samples,
                        const fbpt_opts* opts, uint32_t* seeds_host, uint64_t* gains_host, fbpt_imm_result* result,
                        fbpt_stats* stats) {
    try {
        return imm_impl(g, k, epsilon, ell, seed, max_samples, opts, seeds_host, gains_host, result, stats);
    } catch (const std::exception& e) {
        return fail(FBPT_ENOMEM, std::string("fbpt_imm: ") + e.what());
    }
}

extern "C" int fbpt_policy_width(fbpt_graph* g, uint64_t seed, uint64_t S, const fbpt_opts* base,
                                 uint32_t* row_words, float* scores) {
    try {
        return policy_width_impl(g, seed, S, base, row_words, scores);
    } catch (const std::exception& e) {
        return fail(FBPT_ENOMEM, std::string("fbpt_policy_width: ") + e.what());
    }
}

extern "C" int fbpt_graph_set_tuning(fbpt_graph* g, const fbpt_tuning* t) {
    if (!g || !t) return fail(FBPT_EINVAL, "fbpt_graph_set_tuning: null argument");
    if (t->words != 1 && t->words != 2 && t->words != 4 && t->words != 8)
        return fail(FBPT_EINVAL, "fbpt_graph_set_tuning: words must be 1, 2, 4 or 8");
    if (t->slots < 1 || t->words * t->slots > 64) return fail(FBPT_EINVAL, "fbpt_graph_set_tuning: words * slots > 64");
    if (t->refill > FBPT_REFILL_BATCH || t->schedule > FBPT_SCHED_FILTERED)
        return fail(FBPT_EINVAL, "fbpt_graph_set_tuning: bad refill or schedule");
    g->tuned = *t;
    g->tuned_valid = true;
    return FBPT_OK;
}

extern "C" int fbpt_graph_tuning(const fbpt_graph* g, fbpt_tuning* out) {
    if (!g || !out) return fail(FBPT_EINVAL, "fbpt_graph_tuning: null argument");
    if (!g->tuned_valid) return fail(FBPT_EINVAL, "fbpt_graph_tuning: graph was never tuned");
    *out = g->tuned;
    return FBPT_OK;
}

extern "C" int fbpt_rrsets_free(fbpt_rrsets* rr) {
    if (!rr) return FBPT_OK;
    cudaStream_t st = (cudaStream_t)rr->stream;
    if (rr->offsets) cudaFreeAsync(rr->offsets, st);
    if (rr->verts) cudaFreeAsync(rr->verts, st);
    if (rr->starts) cudaFreeAsync(rr->starts, st);
    if (rr->vcount) cudaFreeAsync(rr->vcount, st);
    std::memset(rr, 0, sizeof(*rr));
    return FBPT_OK;
}

extern "C" int fbpt_rrsets_copy_to_host(const fbpt_rrsets* rr, uint64_t* offsets, uint32_t* verts, uint32_t* starts,
                                        uint32_t* vcount) {
    if (!rr) return fail(FBPT_EINVAL, "fbpt_rrsets_copy_to_host: null rrsets");
    cudaStream_t st = (cudaStream_t)rr->stream;
    if (offsets) FBPT_CUDA_TRY(cudaMemcpyAsync(offsets, rr->offsets, sizeof(uint64_t) * (rr->S + 1), cudaMemcpyDeviceToHost, st));
    if (verts && rr->total) FBPT_CUDA_TRY(cudaMemcpyAsync(verts, rr->verts, sizeof(uint32_t) * rr->total, cudaMemcpyDeviceToHost, st));
    if (starts) FBPT_CUDA_TRY(cudaMemcpyAsync(starts, rr->starts, sizeof(uint32_t) * rr->S, cudaMemcpyDeviceToHost, st));
    if (vcount) FBPT_CUDA_TRY(cudaMemcpyAsync(vcount, rr->vcount, sizeof(uint32_t) * rr->n, cudaMemcpyDeviceToHost, st));
    FBPT_CUDA_TRY(cudaStreamSynchronize(st));
    return FBPT_OK;
}

extern "C" int fbpt_rrsets_copy_rows(const fbpt_rrsets* rr, uint64_t first_row, uint64_t count, uint64_t* offsets_host,
                                     uint32_t* verts_host, uint64_t verts_cap) {
    if (!rr || !offsets_host) return fail(FBPT_EINVAL, "fbpt_rrsets_copy_rows: null argument");
    if (first_row > rr->S || count > rr->S - first_row) return fail(FBPT_EINVAL, "fbpt_rrsets_copy_rows: rows out of range");
    cudaStream_t st = (cudaStream_t)rr->stream;
    FBPT_CUDA_TRY(cudaMemcpyAsync(offsets_host, rr->offsets + first_row, sizeof(uint64_t) * (count + 1),
                                  cudaMemcpyDeviceToHost, st));
    FBPT_CUDA_TRY(cudaStreamSynchronize(st));
    const uint64_t len = offsets_host[count] - offsets_host[0];
    if (len > verts_cap) return fail(FBPT_EINVAL, "fbpt_rrsets_copy_rows: rows hold more than verts_cap vertices");
    if (len) {
        if (!verts_host) return fail(FBPT_EINVAL, "fbpt_rrsets_copy_rows: null verts");
        FBPT_CUDA_TRY(cudaMemcpyAsync(verts_host, rr->verts + offsets_host[0], sizeof(uint32_t) * len,
                                      cudaMemcpyDeviceToHost, st));
        FBPT_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return FBPT_OK;
}

extern "C" int fbpt_edge_draws(uint64_t seed, const uint64_t* s, const uint64_t* e, uint64_t count, uint32_t* out) {
    if (count == 0) return FBPT_OK;
    if (!s || !e || !out) return fail(FBPT_EINVAL, "fbpt_edge_draws: null array");
    uint64_t *ds = nullptr, *de = nullptr;
    uint32_t* dout = nullptr;
    FBPT_CUDA_TRY(cudaMalloc(&ds, count * 8));
    FBPT_CUDA_TRY(cudaMalloc(&de, count * 8));
    FBPT_CUDA_TRY(cudaMalloc(&dout, count * 4));
    cudaMemcpy(ds, s, count * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(de, e, count * 8, cudaMemcpyHostToDevice);
    k_edge_draws<<<(unsigned)std::min<uint64_t>((count + 255) / 256, 4096), 256>>>(seed, ds, de, count, dout);
    cudaError_t err = cudaMemcpy(out, dout, count * 4, cudaMemcpyDeviceToHost);
    cudaFree(ds);
    cudaFree(de);
    cudaFree(dout);
    if (err != cudaSuccess) return fail(FBPT_ECUDA, std::string("fbpt_edge_draws: ") + cudaGetErrorString(err));
    return FBPT_OK;
}

extern "C" int fbpt_start_vertices(uint64_t seed, const uint64_t* s, uint64_t count, uint32_t n, uint32_t* out) {
    if (count == 0) return FBPT_OK;
    if (!s || !out || n == 0) return fail(FBPT_EINVAL, "fbpt_start_vertices: bad argument");
    uint64_t* ds = nullptr;
    uint32_t* dout = nullptr;
    FBPT_CUDA_TRY(cudaMalloc(&ds, count * 8));
    FBPT_CUDA_TRY(cudaMalloc(&dout, count * 4));
    cudaMemcpy(ds, s, count * 8, cudaMemcpyHostToDevice);
    k_starts<<<(unsigned)std::min<uint64_t>((count + 255) / 256, 4096), 256>>>(seed, ds, count, n, dout);
    cudaError_t err = cudaMemcpy(out, dout, count * 4, cudaMemcpyDeviceToHost);
    cudaFree(ds);
    cudaFree(dout);
    if (err != cudaSuccess) return fail(FBPT_ECUDA, std::string("fbpt_start_vertices: ") + cudaGetErrorString(err));
    return FBPT_OK;
}

extern "C" int fbpt_philox_rate(uint64_t seed, uint32_t calls_per_thread, void* stream, double* calls_per_s) {
    if (!calls_per_s || calls_per_thread < 2) return fail(FBPT_EINVAL, "fbpt_philox_rate: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    int per = 0;
    FBPT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_philox_rate, kRateThreads, 0));
    const int blocks = device_sm_count() * std::max(per, 1);
    const uint32_t iters = calls_per_thread / 2;
    uint32_t* sink = nullptr;
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&sink, sizeof(uint32_t), st));
    cudaEvent_t a = nullptr, b = nullptr;
    int rc = FBPT_OK;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = fail(FBPT_ECUDA, "event create failed");
    if (rc == FBPT_OK) {
        k_philox_rate<<<blocks, kRateThreads, 0, st>>>(seed, iters, sink);  // warm-up
        cudaEventRecord(a, st);
        for (int r = 0; r < 3; ++r) k_philox_rate<<<blocks, kRateThreads, 0, st>>>(seed + r, iters, sink);
        cudaEventRecord(b, st);
        const cudaError_t e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
            rc = fail(FBPT_ECUDA, "fbpt_philox_rate: timing failed");
        else
            *calls_per_s = 3.0 * (double)blocks * kRateThreads * 2.0 * iters / (ms * 1e-3);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFreeAsync(sink, st);
    cudaStreamSynchronize(st);
    return rc;
}
