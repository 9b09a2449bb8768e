// Device-wide exclusive scans used by the sampler and the graph builder.
// Three-phase (reduce, scan, apply): no kernel ever waits on another CTA.
#include "internal.cuh"

namespace fbpt {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr uint64_t kScanTile = (uint64_t)kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* s_warp, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T incl = warp_incl_scan(v);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nwarps = blockDim.x >> 5;
        T x = lane < nwarps ? s_warp[lane] : T(0);
        const T xi = warp_incl_scan(x);
        if (lane < nwarps) s_warp[lane] = xi - x;
        if (lane == 31) *total = xi;
    }
    __syncthreads();
    return s_warp[warp] + incl - v;
}

template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_block_sums(const Tin* in, uint64_t n, uint64_t* sums) {
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) s += (uint64_t)in[base + i];
    s = warp_sum(s);
    __shared__ uint64_t s_w[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint64_t x = threadIdx.x < kScanThreads / 32 ? s_w[threadIdx.x] : 0;
        x = warp_sum(x);
        if (threadIdx.x == 0) sums[blockIdx.x] = x;
    }
}

// out[i] = block_off[b] + exclusive prefix within the tile; out[n] = grand total
// (written by the thread holding element n-1).
template <typename Tin>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const Tin* in, uint64_t n, const uint64_t* block_off,
                                                             uint64_t* out) {
    __shared__ uint64_t s_warp[kScanThreads / 32];
    __shared__ uint64_t s_total;
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t v[kScanItems];
    uint64_t t = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? (uint64_t)in[base + i] : 0;
        t += v[i];
    }
    uint64_t off = block_excl_scan<uint64_t>(t, s_warp, &s_total);
    if (block_off) off += block_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = off;
        off += v[i];
        if (base + i + 1 == n) out[n] = off;
    }
}

template <typename Tin>
int scan_impl(const Tin* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    if (n == 0) {
        FBPT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
        return FBPT_OK;
    }
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_scan_apply<Tin><<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        FBPT_CUDA_TRY(cudaGetLastError());
        return FBPT_OK;
    }
    uint64_t* sums = nullptr;
    FBPT_CUDA_TRY(cudaMallocAsync(&sums, sizeof(uint64_t) * (2 * nb + 1), st));
    uint64_t* offs = sums + nb;
    k_block_sums<Tin><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    int rc = scan_impl<uint64_t>(sums, offs, nb, st);
    if (rc == FBPT_OK) {
        k_scan_apply<Tin><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, offs, out);
        if (cudaGetLastError() != cudaSuccess) rc = fail(FBPT_ECUDA, "scan launch failed");
    }
    cudaFreeAsync(sums, st);
    return rc;
}

}  // namespace

int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    return scan_impl<uint32_t>(in, out, n, st);
}

int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    return scan_impl<uint64_t>(in, out, n, st);
}

}  // namespace fbpt
