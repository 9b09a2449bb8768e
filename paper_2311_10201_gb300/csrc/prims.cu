// Device-wide primitives used by the sampler and the graph builder: exclusive
// scans and a stable LSD radix sort of 64-bit keys.  Three-phase designs
// (reduce, scan, apply): no kernel ever waits on another CTA.
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

// ---- radix sort ---------------------------------------------------------------------

constexpr int kRsWarps = 8;
constexpr int kRsThreads = kRsWarps * 32;
constexpr int kRsSteps = 16;                       // 32-key steps per warp
constexpr uint64_t kRsTile = (uint64_t)kRsThreads * kRsSteps;

__global__ void __launch_bounds__(kRsThreads) k_rs_hist(const uint64_t* keys, uint64_t n, uint32_t shift,
                                                        uint32_t nblocks, uint32_t* hist) {
    __shared__ uint32_t s_cnt[256];
    s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
    for (uint32_t i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        const uint64_t k = base + i;
        if (k < n) atomicAdd(&s_cnt[(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * nblocks + blockIdx.x] = s_cnt[threadIdx.x];
}

// Stable scatter: warp w of block b owns keys [b*tile + w*512, +512) and walks
// them in order; equal digits are ranked with match_any within each 32-key step.
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const uint64_t* in, uint64_t* out, uint64_t n,
                                                           uint32_t shift, uint32_t nblocks, const uint64_t* off) {
    __shared__ uint32_t s_w[kRsWarps][256];
    __shared__ uint64_t s_off[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) (&s_w[0][0])[i] = 0;
    __syncthreads();
    const uint64_t wbase = (uint64_t)blockIdx.x * kRsTile + (uint64_t)warp * (32 * kRsSteps);
    const uint32_t lt = lanemask_lt();
    // A: per-warp digit counts
    for (int step = 0; step < kRsSteps; ++step) {
        const uint64_t k = wbase + (uint64_t)step * 32 + lane;
        const bool ok = k < n;
        const uint32_t d = ok ? (uint32_t)((in[k] >> shift) & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (ok && (peers & lt) == 0) s_w[warp][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // B: per-warp bases relative to the block's digit offsets
    {
        const uint32_t d = threadIdx.x;  // 256 threads = 256 digits
        s_off[d] = off[(uint64_t)d * nblocks + blockIdx.x];
        uint32_t run = 0;
        for (int w = 0; w < kRsWarps; ++w) {
            const uint32_t c = s_w[w][d];
            s_w[w][d] = run;
            run += c;
        }
    }
    __syncthreads();
    // C: scatter in order
    for (int step = 0; step < kRsSteps; ++step) {
        const uint64_t k = wbase + (uint64_t)step * 32 + lane;
        const bool ok = k < n;
        const uint64_t key = ok ? in[k] : 0;
        const uint32_t d = ok ? (uint32_t)((key >> shift) & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t rel = 0;
        if (ok) rel = s_w[warp][d];
        __syncwarp();
        if (ok) {
            const uint64_t pos = s_off[d] + rel + __popc(peers & lt);
            out[pos] = key;
            if ((peers & lt) == 0) s_w[warp][d] = rel + __popc(peers);
        }
        __syncwarp();
    }
}

}  // namespace

int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    return scan_impl<uint32_t>(in, out, n, st);
}

int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
    return scan_impl<uint64_t>(in, out, n, st);
}

int radix_sort_u64(uint64_t* keys, uint64_t* tmp, uint64_t n, uint32_t bits, cudaStream_t st) {
    if (n <= 1 || bits == 0) return FBPT_OK;
    const uint64_t nb64 = (n + kRsTile - 1) / kRsTile;
    if (nb64 > 0xFFFFFFFFull / 256) return fail(FBPT_EUNSUPPORTED, "radix sort: too many keys");
    const uint32_t nb = (uint32_t)nb64;
    uint32_t* hist = nullptr;
    uint64_t* off = nullptr;
    if (cudaMallocAsync(&hist, sizeof(uint32_t) * 256ull * nb, st) != cudaSuccess ||
        cudaMallocAsync(&off, sizeof(uint64_t) * (256ull * nb + 1), st) != cudaSuccess) {
        if (hist) cudaFreeAsync(hist, st);
        cudaGetLastError();
        return fail(FBPT_ENOMEM, "radix sort: scratch allocation failed");
    }
    uint64_t* a = keys;
    uint64_t* b = tmp;
    int rc = FBPT_OK;
    for (uint32_t shift = 0; shift < bits && rc == FBPT_OK; shift += 8) {
        k_rs_hist<<<nb, kRsThreads, 0, st>>>(a, n, shift, nb, hist);
        rc = exclusive_scan_u32(hist, off, 256ull * nb, st);
        if (rc != FBPT_OK) break;
        k_rs_scatter<<<nb, kRsThreads, 0, st>>>(a, b, n, shift, nb, off);
        if (cudaGetLastError() != cudaSuccess) rc = fail(FBPT_ECUDA, "radix sort launch failed");
        uint64_t* t = a;
        a = b;
        b = t;
    }
    if (rc == FBPT_OK && a != keys)
        if (cudaMemcpyAsync(keys, a, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
            rc = fail(FBPT_ECUDA, "radix sort copy failed");
    cudaFreeAsync(hist, st);
    cudaFreeAsync(off, st);
    return rc;
}

}  // namespace fbpt
