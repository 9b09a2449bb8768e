// The IMM sampling loop (Tang, Shi and Xiao, SIGMOD 2015), the consumer of the
// sampler that Section 2 describes: estimate a lower bound LB on the optimum
// influence from growing samples, fix theta = ceil(lambda* / LB) RR sets, run
// greedy max-k-cover over them.  The loop is host logic; every sampling step is
// sample_impl and every selection fbpt_select_seeds.  The estimation sample
// grows by appending the RR sets of the next sample ids, never redrawing
// earlier ones; the final selection runs over theta RR sets drawn afresh, with
// the sample ids after the estimation's (Chen 2018: reusing the estimation sets
// breaks the martingale argument behind IMM's guarantee).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace fbpt {
namespace {

__global__ void k_shift_offsets(const uint64_t* src, uint64_t count, uint64_t shift, uint64_t* dst) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + shift;
}

__global__ void k_add_counts(uint32_t* acc, const uint32_t* add, uint64_t n) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        acc[i] += add[i];
}

// acc <- acc ++ add (rows of add after those of acc); add is released.
int rr_append(fbpt_rrsets* acc, fbpt_rrsets* add) {
    if (!acc->offsets) {
        *acc = *add;
        std::memset(add, 0, sizeof(*add));
        return FBPT_OK;
    }
    cudaStream_t st = (cudaStream_t)acc->stream;
    const uint64_t S = acc->S + add->S, total = acc->total + add->total;
    uint64_t* off = nullptr;
    uint32_t *verts = nullptr, *starts = nullptr;
    auto undo = [&](const char* what) {
        if (off) cudaFreeAsync(off, st);
        if (verts) cudaFreeAsync(verts, st);
        if (starts) cudaFreeAsync(starts, st);
        cudaGetLastError();
        return fail(FBPT_ENOMEM, std::string("fbpt_imm: ") + what);
    };
    if (cudaMallocAsync(&off, sizeof(uint64_t) * (S + 1), st) != cudaSuccess) return undo("offsets");
    if (cudaMallocAsync(&verts, sizeof(uint32_t) * std::max<uint64_t>(total, 1), st) != cudaSuccess)
        return undo("vertices");
    if (cudaMallocAsync(&starts, sizeof(uint32_t) * S, st) != cudaSuccess) return undo("starts");
    const int blocks = device_sm_count() * 4;
    bool ok = cudaMemcpyAsync(off, acc->offsets, sizeof(uint64_t) * acc->S, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
    if (ok) k_shift_offsets<<<blocks, 256, 0, st>>>(add->offsets, add->S + 1, acc->total, off + acc->S);
    if (ok && acc->total)
        ok = cudaMemcpyAsync(verts, acc->verts, sizeof(uint32_t) * acc->total, cudaMemcpyDeviceToDevice, st) ==
             cudaSuccess;
    if (ok && add->total)
        ok = cudaMemcpyAsync(verts + acc->total, add->verts, sizeof(uint32_t) * add->total, cudaMemcpyDeviceToDevice,
                             st) == cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(starts, acc->starts, sizeof(uint32_t) * acc->S, cudaMemcpyDeviceToDevice, st) ==
                 cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(starts + acc->S, add->starts, sizeof(uint32_t) * add->S, cudaMemcpyDeviceToDevice,
                                 st) == cudaSuccess;
    if (ok) k_add_counts<<<blocks, 256, 0, st>>>(acc->vcount, add->vcount, acc->n);
    if (!ok || cudaGetLastError() != cudaSuccess) {
        cudaStreamSynchronize(st);  // nothing queued may still touch the buffers freed below
        return undo("device copies");
    }
    cudaFreeAsync(acc->offsets, st);
    cudaFreeAsync(acc->verts, st);
    cudaFreeAsync(acc->starts, st);
    acc->offsets = off;
    acc->verts = verts;
    acc->starts = starts;
    acc->S = S;
    acc->total = total;
    fbpt_rrsets_free(add);
    return FBPT_OK;
}

// ln C(n, k) as the sum over i < min(k, n - k) of ln((n - i) / (i + 1)), in
// that order (each quotient is exact-input, correctly rounded).
double log_binom(double n, double k) {
    const double kk = std::min(k, n - k);
    double s = 0.0;
    for (double i = 0.0; i < kk; i += 1.0) s += std::log((n - i) / (i + 1.0));
    return s;
}

}  // namespace

int imm_impl(fbpt_graph* g, uint32_t k, double epsilon, double ell, uint64_t seed, uint64_t max_samples,
             const fbpt_opts* opts, uint32_t* seeds_host, uint64_t* gains_host, fbpt_imm_result* result,
             fbpt_stats* stats) {
    if (!g) return fail(FBPT_EINVAL, "fbpt_imm: null graph");
    if (g->n < 2) return fail(FBPT_EINVAL, "fbpt_imm: needs n >= 2");
    if (k < 1 || k > g->n) return fail(FBPT_EINVAL, "fbpt_imm: needs 1 <= k <= n");
    if (!(epsilon > 0.0) || !(ell > 0.0)) return fail(FBPT_EINVAL, "fbpt_imm: needs epsilon > 0 and ell > 0");
    const double n = (double)g->n;
    const double e = 2.718281828459045;  // Euler's number (the double nearest e)
    const double ln_n = std::log(n);
    const double ellp = ell * (1.0 + std::log(2.0) / ln_n);
    const double epsp = std::sqrt(2.0) * epsilon;
    const double L = log_binom(n, (double)k);
    const double lam_p = (2.0 + 2.0 * epsp / 3.0) * (L + ellp * ln_n + std::log(std::log2(n))) * n / (epsp * epsp);
    const double alpha = std::sqrt(ellp * ln_n + std::log(2.0));
    const double beta = std::sqrt((1.0 - 1.0 / e) * (L + ellp * ln_n + std::log(2.0)));
    const double ab = (1.0 - 1.0 / e) * alpha + beta;
    const double lam_s = 2.0 * n * ab * ab / (epsilon * epsilon);

    fbpt_rrsets R;
    std::memset(&R, 0, sizeof(R));
    uint64_t have = 0;
    std::vector<uint32_t> seeds(k);
    std::vector<uint64_t> gains(k);
    auto extend = [&](uint64_t target) -> int {
        if (target <= have) return FBPT_OK;
        if (max_samples && target > max_samples)
            return fail(FBPT_EINVAL, "fbpt_imm: the sample needs " + std::to_string(target) +
                                         " RR sets, above max_samples");
        fbpt_rrsets add;
        FBPT_TRY(sample_impl(g, seed, have, target - have, opts, &add, stats));
        const int rc = rr_append(&R, &add);
        if (rc != FBPT_OK) {
            fbpt_rrsets_free(&add);
            return rc;
        }
        have = target;
        return FBPT_OK;
    };
    auto covered = [&]() -> double {
        uint64_t c = 0;
        for (uint32_t i = 0; i < k; ++i) c += gains[i];
        return (double)c / (double)have;
    };
    int rc = FBPT_OK;
    double LB = 1.0;
    uint32_t rounds = 0;
    const int last = (int)std::ceil(std::log2(n)) - 1;
    for (int i = 1; i <= last && rc == FBPT_OK; ++i) {
        const double x = n / std::ldexp(1.0, i);
        rc = extend((uint64_t)std::ceil(lam_p / x));
        if (rc == FBPT_OK) rc = fbpt_select_seeds(&R, k, seeds.data(), gains.data());
        if (rc != FBPT_OK) break;
        rounds = (uint32_t)i;
        const double F = covered();
        if (n * F >= (1.0 + epsp) * x) {
            LB = n * F / (1.0 + epsp);
            break;
        }
    }
    const uint64_t theta = (uint64_t)std::ceil(lam_s / LB);
    const uint64_t first_final = have;
    fbpt_rrsets Fin;
    std::memset(&Fin, 0, sizeof(Fin));
    if (rc == FBPT_OK && max_samples && theta > max_samples)
        rc = fail(FBPT_EINVAL, "fbpt_imm: the final sample needs " + std::to_string(theta) +
                                   " RR sets, above max_samples");
    fbpt_rrsets_free(&R);
    if (rc == FBPT_OK) rc = sample_impl(g, seed, first_final, theta, opts, &Fin, stats);
    if (rc == FBPT_OK) {
        have = theta;
        rc = fbpt_select_seeds(&Fin, k, seeds.data(), gains.data());
    }
    if (rc == FBPT_OK) {
        if (seeds_host) std::memcpy(seeds_host, seeds.data(), sizeof(uint32_t) * k);
        if (gains_host) std::memcpy(gains_host, gains.data(), sizeof(uint64_t) * k);
        if (result) {
            std::memset(result, 0, sizeof(*result));
            result->theta = theta;
            result->samples = have;
            result->lower_bound = LB;
            result->coverage = covered();
            result->lambda_prime = lam_p;
            result->lambda_star = lam_s;
            result->rounds = rounds;
            result->first_final_id = first_final;
        }
    }
    fbpt_rrsets_free(&Fin);
    return rc;
}

}  // namespace fbpt
