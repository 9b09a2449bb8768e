// The schedule policy network: parameters on the device (fbpt_policy) and its
// training kernels.  The network is used by the level scheduler (engine.cu,
// policy_forward) to pick how the coming level expands; it never changes a bit
// of the output.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace fbpt;

extern "C" int fbpt_policy_param_count(void) { return 2 * kPolicyIn + kPolicyParams; }

extern "C" int fbpt_policy_create(const float* params, uint64_t count, fbpt_policy** out) {
    if (!out) return fail(FBPT_EINVAL, "fbpt_policy_create: out is NULL");
    *out = nullptr;
    const uint64_t want = 2 * kPolicyIn + kPolicyParams;
    if (!params || count != want)
        return fail(FBPT_EINVAL, "fbpt_policy_create: needs " + std::to_string(want) + " parameters");
    for (int i = 0; i < kPolicyIn; ++i)
        if (!(params[kPolicyIn + i] > 0.f)) return fail(FBPT_EINVAL, "fbpt_policy_create: input scales must be > 0");
    fbpt_policy* p = new fbpt_policy();
    std::memcpy(p->h_params, params, sizeof(float) * want);
    if (cudaMalloc(&p->d_params, sizeof(float) * want) != cudaSuccess ||
        cudaMemcpy(p->d_params, params, sizeof(float) * want, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p->d_params);
        delete p;
        cudaGetLastError();
        return fail(FBPT_ENOMEM, "fbpt_policy_create: device copy failed");
    }
    *out = p;
    return FBPT_OK;
}

extern "C" int fbpt_policy_destroy(fbpt_policy* p) {
    if (!p) return FBPT_OK;
    cudaFree(p->d_params);
    delete p;
    return FBPT_OK;
}

extern "C" int fbpt_policy_get(const fbpt_policy* p, float* params, uint64_t count) {
    const uint64_t want = 2 * kPolicyIn + kPolicyParams;
    if (!p || !params || count != want) return fail(FBPT_EINVAL, "fbpt_policy_get: bad arguments");
    std::memcpy(params, p->h_params, sizeof(float) * want);
    return FBPT_OK;
}

extern "C" int fbpt_policy_save(const fbpt_policy* p, const char* path) {
    if (!p || !path) return fail(FBPT_EINVAL, "fbpt_policy_save: null argument");
    FILE* f = std::fopen(path, "w");
    if (!f) return fail(FBPT_EINVAL, std::string("fbpt_policy_save: cannot write ") + path);
    const uint64_t want = 2 * kPolicyIn + kPolicyParams;
    bool ok = true;
    for (uint64_t i = 0; i < want && ok; ++i) ok = std::fprintf(f, "%.9g\n", (double)p->h_params[i]) > 0;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? FBPT_OK : fail(FBPT_EINVAL, std::string("fbpt_policy_save: write failed on ") + path);
}

extern "C" int fbpt_policy_load(const char* path, fbpt_policy** out) {
    if (!path || !out) return fail(FBPT_EINVAL, "fbpt_policy_load: null argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(FBPT_EINVAL, std::string("fbpt_policy_load: cannot read ") + path);
    const uint64_t want = 2 * kPolicyIn + kPolicyParams;
    std::vector<float> v;
    char tok[64];
    bool bad = false;
    while (std::fscanf(f, "%63s", tok) == 1) {
        char* end = nullptr;
        const float x = std::strtof(tok, &end);
        if (end == tok || *end != '\0') {
            bad = true;
            break;
        }
        v.push_back(x);
        if (v.size() > want) break;
    }
    std::fclose(f);
    if (bad) return fail(FBPT_EINVAL, std::string("fbpt_policy_load: not a number in ") + path);
    if (v.size() != want)
        return fail(FBPT_EINVAL, "fbpt_policy_load: expected " + std::to_string(want) + " numbers in " + path);
    return fbpt_policy_create(v.data(), want, out);
}

// ---- training ----------------------------------------------------------------------
//
// Rows are levels from traces: six features, the action the level ran with and
// its log2 device time.  Loss: mean over rows of (out[action] - target)^2; only
// the taken action's output gets a gradient.  Full-batch Adam (Kingma and Ba,
// ICLR 2015) on the weights and biases; the input mean and scale stay fixed.

namespace fbpt {
namespace {

constexpr int kNP = 2 * kPolicyIn + kPolicyParams;  // 1,556 floats
constexpr int kOffW1 = 2 * kPolicyIn;
constexpr int kOffB1 = kOffW1 + kPolicyIn * kPolicyHidden;
constexpr int kOffW2 = kOffB1 + kPolicyHidden;
constexpr int kOffB2 = kOffW2 + kPolicyHidden * kPolicyHidden;
constexpr int kOffW3 = kOffB2 + kPolicyHidden;
constexpr int kOffB3 = kOffW3 + kPolicyHidden * kPolicyOut;

// One thread per row: forward, loss term and backpropagation, the gradient
// summed in shared memory and then added to `grad`.
__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                  const uint32_t* __restrict__ act, const float* __restrict__ Y,
                                                  uint64_t rows, float* grad, float* loss) {
    __shared__ float w[kNP];
    __shared__ float g[kNP];
    for (int i = threadIdx.x; i < kNP; i += blockDim.x) {
        w[i] = P[i];
        g[i] = 0.f;
    }
    __syncthreads();
    const float inv = 2.0f / (float)rows;
    float lsum = 0.f;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (uint64_t)gridDim.x * blockDim.x) {
        float xn[kPolicyIn], h1[kPolicyHidden], h2[kPolicyHidden];
        for (int k = 0; k < kPolicyIn; ++k) xn[k] = (X[r * kPolicyIn + k] - w[k]) / w[kPolicyIn + k];
        for (int j = 0; j < kPolicyHidden; ++j) {
            float s = w[kOffB1 + j];
            for (int k = 0; k < kPolicyIn; ++k) s += w[kOffW1 + j * kPolicyIn + k] * xn[k];
            h1[j] = s > 0.f ? s : 0.f;
        }
        for (int j = 0; j < kPolicyHidden; ++j) {
            float s = w[kOffB2 + j];
            for (int k = 0; k < kPolicyHidden; ++k) s += w[kOffW2 + j * kPolicyHidden + k] * h1[k];
            h2[j] = s > 0.f ? s : 0.f;
        }
        const uint32_t a = act[r] < (uint32_t)kPolicyOut ? act[r] : 0u;
        float o = w[kOffB3 + a];
        for (int k = 0; k < kPolicyHidden; ++k) o += w[kOffW3 + a * kPolicyHidden + k] * h2[k];
        const float res = o - Y[r];
        lsum += res * res;
        const float d = inv * res;
        atomicAdd(&g[kOffB3 + a], d);
        float da2[kPolicyHidden];
        for (int k = 0; k < kPolicyHidden; ++k) {
            atomicAdd(&g[kOffW3 + a * kPolicyHidden + k], d * h2[k]);
            da2[k] = h2[k] > 0.f ? d * w[kOffW3 + a * kPolicyHidden + k] : 0.f;
        }
        for (int j = 0; j < kPolicyHidden; ++j) {
            if (da2[j] == 0.f) continue;
            atomicAdd(&g[kOffB2 + j], da2[j]);
            for (int k = 0; k < kPolicyHidden; ++k)
                if (h1[k] > 0.f) atomicAdd(&g[kOffW2 + j * kPolicyHidden + k], da2[j] * h1[k]);
        }
        for (int k = 0; k < kPolicyHidden; ++k) {
            if (h1[k] <= 0.f) continue;
            float s = 0.f;
            for (int j = 0; j < kPolicyHidden; ++j) s += da2[j] * w[kOffW2 + j * kPolicyHidden + k];
            if (s == 0.f) continue;
            atomicAdd(&g[kOffB1 + k], s);
            for (int q = 0; q < kPolicyIn; ++q) atomicAdd(&g[kOffW1 + k * kPolicyIn + q], s * xn[q]);
        }
    }
    lsum = warp_sum(lsum);
    if (lane_id() == 0 && lsum != 0.f) atomicAdd(loss, lsum / (float)rows);
    __syncthreads();
    for (int i = kOffW1 + threadIdx.x; i < kNP; i += blockDim.x)
        if (g[i] != 0.f) atomicAdd(&grad[i], g[i]);
}

// One Adam step (Kingma and Ba, ICLR 2015, Algorithm 1: beta1 = 0.9, beta2 =
// 0.999, eps = 1e-8) on the weights and biases; the input mean and scale
// (the first 12 floats) are not trained.
// The decay factors and their complements are each the float nearest to the
// decimal constant (1 - 0.999f would be 1.3e-5 away from 0.001), and the bias
// corrections 1 - beta^t are formed as -expm1(t log1p(-(1 - beta))), which
// keeps their relative error at a few float ulps for every t.
__global__ void k_adam(float* P, const float* grad, float* m, float* v, int t, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, omb1 = 0.1f, omb2 = 0.001f, eps = 1e-8f;
    const float c1 = -expm1f((float)t * log1pf(-omb1)), c2 = -expm1f((float)t * log1pf(-omb2));
    for (int i = kOffW1 + blockIdx.x * blockDim.x + threadIdx.x; i < kNP; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + omb1 * gi;
        const float vi = b2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Device buffers of one training call, allocated and freed on its stream.
struct TrainBufs {
    cudaStream_t st = nullptr;
    float *P = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr, *X = nullptr, *Y = nullptr;
    uint32_t* A = nullptr;
    explicit TrainBufs(cudaStream_t s) : st(s) {}
    ~TrainBufs() {
        for (void* p : {(void*)P, (void*)grad, (void*)m, (void*)v, (void*)loss, (void*)X, (void*)Y, (void*)A})
            if (p) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    }
};

// Parameters (and, with rows > 0, the trace rows) to the device; Adam moments zeroed.
int upload(TrainBufs& b, const float* params, const float* X, const uint32_t* A, const float* Y, uint64_t rows) {
    const cudaStream_t st = b.st;
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.P, sizeof(float) * kNP, st));
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.grad, sizeof(float) * kNP, st));
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.m, sizeof(float) * kNP, st));
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.v, sizeof(float) * kNP, st));
    FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.loss, sizeof(float), st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(b.P, params, sizeof(float) * kNP, cudaMemcpyHostToDevice, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(b.m, 0, sizeof(float) * kNP, st));
    FBPT_CUDA_TRY(cudaMemsetAsync(b.v, 0, sizeof(float) * kNP, st));
    if (rows) {
        FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.X, sizeof(float) * kPolicyIn * rows, st));
        FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.Y, sizeof(float) * rows, st));
        FBPT_CUDA_TRY(cudaMallocAsync((void**)&b.A, sizeof(uint32_t) * rows, st));
        FBPT_CUDA_TRY(cudaMemcpyAsync(b.X, X, sizeof(float) * kPolicyIn * rows, cudaMemcpyHostToDevice, st));
        FBPT_CUDA_TRY(cudaMemcpyAsync(b.Y, Y, sizeof(float) * rows, cudaMemcpyHostToDevice, st));
        FBPT_CUDA_TRY(cudaMemcpyAsync(b.A, A, sizeof(uint32_t) * rows, cudaMemcpyHostToDevice, st));
    }
    return FBPT_OK;
}

int grad_pass(TrainBufs& b, uint64_t rows) {
    FBPT_CUDA_TRY(cudaMemsetAsync(b.grad, 0, sizeof(float) * kNP, b.st));
    FBPT_CUDA_TRY(cudaMemsetAsync(b.loss, 0, sizeof(float), b.st));
    const int blocks = (int)std::min<uint64_t>((rows + 255) / 256, (uint64_t)device_sm_count() * 2);
    k_mlp_grad<<<std::max(blocks, 1), 256, 0, b.st>>>(b.P, b.X, b.A, b.Y, rows, b.grad, b.loss);
    FBPT_CUDA_TRY(cudaGetLastError());
    return FBPT_OK;
}

// Deterministic initial weights: He-scaled normals from SplitMix64 + Box-Muller.
uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double normal01(uint64_t& s) {
    const double u1 = ((splitmix(s) >> 11) + 0.5) / 9007199254740992.0;
    const double u2 = ((splitmix(s) >> 11) + 0.5) / 9007199254740992.0;
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace
}  // namespace fbpt

extern "C" int fbpt_policy_loss_grad(const float* params, const float* features, const uint32_t* actions,
                                     const float* targets, uint64_t rows, float* loss, float* grad, void* stream) {
    if (!params || !features || !actions || !targets || rows == 0 || !loss || !grad)
        return fail(FBPT_EINVAL, "fbpt_policy_loss_grad: bad arguments");
    TrainBufs b((cudaStream_t)stream);
    FBPT_TRY(upload(b, params, features, actions, targets, rows));
    FBPT_TRY(grad_pass(b, rows));
    FBPT_CUDA_TRY(cudaMemcpyAsync(grad, b.grad, sizeof(float) * kNP, cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(loss, b.loss, sizeof(float), cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaStreamSynchronize(b.st));
    for (int i = 0; i < kOffW1; ++i) grad[i] = 0.f;
    return FBPT_OK;
}

extern "C" int fbpt_policy_adam_step(float* params, const float* grad, float* m, float* v, uint32_t t, float lr,
                                     void* stream) {
    if (!params || !grad || !m || !v || t == 0 || !(lr > 0.f))
        return fail(FBPT_EINVAL, "fbpt_policy_adam_step: bad arguments");
    TrainBufs b((cudaStream_t)stream);
    FBPT_TRY(upload(b, params, nullptr, nullptr, nullptr, 0));
    FBPT_CUDA_TRY(cudaMemcpyAsync(b.grad, grad, sizeof(float) * kNP, cudaMemcpyHostToDevice, b.st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(b.m, m, sizeof(float) * kNP, cudaMemcpyHostToDevice, b.st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(b.v, v, sizeof(float) * kNP, cudaMemcpyHostToDevice, b.st));
    k_adam<<<8, 256, 0, b.st>>>(b.P, b.grad, b.m, b.v, (int)t, lr);
    FBPT_CUDA_TRY(cudaGetLastError());
    FBPT_CUDA_TRY(cudaMemcpyAsync(params, b.P, sizeof(float) * kNP, cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(m, b.m, sizeof(float) * kNP, cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaMemcpyAsync(v, b.v, sizeof(float) * kNP, cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaStreamSynchronize(b.st));
    return FBPT_OK;
}

extern "C" int fbpt_policy_train(const float* features, const uint32_t* actions, const float* targets, uint64_t rows,
                                 const fbpt_train_opts* opts, const float* init_params, fbpt_policy** out,
                                 float* final_loss) {
    if (!features || !actions || !targets || rows == 0 || !out) return fail(FBPT_EINVAL, "fbpt_policy_train: bad arguments");
    fbpt_train_opts o = {};
    if (opts) o = *opts;
    const uint32_t steps = o.steps ? o.steps : 2000;
    const float lr = o.lr > 0.f ? o.lr : 3e-3f;
    float P[kNP];
    if (init_params) {
        std::memcpy(P, init_params, sizeof(P));
    } else {
        for (int k = 0; k < kPolicyIn; ++k) {  // input mean and scale from the data
            double s = 0, s2 = 0;
            for (uint64_t r = 0; r < rows; ++r) {
                const double x = features[r * kPolicyIn + k];
                s += x;
                s2 += x * x;
            }
            const double mu = s / rows, var = s2 / rows - mu * mu;
            P[k] = (float)mu;
            P[kPolicyIn + k] = (float)(var > 1e-6 ? std::sqrt(var) : 1.0);
        }
        uint64_t st = o.seed ^ 0x5EEDull;
        auto fill = [&](int off, int count, int fan_in) {
            const double sc = std::sqrt(2.0 / fan_in);
            for (int i = 0; i < count; ++i) P[off + i] = (float)(sc * normal01(st));
        };
        fill(kOffW1, kPolicyIn * kPolicyHidden, kPolicyIn);
        fill(kOffW2, kPolicyHidden * kPolicyHidden, kPolicyHidden);
        fill(kOffW3, kPolicyHidden * kPolicyOut, kPolicyHidden);
        for (int i = 0; i < kPolicyHidden; ++i) P[kOffB1 + i] = P[kOffB2 + i] = 0.f;
        double ym = 0;  // start the outputs at the mean target
        for (uint64_t r = 0; r < rows; ++r) ym += targets[r];
        for (int i = 0; i < kPolicyOut; ++i) P[kOffB3 + i] = (float)(ym / rows);
    }
    TrainBufs b((cudaStream_t)o.stream);
    FBPT_TRY(upload(b, P, features, actions, targets, rows));
    for (uint32_t t = 1; t <= steps; ++t) {
        FBPT_TRY(grad_pass(b, rows));
        k_adam<<<8, 256, 0, b.st>>>(b.P, b.grad, b.m, b.v, (int)t, lr);
    }
    FBPT_TRY(grad_pass(b, rows));
    FBPT_CUDA_TRY(cudaMemcpyAsync(P, b.P, sizeof(P), cudaMemcpyDeviceToHost, b.st));
    float fl = 0.f;
    FBPT_CUDA_TRY(cudaMemcpyAsync(&fl, b.loss, sizeof(float), cudaMemcpyDeviceToHost, b.st));
    FBPT_CUDA_TRY(cudaStreamSynchronize(b.st));
    if (final_loss) *final_loss = fl;
    return fbpt_policy_create(P, kNP, out);
}
