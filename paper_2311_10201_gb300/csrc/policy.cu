// The schedule policy network: parameters on the device (fbpt_policy) and its
// training kernels.  The network is used by the level scheduler (engine.cu,
// policy_forward) to pick how the coming level expands; it never changes a bit
// of the output.
#include <cstring>
#include <string>

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
