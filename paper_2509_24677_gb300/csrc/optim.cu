// a11: Adam on the FP32 master parameters (Sec. 4.2: Adam, learning rate 1e-3, "decay" 1e-10,
// read as L2 weight decay added to the gradient; beta1, beta2 and epsilon are not given in the
// paper and default to 0.9, 0.999, 1e-8).
//
// The step counter lives on the device so that a captured training step can be replayed: every
// CTA reads t = state[0] + 1, and the last CTA to finish stores t back. The BF16 tensor-core
// weights are produced from the updated master copy by npvs_pack_weights.
#include "common.cuh"

namespace npvs {
namespace {

__global__ void __launch_bounds__(256) adam_kernel(float* __restrict__ theta, const float* __restrict__ grad,
                                                   float* __restrict__ m, float* __restrict__ v, long long n,
                                                   npvs_adam_params prm, int32_t* __restrict__ state) {
    pdl_begin();
    __shared__ float s_c1, s_c2;
    __shared__ bool last;
    if (threadIdx.x == 0) {
        const int t = state[0] + 1;
        s_c1 = (float)(1.0 / (1.0 - pow((double)prm.beta1, (double)t)));
        s_c2 = (float)(1.0 / (1.0 - pow((double)prm.beta2, (double)t)));
    }
    __syncthreads();
    const float c1 = s_c1, c2 = s_c2;
    const float b1 = prm.beta1, b2 = prm.beta2;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float th = theta[i];
        const float g = grad[i] + prm.weight_decay * th;
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        theta[i] = th - prm.lr * (mi * c1) / (sqrtf(vi * c2) + prm.eps);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(reinterpret_cast<unsigned int*>(state + 1), 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        state[0] = state[0] + 1;
        state[1] = 0;
    }
}

}  // namespace
}  // namespace npvs

using namespace npvs;

extern "C" npvs_status npvs_adam_step(float* theta, const float* grad, float* m, float* v, int64_t n,
                                      const npvs_adam_params* prm, int32_t* state, void* stream) {
    NPVS_REQUIRE(theta && grad && m && v && prm && state && n >= 0, NPVS_ERR_INVALID_ARG, "npvs_adam_step: bad arguments");
    NPVS_REQUIRE(prm->beta1 >= 0.0f && prm->beta1 < 1.0f && prm->beta2 >= 0.0f && prm->beta2 < 1.0f,
                 NPVS_ERR_INVALID_ARG, "npvs_adam_step: betas must lie in [0, 1)");
    if (n == 0) return NPVS_OK;
    const int grid = std::max(1, std::min(ceil_div(n, 256), kNumSMs * 8));
    launch_k(adam_kernel, grid, 256, 0, as_stream(stream), theta, grad, m, v, (long long)n, *prm, state);
    return check_launch("adam_kernel");
}
