// Gradients with respect to the scalar parameters lambda and v, from the
// per-element terms the reverse sweep leaves (dL/dlambda: each element's
// adjoint times d c / d lambda of its parent edge, summed over the pass
// applications; dL/dv: M * G0 with G0 the adjoint of D0 = v M), summed in
// float64 by a fixed-shape tree so that every run gives the same bits.
#include <cuda_runtime.h>

#include <algorithm>

#include "fgx_internal.h"

namespace fgx {
namespace {

constexpr int kSumThreads = 1024;

__global__ void __launch_bounds__(256) v_terms_kernel(const float* mask, const float* g0,
                                                      float* v_terms, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v_terms[i] = __fmul_rn(mask[i], g0[i]);
}

// Block 0 sums terms[0], block 1 terms[1]: thread j adds elements j, j + 1024,
// ... in order in float64, then a pairwise tree over the 1024 partial sums.
__global__ void __launch_bounds__(kSumThreads) sum_terms_kernel(const float* t0, const float* t1,
                                                                double* out0, double* out1,
                                                                int64_t n) {
    __shared__ double part[kSumThreads];
    const float* t = blockIdx.x == 0 ? t0 : t1;
    double* out = blockIdx.x == 0 ? out0 : out1;
    if (!t || !out) return;  // uniform over the block
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kSumThreads) acc = __dadd_rn(acc, (double)t[i]);
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int stride = kSumThreads / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
            part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + stride]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

}  // namespace

int run_param_sums(const float* mask, const float* g0, float* v_terms, const float* lambda_terms,
                   double* grad_lambda, double* grad_v, int64_t n, int sms, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8));
        v_terms_kernel<<<grid, 256, 0, s>>>(mask, g0, v_terms, n);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    if (grad_lambda || grad_v) {
        sum_terms_kernel<<<2, kSumThreads, 0, s>>>(lambda_terms, v_terms, grad_lambda, grad_v, n);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

}  // namespace fgx

