// Gradients with respect to the scalar parameters lambda and v, from the
// per-element terms the reverse sweep leaves (dL/dlambda: each element's
// adjoint times d c / d lambda of its parent edge, summed over the pass
// applications; dL/dv: M * G0 with G0 the adjoint of D0 = v M), summed in
// float64 by a fixed-shape two-stage tree (512 contiguous ranges, 256 strided
// partials each, then pairwise trees) so that every run, on any GPU, gives
// the same bits.
#include <cuda_runtime.h>

#include <algorithm>

#include "fgx_internal.h"

namespace fgx {
namespace {

constexpr int kSumBlocks = 512;   // partial sums per term (fixed: the bits do not depend on the GPU)
constexpr int kSumThreads = 256;

__global__ void __launch_bounds__(256) v_terms_kernel(const float* mask, const float* g0,
                                                      float* v_terms, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        v_terms[i] = __fmul_rn(mask[i], g0[i]);
}

// Pairwise tree over the first `count` (a power of two) doubles of part.
__device__ __forceinline__ void tree_sum(double* part, int count) {
    for (int stride = count / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
            part[threadIdx.x] = __dadd_rn(part[threadIdx.x], part[threadIdx.x + stride]);
        __syncthreads();
    }
}

// Stage 1 (blockIdx.y = term): block b sums the contiguous range b of
// kSumBlocks equal ranges; thread j adds elements j, j + 256, ... of the
// range in order in float64, then a pairwise tree over the 256 partials.
__global__ void __launch_bounds__(kSumThreads) sum_terms_kernel(const float* t0, const float* t1,
                                                                double* partials, int64_t n) {
    __shared__ double part[kSumThreads];
    const float* t = blockIdx.y == 0 ? t0 : t1;
    if (!t) return;  // uniform over the block
    const int64_t chunk = (n + kSumBlocks - 1) / kSumBlocks;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(n, lo + chunk);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kSumThreads) acc = __dadd_rn(acc, (double)t[i]);
    part[threadIdx.x] = acc;
    __syncthreads();
    tree_sum(part, kSumThreads);
    if (threadIdx.x == 0) partials[blockIdx.y * kSumBlocks + blockIdx.x] = part[0];
}

// Stage 2 (blockIdx.x = term): a pairwise tree over the kSumBlocks partials.
__global__ void __launch_bounds__(kSumBlocks) sum_partials_kernel(const double* partials,
                                                                  double* out0, double* out1) {
    __shared__ double part[kSumBlocks];
    double* out = blockIdx.x == 0 ? out0 : out1;
    if (!out) return;  // uniform over the block
    part[threadIdx.x] = partials[blockIdx.x * kSumBlocks + threadIdx.x];
    __syncthreads();
    tree_sum(part, kSumBlocks);
    if (threadIdx.x == 0) *out = part[0];
}

}  // namespace

size_t param_partials_bytes() { return 2 * (size_t)kSumBlocks * sizeof(double); }

int run_param_sums(const float* mask, const float* g0, float* v_terms, const float* lambda_terms,
                   double* grad_lambda, double* grad_v, double* partials, int64_t n, int sms,
                   void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8));
        v_terms_kernel<<<grid, 256, 0, s>>>(mask, g0, v_terms, n);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    if (grad_lambda || grad_v) {
        sum_terms_kernel<<<dim3(kSumBlocks, 2), kSumThreads, 0, s>>>(
            grad_lambda ? lambda_terms : nullptr, grad_v ? v_terms : nullptr, partials, n);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
        sum_partials_kernel<<<2, kSumBlocks, 0, s>>>(partials, grad_lambda, grad_v);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

}  // namespace fgx

