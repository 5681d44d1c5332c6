// Signed generalised geodesic distance: dist = GDT(M) - GDT(1 - M).
//
// The paper lists signed geodesic distance among the applications of the
// transform without defining it; the reading used here subtracts the
// transform seeded by the region M = 0 from the one seeded by M = 1 (the
// complement 1 - M and the difference are rounded to float32), which is
// negative inside the region M = 0, positive where M = 1, and odd under
// M -> 1 - M.  Both transforms are the library's single-call forward on the
// same stream; the workspace holds the forward's scratch, the second
// distance map and the status word of the first transform.
#include <cuda_runtime.h>

#include <algorithm>

#include "fgx_internal.h"

namespace fgx {
namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

__global__ void __launch_bounds__(256) complement_kernel(const float* mask, float* out,
                                                         int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __fsub_rn(1.0f, mask[i]);
}

// The first transform's status word, kept before the second one clears it.
__global__ void save_status_kernel(const int* status, int* saved) { *saved = *status; }

__global__ void __launch_bounds__(256) difference_kernel(float* dist, const float* other,
                                                         int64_t n, int* status,
                                                         const int* saved) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && *status == 0 && *saved != 0) *status = *saved;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dist[i] = __fsub_rn(dist[i], other[i]);
}

}  // namespace

size_t signed_workspace_bytes(size_t forward_bytes, int64_t n) {
    return al256(forward_bytes) + al256((size_t)n * sizeof(float)) + 256;
}

int run_signed(int ndim, const float* image, const float* mask, float* dist, int64_t B,
               int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
               float lambda, int iterations, void* workspace, size_t ws_bytes,
               const fgx_options* opt, void* stream) {
    size_t fwd = 0;
    int st = fgx_geodesic_workspace_size(ndim, B, C, D, H, W, opt, &fwd);
    if (st != FGX_OK) return st;
    const int64_t n = B * D * H * W;
    auto forward = [&](const float* m, float* d) {
        return ndim == 2 ? fgx_geodesic2d(image, m, d, B, C, H, W, v, lambda, iterations,
                                          workspace, fwd, opt, stream)
                         : fgx_geodesic3d(image, m, d, B, C, D, H, W, spacing, v, lambda,
                                          iterations, workspace, fwd, opt, stream);
    };
    if (n == 0) return forward(mask, dist);  // argument checks and a clean status word
    if (!workspace || ws_bytes < signed_workspace_bytes(fwd, n)) return FGX_ERR_WORKSPACE;
    if (!mask || !dist) return FGX_ERR_ARG;
    if (!device_pointer(workspace) || !device_pointer(mask)) return FGX_ERR_NOT_DEVICE_PTR;
    char* w = (char*)workspace;
    float* other = (float*)(w + al256(fwd));
    int* saved = (int*)(w + al256(fwd) + al256((size_t)n * sizeof(float)));
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FGX_ERR_CUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8));
    complement_kernel<<<grid, 256, 0, s>>>(mask, other, n);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if ((st = forward(other, other)) != FGX_OK) return st;
    save_status_kernel<<<1, 1, 0, s>>>((const int*)workspace, saved);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if ((st = forward(mask, dist)) != FGX_OK) return st;
    difference_kernel<<<grid, 256, 0, s>>>(dist, other, n, (int*)workspace, saved);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
