// Signed generalised geodesic distance: dist = GDT(M) - GDT(1 - M).
//
// The paper lists signed geodesic distance among the applications of the
// transform without defining it; the reading used here subtracts the
// transform seeded by the region M = 0 from the one seeded by M = 1 (the
// complement 1 - M and the difference are rounded to float32), which is
// negative inside the region M = 0, positive where M = 1, and odd under
// M -> 1 - M.  Both transforms of every instance run as one batched launch
// of 2B transforms of the same B images (masks [M; 1 - M]); the workspace
// holds that launch's scratch (status word first), the 2B masks and the 2B
// distance maps.
#include <cuda_runtime.h>

#include <algorithm>

#include "fgx_internal.h"

namespace fgx {
namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// masks [M; 1 - M] of the batched launch
__global__ void __launch_bounds__(256) pair_masks_kernel(const float* mask, float* out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float m = mask[i];
        out[i] = m;
        out[n + i] = __fsub_rn(1.0f, m);
    }
}

__global__ void __launch_bounds__(256) difference_kernel(float* dist, const float* pair,
                                                         int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dist[i] = __fsub_rn(pair[i], pair[n + i]);
}

}  // namespace

size_t signed_workspace_bytes(size_t forward_bytes, int64_t n) {
    return al256(forward_bytes) + 2 * al256((size_t)(2 * n) * sizeof(float));
}

int run_signed(int ndim, const float* image, const float* mask, float* dist, int64_t B,
               int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
               float lambda, int iterations, void* workspace, size_t ws_bytes,
               const fgx_options* opt, void* stream) {
    size_t fwd = 0;
    int st = fgx_geodesic_workspace_size(ndim, 2 * B, C, D, H, W, opt, &fwd);
    if (st != FGX_OK) return st;
    const int64_t n = B * D * H * W;
    if (n == 0)  // argument checks and a clean status word
        return ndim == 2 ? fgx_geodesic2d(image, mask, dist, B, C, H, W, v, lambda, iterations,
                                          workspace, ws_bytes, opt, stream)
                         : fgx_geodesic3d(image, mask, dist, B, C, D, H, W, spacing, v, lambda,
                                          iterations, workspace, ws_bytes, opt, stream);
    if (!workspace || ws_bytes < signed_workspace_bytes(fwd, n)) return FGX_ERR_WORKSPACE;
    if (!mask || !dist) return FGX_ERR_ARG;
    if (!device_pointer(workspace) || !device_pointer(mask) || !device_pointer(dist))
        return FGX_ERR_NOT_DEVICE_PTR;
    char* w = (char*)workspace;
    float* masks = (float*)(w + al256(fwd));
    float* pair = (float*)(w + al256(fwd) + al256((size_t)(2 * n) * sizeof(float)));
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FGX_ERR_CUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8));
    pair_masks_kernel<<<grid, 256, 0, s>>>(mask, masks, n);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    const float unit[3] = {1.f, 1.f, 1.f};
    st = run_forward_batch(ndim, image, B, masks, pair, 2 * B, C, ndim == 3 ? D : 1, H, W,
                           ndim == 3 ? spacing : unit, v, lambda, iterations, workspace, fwd, opt,
                           stream);
    if (st != FGX_OK) return st;
    difference_kernel<<<grid, 256, 0, s>>>(dist, pair, n);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
