// Geodesic symmetric filtering (GSF) of a segmentation indicator F.
//
// The paper names GSF among the applications of the transform without
// defining it; the reading used here composes the library's transform into
// geodesic erosion and dilation and combines them symmetrically:
//   S(X)  = GDT(1 - X) - GDT(X)              signed distance, < 0 inside X
//   F_e   = [S(F) < -theta_e],   F_d = [S(F) < theta_d]
//   out   = [(S(F_e) + S(F_d)) + (theta_d - theta_e) < 0]
// every complement, difference and sum rounded to float32.  The two
// transforms of the first stage and the four of the second run as one
// batched launch each over the same B images.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "fgx_internal.h"

namespace fgx {
namespace {

size_t al256g(size_t x) { return (x + 255) & ~size_t(255); }

// masks [1 - F; F] of the first stage
__global__ void __launch_bounds__(256) stage1_masks_kernel(const float* f, float* m, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = f[i];
        m[i] = __fsub_rn(1.0f, x);
        m[n + i] = x;
    }
}

// S(F) from the first stage's pair, then the masks [1 - F_e; F_e; 1 - F_d;
// F_d] of the second
__global__ void __launch_bounds__(256) stage2_masks_kernel(const float* pair, float* m, int64_t n,
                                                           float theta_d, float neg_theta_e) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float s = __fsub_rn(pair[i], pair[n + i]);
        const float fe = s < neg_theta_e ? 1.0f : 0.0f;
        const float fd = s < theta_d ? 1.0f : 0.0f;
        m[i] = __fsub_rn(1.0f, fe);
        m[n + i] = fe;
        m[2 * n + i] = __fsub_rn(1.0f, fd);
        m[3 * n + i] = fd;
    }
}

__global__ void __launch_bounds__(256) combine_kernel(const float* quad, float* out, int64_t n,
                                                      float c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float se = __fsub_rn(quad[i], quad[n + i]);
        const float sd = __fsub_rn(quad[2 * n + i], quad[3 * n + i]);
        out[i] = __fadd_rn(__fadd_rn(se, sd), c) < 0.0f ? 1.0f : 0.0f;
    }
}

// The first status word keeps the first device error of the call.
__global__ void gsf_merge_status_kernel(int* dst, const int* src) {
    if (*dst == 0 && *src != 0) *dst = *src;
}

struct GsfLayout {
    size_t fwd = 0, masks_off = 0, dist_off = 0, carry_off = 0, total = 0;
};

int gsf_layout(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
               const fgx_options* opt, GsfLayout* L) {
    int st = fgx_geodesic_workspace_size(ndim, 4 * B, C, D, H, W, opt, &L->fwd);
    if (st != FGX_OK) return st;
    const size_t quad = al256g((size_t)(4 * B * D * H * W) * sizeof(float));
    L->masks_off = al256g(L->fwd);
    L->dist_off = L->masks_off + quad;
    L->carry_off = L->dist_off + quad;  // the first stage's status word
    L->total = L->carry_off + 256;
    return FGX_OK;
}

int run_gsf(int ndim, const float* image, const float* mask, float* out, int64_t B, int64_t C,
            int64_t D, int64_t H, int64_t W, const float spacing[3], float v, float lambda,
            int iterations, float theta_d, float theta_e, void* workspace, size_t ws_bytes,
            const fgx_options* opt, void* stream) {
    if (!(std::isfinite(theta_d) && theta_d >= 0.f && std::isfinite(theta_e) && theta_e >= 0.f))
        return FGX_ERR_ARG;
    GsfLayout L;
    int st = gsf_layout(ndim, B, C, D, H, W, opt, &L);
    if (st != FGX_OK) return st;
    const int64_t n = B * D * H * W;
    if (n == 0)  // argument checks and a clean status word
        return ndim == 2 ? fgx_geodesic2d(image, mask, out, B, C, H, W, v, lambda, iterations,
                                          workspace, ws_bytes, opt, stream)
                         : fgx_geodesic3d(image, mask, out, B, C, D, H, W, spacing, v, lambda,
                                          iterations, workspace, ws_bytes, opt, stream);
    if (!workspace || ws_bytes < L.total) return FGX_ERR_WORKSPACE;
    if (!mask || !out) return FGX_ERR_ARG;
    if (!device_pointer(workspace) || !device_pointer(mask) || !device_pointer(out))
        return FGX_ERR_NOT_DEVICE_PTR;
    char* w = (char*)workspace;
    float* masks = (float*)(w + L.masks_off);
    float* dists = (float*)(w + L.dist_off);
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FGX_ERR_CUDA;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 8));
    const float unit[3] = {1.f, 1.f, 1.f};
    const float* sp = ndim == 3 ? spacing : unit;
    const int64_t Dd = ndim == 3 ? D : 1;
    stage1_masks_kernel<<<grid, 256, 0, s>>>(mask, masks, n);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    st = run_forward_batch(ndim, image, B, masks, dists, 2 * B, C, Dd, H, W, sp, v, lambda,
                           iterations, workspace, L.fwd, opt, stream);
    if (st != FGX_OK) return st;
    stage2_masks_kernel<<<grid, 256, 0, s>>>(dists, masks, n, theta_d, -theta_e);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    // the second launch clears the status word: keep a first-stage error
    int* carry = (int*)(w + L.carry_off);
    if (cudaMemcpyAsync(carry, workspace, sizeof(int), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    st = run_forward_batch(ndim, image, B, masks, dists, 4 * B, C, Dd, H, W, sp, v, lambda,
                           iterations, workspace, L.fwd, opt, stream);
    if (st != FGX_OK) return st;
    gsf_merge_status_kernel<<<1, 1, 0, s>>>((int*)workspace, carry);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    volatile float c = theta_d - theta_e;  // rounded to float32 on the host
    combine_kernel<<<grid, 256, 0, s>>>(dists, out, n, c);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace
}  // namespace fgx

using namespace fgx;

extern "C" {

int fgx_gsf_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                           const fgx_options* opt, size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    GsfLayout L;
    const int st = gsf_layout(ndim, B, C, ndim == 3 ? D : 1, H, W, opt, &L);
    if (st != FGX_OK) return st;
    *bytes = L.total;
    return FGX_OK;
}

int fgx_gsf2d(const float* image, const float* mask, float* out, int64_t B, int64_t C, int64_t H,
              int64_t W, float v, float lambda, int iterations, float theta_d, float theta_e,
              void* workspace, size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_gsf(2, image, mask, out, B, C, 1, H, W, nullptr, v, lambda, iterations, theta_d,
                   theta_e, workspace, workspace_bytes, opt, stream);
}

int fgx_gsf3d(const float* image, const float* mask, float* out, int64_t B, int64_t C, int64_t D,
              int64_t H, int64_t W, const float spacing[3], float v, float lambda,
              int iterations, float theta_d, float theta_e, void* workspace,
              size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_gsf(3, image, mask, out, B, C, D, H, W, spacing, v, lambda, iterations, theta_d,
                   theta_e, workspace, workspace_bytes, opt, stream);
}

}  // extern "C"
