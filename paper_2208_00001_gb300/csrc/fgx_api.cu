// C ABI entry points (include/fgx.h): argument checks, planning of the pass
// geometry and tiling, workspace layout, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "fgx_internal.h"

namespace fgx {

// The paper's pass order (Implementation section): 2D top-bottom,
// bottom-top, left-right, right-left; 3D front-back, back-front, then the 2D
// order.  Axis 0 = D, 1 = H, 2 = W.
static const int kSched2D[4][2] = {{1, +1}, {1, -1}, {2, +1}, {2, -1}};
static const int kSched3D[6][2] = {{0, +1}, {0, -1}, {1, +1}, {1, -1}, {2, +1}, {2, -1}};

// t_k = (1 - lambda) * s2_k with s2_k = ((dD sD)^2 + (dH sH)^2) + (dW sW)^2 for
// the stencil offsets of a pass, numbered row-major over the in-line axes
// (outer p, inner q, in (D, H, W) order); the pass-axis component is 1.
// Each product and sum is rounded to float separately: the volatile
// temporaries keep the host compiler from fusing or widening them (the
// library is also compiled with -ffp-contract=off).
void pass_offsets_t(int ndim, int axis, const float sp[3], float lambda, float t[9]) {
    int pa, qa;
    if (axis == 0) { pa = 1; qa = 2; } else if (axis == 1) { pa = 0; qa = 2; } else { pa = 0; qa = 1; }
    const int dpmin = ndim == 3 ? -1 : 0, dpmax = ndim == 3 ? 1 : 0;
    int k = 0;
    for (int dp = dpmin; dp <= dpmax; ++dp) {
        for (int dq = -1; dq <= 1; ++dq) {
            float delta[3] = {0.f, 0.f, 0.f};
            delta[axis] = 1.f;
            delta[pa] = (float)dp;
            delta[qa] = (float)dq;
            volatile float e0 = delta[0] * sp[0], e1 = delta[1] * sp[1], e2 = delta[2] * sp[2];
            volatile float a0 = e0 * e0, a1 = e1 * e1, a2 = e2 * e2;
            volatile float s01 = a0 + a1;
            volatile float s2 = s01 + a2;
            volatile float om = 1.0f - lambda;
            t[k++] = om * s2;
        }
    }
    for (; k < 9; ++k) t[k] = 0.f;
}

void pass_extents(int axis, const int64_t ext[3], PassGeom* g) {
    const int64_t st[3] = {ext[1] * ext[2], ext[2], 1};
    int pa, qa;
    if (axis == 0) { pa = 1; qa = 2; } else if (axis == 1) { pa = 0; qa = 2; } else { pa = 0; qa = 1; }
    g->axis = axis;
    g->L = ext[axis];
    g->P = ext[pa];
    g->Q = ext[qa];
    g->sl = st[axis];
    g->sp = st[pa];
    g->sq = st[qa];
}

namespace {

struct DeviceInfo {
    int dev = -1, sms = 0, ok = 0;
};

int current_device(DeviceInfo* info) {
    static DeviceInfo cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FGX_ERR_DEVICE;
    if (dev < 0 || dev >= 64) return FGX_ERR_DEVICE;
    if (cache[dev].dev != dev) {
        int major = 0, minor = 0, sms = 0;
        if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return FGX_ERR_DEVICE;
        cache[dev].sms = sms;
        cache[dev].ok = (major == 10 && minor == 3);
        cache[dev].dev = dev;
    }
    *info = cache[dev];
    return info->ok ? FGX_OK : FGX_ERR_DEVICE;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + nb && y < x + na;
}

bool finite_pos(float x) { return std::isfinite(x) && x > 0.f; }

// Plan of one forward call.
struct Plan {
    SweepArgs args;
    int grid = 0;
    size_t smem = 0;
    size_t ws_bytes = 0;      // tiled sweep kernel
    size_t chain_bytes = 0;   // 2D warp-chain kernel (0 when not applicable)
    size_t vol3d_bytes = 0;   // 3D plane-tile kernel (0 when not applicable)
    int sms = 0;
};

int plan_forward(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                 const float spacing[3], float lambda, int iterations, const fgx_options* opt,
                 Plan* pl) {
    if (opt && opt->size != sizeof(fgx_options)) return FGX_ERR_ARG;
    if (opt && (opt->tile_lines < 0 || opt->tile_width < 0 || opt->tile_height < 0 ||
                opt->max_blocks < 0 || opt->timeout_ms < 0 || opt->segments < 0 ||
                opt->fast_math < 0 || opt->fast_math > 1))
        return FGX_ERR_ARG;
    if (ndim != 2 && ndim != 3) return FGX_ERR_ARG;
    if (B < 0 || C < 1 || D < 0 || H < 0 || W < 0) return FGX_ERR_SHAPE;
    if (ndim == 2 && D != 1) return FGX_ERR_SHAPE;
    if (C > 64) return FGX_ERR_UNSUPPORTED;
    DeviceInfo dev;
    int st = current_device(&dev);
    if (st != FGX_OK) return st;
    SweepArgs& a = pl->args;
    std::memset(&a, 0, sizeof(a));
    a.B = B;
    a.C = C;
    a.N = D * H * W;
    a.nimg = std::max<int64_t>(B, 1);
    a.ndim = ndim;
    a.lambda = lambda;
    a.iterations = iterations;
    a.npass = ndim == 3 ? 6 : 4;
    a.timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) * 1000000LL;
    const int64_t ext[3] = {D, H, W};
    const float unit[3] = {1.f, 1.f, 1.f};
    const float* sp = ndim == 3 ? spacing : unit;
    int max_tiles = 1;
    int64_t region = 1;
    for (int i = 0; i < a.npass; ++i) {
        PassGeom& g = a.pass[i];
        const int axis = ndim == 3 ? kSched3D[i][0] : kSched2D[i][0];
        g.dir = ndim == 3 ? kSched3D[i][1] : kSched2D[i][1];
        pass_extents(axis, ext, &g);
        pass_offsets_t(ndim, axis, sp, lambda, g.t);
        for (int k = 0; k < 9; ++k) g.c[k] = std::sqrt(g.t[k]);  // IEEE square root
        // 3D tile_lines alone sets the plane-tile kernel's ring width: the
        // tiled engine keeps its own default then
        const bool ring_only = ndim == 3 && opt && !opt->tile_width && !opt->tile_height;
        int K = (opt && opt->tile_lines && !ring_only) ? opt->tile_lines : (ndim == 3 ? 4 : 16);
        int tq = (opt && opt->tile_width) ? opt->tile_width : (ndim == 3 ? 16 : 128);
        int tp = ndim == 3 ? ((opt && opt->tile_height) ? opt->tile_height : 16) : 1;
        tq = (int)std::max<int64_t>(1, std::min<int64_t>(tq, std::max<int64_t>(g.Q, 1)));
        tp = (int)std::max<int64_t>(1, std::min<int64_t>(tp, std::max<int64_t>(g.P, 1)));
        // a ring must lie within the neighbouring tiles: full tiles are >= K
        if (g.Q > tq) K = std::min(K, tq);
        if (g.P > tp) K = std::min(K, tp);
        K = std::max(1, K);
        g.K = K;
        g.tp = tp;
        g.tq = tq;
        g.ntp = (int)std::max<int64_t>(1, (g.P + tp - 1) / tp);
        g.ntq = (int)std::max<int64_t>(1, (g.Q + tq - 1) / tq);
        max_tiles = std::max(max_tiles, g.ntp * g.ntq);
        const int64_t rp = std::min<int64_t>(std::max<int64_t>(g.P, 1), tp + 2 * K);
        const int64_t rq = std::min<int64_t>(std::max<int64_t>(g.Q, 1), tq + 2 * K);
        if (rp * rq > kMaxRegion) return FGX_ERR_UNSUPPORTED;
        // shared buffers carry a one-element border (none along p in 2D)
        region = std::max(region, (rp + (ndim == 3 ? 2 : 0)) * (rq + 2));
    }
    int kmax = 1;
    for (int i = 0; i < a.npass; ++i) kmax = std::max(kmax, a.pass[i].K);
    a.max_tiles = max_tiles;
    a.smem_region = (int)region;
    a.kmax = kmax;
    a.cost_mode = lambda == 0.0f ? kCostConst
                  : (lambda == 1.0f && C == 1) ? kCostAbs
                  : (opt && opt->fast_math) ? kCostFast : kCostGeneral;
    pl->smem = sweep_smem_bytes(a.cost_mode == kCostConst ? 0 : C, (int)region, kmax);
    if (pl->smem > 200 * 1024) return FGX_ERR_UNSUPPORTED;
    int per_sm = 0;
    st = sweep_max_blocks_per_sm(pl->smem, &per_sm);
    if (st != FGX_OK) return st;
    if (per_sm < 1) return FGX_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)per_sm * dev.sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, B * max_tiles));
    if (grid < max_tiles) return FGX_ERR_UNSUPPORTED;  // a pass's tiles must be co-resident
    pl->grid = (int)grid;
    pl->sms = dev.sms;
    pl->ws_bytes = kHeaderBytes + (size_t)std::max<int64_t>(B, 1) * max_tiles * 8;
    pl->chain_bytes = 0;
    if (ndim == 2) pl->chain_bytes = chain2d_workspace_bytes(B, C, H, W, opt);
    if (ndim == 3) pl->vol3d_bytes = vol3d_workspace_bytes(a, opt, dev.sms);
    return FGX_OK;
}

int run_forward(int ndim, const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                int64_t D, int64_t H, int64_t W, const float spacing[3], float v, float lambda,
                int iterations, uint8_t* codes, size_t codes_bytes, void* workspace,
                size_t ws_bytes, const fgx_options* opt, void* stream,
                bool fast_kernels = false, int64_t nimg = 0) {
    if (!(std::isfinite(v) && v > 0.f)) return FGX_ERR_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return FGX_ERR_ARG;
    if (iterations < 0) return FGX_ERR_ARG;
    if (ndim == 3) {
        if (!spacing) return FGX_ERR_ARG;
        for (int i = 0; i < 3; ++i)
            if (!finite_pos(spacing[i])) return FGX_ERR_ARG;
    }
    Plan pl;
    int st = plan_forward(ndim, B, C, D, H, W, spacing, lambda, iterations, opt, &pl);
    if (st != FGX_OK) return st;
    const int64_t N = D * H * W;
    cudaStream_t s = (cudaStream_t)stream;
    if (B * N == 0) {
        // nothing to compute; still leave a clean status word for the caller
        if (workspace && ws_bytes >= sizeof(int) && is_device_ptr(workspace) &&
            cudaMemsetAsync(workspace, 0, std::min(ws_bytes, kHeaderBytes), s) != cudaSuccess)
            return FGX_ERR_CUDA;
        return FGX_OK;
    }
    // no image is read when lambda = 0 (the Euclidean entry passes none)
    if (!mask || !dist || (!image && lambda != 0.f)) return FGX_ERR_ARG;
    if ((image && !is_device_ptr(image)) || !is_device_ptr(mask) || !is_device_ptr(dist))
        return FGX_ERR_NOT_DEVICE_PTR;
    // nimg: instance b reads image b % nimg (a batch of transforms of the
    // same images; internal callers only)
    if (nimg <= 0) nimg = B;
    const size_t nb = (size_t)(B * N) * sizeof(float);
    if (image && overlaps(dist, nb, image, (size_t)(nimg * C * N) * sizeof(float)))
        return FGX_ERR_ARG;
    const size_t need_codes = (size_t)iterations * pl.args.npass * (size_t)(B * N);
    // recorded codes come from the exact costs (fast math serves inference)
    if (codes && pl.args.cost_mode == kCostFast) pl.args.cost_mode = kCostGeneral;
    if (codes) {
        if (codes_bytes < need_codes) return FGX_ERR_WORKSPACE;
        if (!is_device_ptr(codes)) return FGX_ERR_NOT_DEVICE_PTR;
    }
    // the 2D chain kernel and the 3D plane-tile kernel serve the public
    // calls; the allocation-free entry keeps to the tiled engine
    if (fast_kernels && ndim == 2) {
        if (!workspace || ws_bytes < pl.chain_bytes) return FGX_ERR_WORKSPACE;
        if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
        return run_chain2d(image, mask, dist, codes, B, C, H, W, v, lambda, iterations,
                           workspace, ws_bytes, opt, pl.sms, stream, nimg);
    }
    if (fast_kernels && ndim == 3 && pl.vol3d_bytes && workspace &&
        ws_bytes >= pl.vol3d_bytes && vol3d_supports(pl.args, opt, pl.sms)) {
        if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
        return run_vol3d(pl.args, image, mask, dist, codes, v, workspace, ws_bytes, opt, pl.sms,
                         stream, false, nimg);
    }
    if (!workspace || ws_bytes < pl.ws_bytes) return FGX_ERR_WORKSPACE;
    if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    SweepArgs& a = pl.args;
    a.image = image;
    a.nimg = nimg;
    a.mask = mask;
    a.dist = dist;
    a.v = v;
    a.codes = codes;
    a.status = (int*)workspace;
    a.barrier = (unsigned int*)((char*)workspace + 64);
    a.flags = (unsigned long long*)((char*)workspace + kHeaderBytes);
    if (cudaMemsetAsync(workspace, 0, pl.ws_bytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    if (codes && need_codes && cudaMemsetAsync(codes, 0, need_codes, s) != cudaSuccess)
        return FGX_ERR_CUDA;
    return launch_sweep(a, pl.grid, pl.smem, stream);
}

}  // namespace

int run_forward_batch(int ndim, const float* image, int64_t nimg, const float* mask, float* dist,
                      int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                      const float spacing[3], float v, float lambda, int iterations,
                      void* workspace, size_t ws_bytes, const fgx_options* opt, void* stream) {
    if (nimg < 1 || (B > 0 && B % nimg)) return FGX_ERR_ARG;
    return run_forward(ndim, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                       nullptr, 0, workspace, ws_bytes, opt, stream, true, nimg);
}

int plan_instance(int ndim, int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                  float lambda, const fgx_options* opt, SweepArgs* args, int* sms) {
    Plan pl;
    const int st = plan_forward(ndim, 1, C, D, H, W, spacing, lambda, 1, opt, &pl);
    if (st != FGX_OK) return st;
    *args = pl.args;
    *sms = pl.sms;
    return FGX_OK;
}

bool device_pointer(const void* p) { return is_device_ptr(p); }

}  // namespace fgx

using namespace fgx;

extern "C" {

const char* fgx_status_string(int status) {
    switch (status) {
        case FGX_OK: return "ok";
        case FGX_ERR_ARG: return "invalid argument";
        case FGX_ERR_NOT_DEVICE_PTR: return "pointer is not device memory";
        case FGX_ERR_SHAPE: return "invalid shape";
        case FGX_ERR_WORKSPACE: return "workspace missing or too small";
        case FGX_ERR_CUDA: return "CUDA runtime error";
        case FGX_ERR_TIMEOUT: return "device wait timed out";
        case FGX_ERR_DEVICE: return "no usable sm_103 device";
        case FGX_ERR_UNSUPPORTED: return "unsupported request";
        default: return "unknown status";
    }
}

int fgx_version(void) { return 100; }

int fgx_geodesic_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                const fgx_options* opt, size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    const float unit[3] = {1.f, 1.f, 1.f};
    Plan pl;
    int st = plan_forward(ndim, B, C, D, H, W, unit, 0.5f, 1, opt, &pl);
    if (st != FGX_OK) return st;
    *bytes = std::max(std::max(pl.ws_bytes, pl.chain_bytes), pl.vol3d_bytes);
    return FGX_OK;
}

int fgx_geodesic2d(const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                   int64_t H, int64_t W, float v, float lambda, int iterations, void* workspace,
                   size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_forward(2, image, mask, dist, B, C, 1, H, W, nullptr, v, lambda, iterations,
                       nullptr, 0, workspace, workspace_bytes, opt, stream, true);
}

int fgx_geodesic3d(const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                   int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
                   float lambda, int iterations, void* workspace, size_t workspace_bytes,
                   const fgx_options* opt, void* stream) {
    return run_forward(3, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                       nullptr, 0, workspace, workspace_bytes, opt, stream, true);
}

int fgx_probe_wait_timeout(void* workspace, size_t workspace_bytes, int timeout_ms,
                           void* stream) {
    if (!workspace || workspace_bytes < kHeaderBytes + 8) return FGX_ERR_WORKSPACE;
    if (timeout_ms < 1 || timeout_ms > 10000) return FGX_ERR_ARG;
    if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, kHeaderBytes + 8, s) != cudaSuccess) return FGX_ERR_CUDA;
    char* w = (char*)workspace;
    launch_wait_probe((const unsigned long long*)(w + kHeaderBytes), (int*)w,
                      (long long)timeout_ms * 1000000LL, stream);
    return cudaGetLastError() == cudaSuccess ? FGX_OK : FGX_ERR_CUDA;
}

int fgx_autotune(int ndim, const float* image, const float* mask, float* dist, int64_t B,
                 int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3], float v,
                 float lambda, int iterations, void* workspace, size_t workspace_bytes,
                 const fgx_options* candidates, int n, int reps, int* best_index, float* best_ms,
                 void* stream) {
    if (!candidates || n < 1 || reps < 1 || !best_index || !best_ms) return FGX_ERR_ARG;
    if (ndim != 2 && ndim != 3) return FGX_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FGX_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FGX_ERR_CUDA;
    }
    auto call = [&](const fgx_options* o) {
        return ndim == 2 ? fgx_geodesic2d(image, mask, dist, B, C, H, W, v, lambda, iterations,
                                          workspace, workspace_bytes, o, stream)
                         : fgx_geodesic3d(image, mask, dist, B, C, D, H, W, spacing, v, lambda,
                                          iterations, workspace, workspace_bytes, o, stream);
    };
    int st = FGX_OK, best = -1;
    float best_t = 0.f;
    for (int i = 0; i < n && st == FGX_OK; ++i) {
        int r = call(candidates + i);
        if (r == FGX_ERR_UNSUPPORTED) continue;
        if (r != FGX_OK) { st = r; break; }
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = FGX_ERR_CUDA; break; }
        for (int k = 0; k < reps && r == FGX_OK; ++k) r = call(candidates + i);
        if (r != FGX_OK) { st = r; break; }
        float ms = 0.f;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            st = FGX_ERR_CUDA;
            break;
        }
        ms /= (float)reps;
        if (best < 0 || ms < best_t) {
            best = i;
            best_t = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FGX_OK) return st;
    if (best < 0) return FGX_ERR_UNSUPPORTED;
    *best_index = best;
    *best_ms = best_t;
    return FGX_OK;
}

int fgx_euclidean2d(const float* mask, float* dist, int64_t B, int64_t H, int64_t W, float v,
                    int iterations, void* workspace, size_t workspace_bytes,
                    const fgx_options* opt, void* stream) {
    return run_forward(2, nullptr, mask, dist, B, 1, 1, H, W, nullptr, v, 0.0f, iterations,
                       nullptr, 0, workspace, workspace_bytes, opt, stream, true);
}

int fgx_euclidean3d(const float* mask, float* dist, int64_t B, int64_t D, int64_t H, int64_t W,
                    const float spacing[3], float v, int iterations, void* workspace,
                    size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_forward(3, nullptr, mask, dist, B, 1, D, H, W, spacing, v, 0.0f, iterations,
                       nullptr, 0, workspace, workspace_bytes, opt, stream, true);
}

int fgx_signed_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                              const fgx_options* opt, size_t* bytes) {
    size_t fwd = 0;
    const int st = fgx_geodesic_workspace_size(ndim, 2 * B, C, D, H, W, opt, &fwd);
    if (st != FGX_OK) return st;
    *bytes = signed_workspace_bytes(fwd, B * D * H * W);
    return FGX_OK;
}

int fgx_signed_geodesic2d(const float* image, const float* mask, float* dist, int64_t B,
                          int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                          void* workspace, size_t workspace_bytes, const fgx_options* opt,
                          void* stream) {
    return run_signed(2, image, mask, dist, B, C, 1, H, W, nullptr, v, lambda, iterations,
                      workspace, workspace_bytes, opt, stream);
}

int fgx_signed_geodesic3d(const float* image, const float* mask, float* dist, int64_t B,
                          int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                          float v, float lambda, int iterations, void* workspace,
                          size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_signed(3, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                      workspace, workspace_bytes, opt, stream);
}

int fgx_workspace_status(const void* workspace, void* stream) {
    if (!workspace) return FGX_ERR_ARG;
    int h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, workspace, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FGX_ERR_CUDA;
    return h;
}

int fgx_train_saved_size(int ndim, int64_t B, int64_t D, int64_t H, int64_t W, int iterations,
                         size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    if (ndim != 2 && ndim != 3) return FGX_ERR_ARG;
    if (B < 0 || D < 0 || H < 0 || W < 0 || iterations < 0) return FGX_ERR_SHAPE;
    if (ndim == 2 && D != 1) return FGX_ERR_SHAPE;
    *bytes = (size_t)iterations * (ndim == 3 ? 6 : 4) * (size_t)(B * D * H * W);
    return FGX_OK;
}

int fgx_geodesic2d_fwd_train(const float* image, const float* mask, float* dist, int64_t B,
                             int64_t C, int64_t H, int64_t W, float v, float lambda,
                             int iterations, void* saved, size_t saved_bytes, void* workspace,
                             size_t workspace_bytes, const fgx_options* opt, void* stream) {
    if (!saved && (size_t)iterations * B * H * W > 0) return FGX_ERR_WORKSPACE;
    return run_forward(2, image, mask, dist, B, C, 1, H, W, nullptr, v, lambda, iterations,
                       (uint8_t*)saved, saved_bytes, workspace, workspace_bytes, opt, stream,
                       true);
}

int fgx_geodesic3d_fwd_train(const float* image, const float* mask, float* dist, int64_t B,
                             int64_t C, int64_t D, int64_t H, int64_t W,
                             const float spacing[3], float v, float lambda, int iterations,
                             void* saved, size_t saved_bytes, void* workspace,
                             size_t workspace_bytes, const fgx_options* opt, void* stream) {
    if (!saved && (size_t)iterations * B * D * H * W > 0) return FGX_ERR_WORKSPACE;
    return run_forward(3, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                       (uint8_t*)saved, saved_bytes, workspace, workspace_bytes, opt, stream,
                       true);
}

}  // extern "C"

// ---------------------------------------------------------------- backward

namespace fgx {
namespace {

struct BwdPlan {
    AdjointArgs args;
    int grid = 0;
    size_t smem = 0;
    size_t ws_bytes = 0;
    size_t flags_bytes = 0;
    SweepArgs fwd;  // geometry of the forward sweep (3D plane-tile reverse sweep)
    int sms = 0;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int plan_backward(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                  const float spacing[3], float lambda, int iterations, const fgx_options* opt,
                  BwdPlan* bp) {
    Plan pl;
    int st = plan_forward(ndim, B, C, D, H, W, spacing, lambda, iterations, opt, &pl);
    if (st != FGX_OK) return st;
    AdjointArgs& a = bp->args;
    std::memset(&a, 0, sizeof(a));
    const SweepArgs& f = pl.args;
    bp->fwd = f;
    bp->sms = pl.sms;
    a.B = B;
    a.C = C;
    a.N = f.N;
    a.ndim = ndim;
    a.lambda = lambda;
    a.iterations = iterations;
    a.npass = f.npass;
    for (int i = 0; i < kMaxPasses; ++i) a.pass[i] = f.pass[i];
    a.timeout_ns = f.timeout_ns;
    a.max_tiles = f.max_tiles;
    a.smem_region = f.smem_region;
    bp->smem = (size_t)(4 + 2 * C) * (size_t)f.smem_region * sizeof(float);
    if (bp->smem > 200 * 1024) return FGX_ERR_UNSUPPORTED;
    int per_sm = 0;
    st = adjoint_max_blocks_per_sm(bp->smem, &per_sm);
    if (st != FGX_OK) return st;
    if (per_sm < 1) return FGX_ERR_UNSUPPORTED;
    int64_t grid = (int64_t)per_sm * pl.sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, B * f.max_tiles));
    if (grid < f.max_tiles) return FGX_ERR_UNSUPPORTED;
    bp->grid = (int)grid;
    bp->flags_bytes = align256((size_t)std::max<int64_t>(B, 1) * f.max_tiles * 8);
    bp->ws_bytes = kHeaderBytes + bp->flags_bytes + 2 * align256((size_t)(B * f.N) * 4);
    return FGX_OK;
}

// g0 / lambda_terms (nullable): the adjoint of D0 and the per-element terms of
// dL/dlambda, which only the warp-chain (2D) and plane-tile (3D) reverse
// sweeps produce.
int run_backward(int ndim, const float* grad_dist, const float* image, const void* saved,
                 size_t saved_bytes, float* grad_image, float* grad_mask, int64_t B, int64_t C,
                 int64_t D, int64_t H, int64_t W, const float spacing[3], float v, float lambda,
                 int iterations, void* workspace, size_t ws_bytes, const fgx_options* opt,
                 void* stream, float* g0 = nullptr, float* lambda_terms = nullptr) {
    if (!(std::isfinite(v) && v > 0.f)) return FGX_ERR_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return FGX_ERR_ARG;
    if (iterations < 0) return FGX_ERR_ARG;
    if (ndim == 3) {
        if (!spacing) return FGX_ERR_ARG;
        for (int i = 0; i < 3; ++i)
            if (!finite_pos(spacing[i])) return FGX_ERR_ARG;
    }
    BwdPlan bp;
    int st = plan_backward(ndim, B, C, D, H, W, spacing, lambda, iterations, opt, &bp);
    if (st != FGX_OK) return st;
    const int64_t N = D * H * W;
    cudaStream_t s = (cudaStream_t)stream;
    if (B * N == 0) {
        if (workspace && ws_bytes >= sizeof(int) && is_device_ptr(workspace) &&
            cudaMemsetAsync(workspace, 0, std::min(ws_bytes, kHeaderBytes), s) != cudaSuccess)
            return FGX_ERR_CUDA;
        return FGX_OK;
    }
    if (!grad_dist || !image) return FGX_ERR_ARG;
    const bool params = g0 || lambda_terms;
    if (!grad_image && !grad_mask && !params) return FGX_ERR_ARG;
    if (!is_device_ptr(grad_dist) || !is_device_ptr(image)) return FGX_ERR_NOT_DEVICE_PTR;
    if (grad_image && !is_device_ptr(grad_image)) return FGX_ERR_NOT_DEVICE_PTR;
    if (grad_mask && !is_device_ptr(grad_mask)) return FGX_ERR_NOT_DEVICE_PTR;
    const size_t need_codes = (size_t)iterations * bp.args.npass * (size_t)(B * N);
    if (need_codes) {
        if (!saved || saved_bytes < need_codes) return FGX_ERR_WORKSPACE;
        if (!is_device_ptr(saved)) return FGX_ERR_NOT_DEVICE_PTR;
    }
    if (params && iterations == 0) {
        // D = v M: the adjoint of D0 is dL/dD, and no edge cost is used
        const size_t nb = (size_t)(B * N) * sizeof(float);
        if (g0 && cudaMemcpyAsync(g0, grad_dist, nb, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return FGX_ERR_CUDA;
        if (lambda_terms && cudaMemsetAsync(lambda_terms, 0, nb, s) != cudaSuccess)
            return FGX_ERR_CUDA;
        if (!grad_image && !grad_mask) {
            if (workspace && ws_bytes >= kHeaderBytes &&
                cudaMemsetAsync(workspace, 0, kHeaderBytes, s) != cudaSuccess)
                return FGX_ERR_CUDA;
            return FGX_OK;
        }
        g0 = lambda_terms = nullptr;
    }

    if (ndim == 2 && iterations > 0 && workspace &&
        ws_bytes >= adj2d_workspace_bytes(B, H, W, iterations, opt)) {
        if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
        DeviceInfo dev;
        st = current_device(&dev);
        if (st != FGX_OK) return st;
        st = run_adj2d(grad_dist, image, (const uint8_t*)saved, grad_image, grad_mask, B, C, H,
                       W, v, lambda, iterations, workspace, ws_bytes, opt, dev.sms, stream, g0,
                       lambda_terms);
        if (st != FGX_ERR_UNSUPPORTED) return st;
    }
    if (ndim == 3 && iterations > 0 && workspace) {
        const size_t need = adj3d_workspace_bytes(bp.fwd, iterations, opt, bp.sms);
        if (need && ws_bytes >= need) {
            if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
            // |offset|^2 per pass and stencil offset: the offsets with lambda = 0
            float s2[kMaxPasses * 9];
            for (int i = 0; i < kMaxPasses; ++i)
                pass_offsets_t(3, kSched3D[i][0], spacing, 0.0f, s2 + 9 * i);
            st = run_adj3d(bp.fwd, grad_dist, image, (const uint8_t*)saved, grad_image,
                           grad_mask, v, iterations, workspace, ws_bytes, opt, bp.sms, stream,
                           g0, lambda_terms, s2);
            if (st != FGX_ERR_UNSUPPORTED) return st;
        }
    }
    // the tiled engine's reverse sweep has no parameter terms
    if (g0 || lambda_terms) return FGX_ERR_UNSUPPORTED;
    if (!workspace || ws_bytes < bp.ws_bytes) return FGX_ERR_WORKSPACE;
    if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    AdjointArgs& a = bp.args;
    char* w = (char*)workspace;
    a.image = image;
    a.codes = (const uint8_t*)saved;
    a.grad_dist = grad_dist;
    a.grad_image = grad_image;
    a.grad_mask = grad_mask;
    a.v = v;
    a.status = (int*)w;
    a.barrier = (unsigned int*)(w + 64);
    a.flags = (unsigned long long*)(w + kHeaderBytes);
    a.G[0] = (float*)(w + kHeaderBytes + bp.flags_bytes);
    a.G[1] = (float*)(w + kHeaderBytes + bp.flags_bytes + align256((size_t)(B * N) * 4));
    if (cudaMemsetAsync(workspace, 0, kHeaderBytes + bp.flags_bytes, s) != cudaSuccess)
        return FGX_ERR_CUDA;
    return launch_adjoint(a, bp.grid, bp.smem, stream);
}

// ---------------------------------------------------- checkpointed 3D training
//
// The training forward keeps D at the start of every `interval`-th
// iteration instead of the parent codes; the backward replays each segment
// of `interval` iterations from its checkpoint (D0 = v M from the mask for
// the first) with codes into the workspace, then sweeps that segment's pass
// applications in reverse.  Every segment is replayed once, so the backward
// costs one extra forward.

struct CkptLayout {
    int k = 0, nseg = 0;          // iterations per segment, segments
    size_t adj = 0, fwd = 0;      // workspace bytes of the reverse sweep and the replay
    size_t fwd_off = 0, dwork_off = 0, codes_off = 0, total = 0;
};

int plan_checkpoint(int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                    const float spacing[3], float lambda, int iterations, int interval,
                    const fgx_options* opt, Plan* pl, CkptLayout* L) {
    if (iterations < 1 || interval < 1) return FGX_ERR_ARG;
    int st = plan_forward(3, B, C, D, H, W, spacing, lambda, iterations, opt, pl);
    if (st != FGX_OK) return st;
    if (!vol3d_supports(pl->args, opt, pl->sms)) return FGX_ERR_UNSUPPORTED;
    L->k = std::min(interval, iterations);
    L->nseg = (iterations + L->k - 1) / L->k;
    L->adj = adj3d_workspace_bytes(pl->args, L->k, opt, pl->sms);
    L->fwd = vol3d_workspace_bytes(pl->args, opt, pl->sms);
    if (!L->adj || !L->fwd) return FGX_ERR_UNSUPPORTED;
    const size_t n = (size_t)(B * D * H * W);
    L->fwd_off = align256(L->adj);
    L->dwork_off = align256(L->fwd_off + L->fwd);
    L->codes_off = align256(L->dwork_off + n * sizeof(float));
    L->total = L->codes_off + (size_t)L->k * kMaxPasses * n;
    return FGX_OK;
}

// The first status word keeps the first device error of the call.
__global__ void merge_status_kernel(int* dst, const int* src) {
    if (*dst == 0 && *src != 0) *dst = *src;
}

int check_3d_args(const float spacing[3], float v, float lambda, int iterations) {
    if (!(std::isfinite(v) && v > 0.f)) return FGX_ERR_ARG;
    if (!(lambda >= 0.f && lambda <= 1.f)) return FGX_ERR_ARG;
    if (iterations < 0 || !spacing) return FGX_ERR_ARG;
    for (int i = 0; i < 3; ++i)
        if (!finite_pos(spacing[i])) return FGX_ERR_ARG;
    return FGX_OK;
}

struct ParamsLayout {
    size_t g0_off, lt_off, vt_off, part_off, total;
};

// Workspace of the parameter gradients: the reverse sweep's workspace, then
// G0, scratch for the two per-element term arrays and the float64 partial
// sums.
ParamsLayout params_layout(size_t bwd, int64_t n) {
    ParamsLayout l;
    const size_t arr = align256((size_t)std::max<int64_t>(n, 1) * sizeof(float));
    l.g0_off = align256(bwd);
    l.lt_off = l.g0_off + arr;
    l.vt_off = l.lt_off + arr;
    l.part_off = l.vt_off + arr;
    l.total = l.part_off + align256(param_partials_bytes());
    return l;
}

}  // namespace
}  // namespace fgx

extern "C" {

int fgx_backward_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                int iterations, const fgx_options* opt, size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    if (iterations < 0) return FGX_ERR_ARG;
    const float unit[3] = {1.f, 1.f, 1.f};
    BwdPlan bp;
    int st = plan_backward(ndim, B, C, D, H, W, unit, 0.5f, std::max(iterations, 1), opt, &bp);
    if (st != FGX_OK) return st;
    *bytes = bp.ws_bytes;
    if (ndim == 2 && iterations > 0)
        *bytes = std::max(*bytes, adj2d_workspace_bytes(B, H, W, iterations, opt));
    if (ndim == 3 && iterations > 0)
        *bytes = std::max(*bytes, adj3d_workspace_bytes(bp.fwd, iterations, opt, bp.sms));
    return FGX_OK;
}

int fgx_geodesic2d_bwd(const float* grad_dist, const float* image, const void* saved,
                       size_t saved_bytes, float* grad_image, float* grad_mask, int64_t B,
                       int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                       void* workspace, size_t workspace_bytes, const fgx_options* opt,
                       void* stream) {
    return run_backward(2, grad_dist, image, saved, saved_bytes, grad_image, grad_mask, B, C, 1,
                        H, W, nullptr, v, lambda, iterations, workspace, workspace_bytes, opt,
                        stream);
}

int fgx_geodesic3d_bwd(const float* grad_dist, const float* image, const void* saved,
                       size_t saved_bytes, float* grad_image, float* grad_mask, int64_t B,
                       int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                       float v, float lambda, int iterations, void* workspace,
                       size_t workspace_bytes, const fgx_options* opt, void* stream) {
    return run_backward(3, grad_dist, image, saved, saved_bytes, grad_image, grad_mask, B, C, D,
                        H, W, spacing, v, lambda, iterations, workspace, workspace_bytes, opt,
                        stream);
}

int fgx_checkpoint_saved_size(int64_t B, int64_t D, int64_t H, int64_t W, int iterations,
                              int interval, size_t* bytes) {
    if (!bytes || interval < 1) return FGX_ERR_ARG;
    if (B < 0 || D < 0 || H < 0 || W < 0 || iterations < 0) return FGX_ERR_SHAPE;
    const int k = std::max(1, std::min(interval, std::max(iterations, 1)));
    const int nseg = (iterations + k - 1) / k;
    *bytes = (size_t)std::max(nseg - 1, 0) * (size_t)(B * D * H * W) * sizeof(float);
    return FGX_OK;
}

int fgx_checkpoint_workspace_size(int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                  int iterations, int interval, const fgx_options* opt,
                                  size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    const float unit[3] = {1.f, 1.f, 1.f};
    Plan pl;
    CkptLayout L;
    const int st = plan_checkpoint(B, C, D, H, W, unit, 0.5f, std::max(iterations, 1), interval,
                                   opt, &pl, &L);
    if (st != FGX_OK) return st;
    *bytes = L.total;
    return FGX_OK;
}

int fgx_geodesic3d_fwd_checkpoint(const float* image, const float* mask, float* dist, int64_t B,
                                  int64_t C, int64_t D, int64_t H, int64_t W,
                                  const float spacing[3], float v, float lambda, int iterations,
                                  int interval, void* saved, size_t saved_bytes, void* workspace,
                                  size_t workspace_bytes, const fgx_options* opt, void* stream) {
    int st = check_3d_args(spacing, v, lambda, iterations);
    if (st != FGX_OK) return st;
    if (interval < 1) return FGX_ERR_ARG;
    const int64_t n = B * D * H * W;
    if (iterations == 0 || n == 0)
        return run_forward(3, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                           nullptr, 0, workspace, workspace_bytes, opt, stream, true);
    Plan pl;
    CkptLayout L;
    if ((st = plan_checkpoint(B, C, D, H, W, spacing, lambda, iterations, interval, opt, &pl,
                              &L)) != FGX_OK)
        return st;
    if (!image || !mask || !dist) return FGX_ERR_ARG;
    if (!is_device_ptr(image) || !is_device_ptr(mask) || !is_device_ptr(dist))
        return FGX_ERR_NOT_DEVICE_PTR;
    if (overlaps(dist, (size_t)n * 4, image, (size_t)(n * C) * 4)) return FGX_ERR_ARG;
    const size_t need = (size_t)(L.nseg - 1) * (size_t)n * sizeof(float);
    if (need && (!saved || saved_bytes < need)) return FGX_ERR_WORKSPACE;
    if (need && !is_device_ptr(saved)) return FGX_ERR_NOT_DEVICE_PTR;
    if (!workspace || workspace_bytes < L.total) return FGX_ERR_WORKSPACE;
    if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)workspace;
    // the caller reads the status word at offset 0; every segment's launch
    // clears its own (at the replay region) and its first error is merged
    if (cudaMemsetAsync(w, 0, kHeaderBytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    for (int seg = 0; seg < L.nseg; ++seg) {
        SweepArgs f = pl.args;
        f.iterations = std::min(L.k, iterations - seg * L.k);
        if (seg > 0 && cudaMemcpyAsync((char*)saved + (size_t)(seg - 1) * n * sizeof(float), dist,
                                       (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice,
                                       s) != cudaSuccess)
            return FGX_ERR_CUDA;
        st = run_vol3d(f, image, mask, dist, nullptr, v, w + L.fwd_off, L.fwd, opt, pl.sms, stream,
                       seg > 0);
        if (st != FGX_OK) return st;
        merge_status_kernel<<<1, 1, 0, s>>>((int*)w, (const int*)(w + L.fwd_off));
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

int fgx_geodesic3d_bwd_checkpoint(const float* grad_dist, const float* image, const float* mask,
                                  const void* saved, size_t saved_bytes, float* grad_image,
                                  float* grad_mask, int64_t B, int64_t C, int64_t D, int64_t H,
                                  int64_t W, const float spacing[3], float v, float lambda,
                                  int iterations, int interval, void* workspace,
                                  size_t workspace_bytes, const fgx_options* opt, void* stream) {
    int st = check_3d_args(spacing, v, lambda, iterations);
    if (st != FGX_OK) return st;
    if (interval < 1) return FGX_ERR_ARG;
    const int64_t n = B * D * H * W;
    if (iterations == 0 || n == 0)
        return run_backward(3, grad_dist, image, nullptr, 0, grad_image, grad_mask, B, C, D, H, W,
                            spacing, v, lambda, iterations, workspace, workspace_bytes, opt,
                            stream);
    Plan pl;
    CkptLayout L;
    if ((st = plan_checkpoint(B, C, D, H, W, spacing, lambda, iterations, interval, opt, &pl,
                              &L)) != FGX_OK)
        return st;
    if (!grad_dist || !image || !mask || (!grad_image && !grad_mask)) return FGX_ERR_ARG;
    for (const void* p : {(const void*)grad_dist, (const void*)image, (const void*)mask})
        if (!is_device_ptr(p)) return FGX_ERR_NOT_DEVICE_PTR;
    if ((grad_image && !is_device_ptr(grad_image)) || (grad_mask && !is_device_ptr(grad_mask)))
        return FGX_ERR_NOT_DEVICE_PTR;
    const size_t need = (size_t)(L.nseg - 1) * (size_t)n * sizeof(float);
    if (need && (!saved || saved_bytes < need)) return FGX_ERR_WORKSPACE;
    if (need && !is_device_ptr(saved)) return FGX_ERR_NOT_DEVICE_PTR;
    if (!workspace || workspace_bytes < L.total) return FGX_ERR_WORKSPACE;
    if (!is_device_ptr(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    float s2[kMaxPasses * 9];
    for (int i = 0; i < kMaxPasses; ++i) pass_offsets_t(3, kSched3D[i][0], spacing, 0.0f, s2 + 9 * i);
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)workspace;
    float* dwork = (float*)(w + L.dwork_off);
    uint8_t* codes = (uint8_t*)(w + L.codes_off);
    int in_idx = -1;
    for (int seg = L.nseg - 1; seg >= 0; --seg) {
        SweepArgs f = pl.args;
        f.iterations = std::min(L.k, iterations - seg * L.k);
        if (seg > 0 && cudaMemcpyAsync(dwork, (const char*)saved + (size_t)(seg - 1) * n * 4,
                                       (size_t)n * 4, cudaMemcpyDeviceToDevice,
                                       s) != cudaSuccess)
            return FGX_ERR_CUDA;
        // replay of the segment's iterations, recording their codes
        st = run_vol3d(f, image, mask, dwork, codes, v, w + L.fwd_off, L.fwd, opt, pl.sms, stream,
                       seg > 0);
        if (st != FGX_OK) return st;
        const int t_lo = seg * L.k * kMaxPasses;
        const int t_hi = t_lo + f.iterations * kMaxPasses;
        st = run_adj3d(pl.args, grad_dist, image, codes, grad_image, grad_mask, v, iterations, w,
                       L.adj, opt, pl.sms, stream, nullptr, nullptr, s2, t_lo, t_hi, in_idx,
                       &in_idx, seg == L.nseg - 1);
        if (st != FGX_OK) return st;
        // the reverse sweep's status word (offset 0; cleared only by the
        // first range) also takes the replay's first error
        merge_status_kernel<<<1, 1, 0, s>>>((int*)w, (const int*)(w + L.fwd_off));
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

int fgx_params_workspace_size(int ndim, int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                              int iterations, const fgx_options* opt, size_t* bytes) {
    size_t bwd = 0;
    const int st = fgx_backward_workspace_size(ndim, B, C, D, H, W, iterations, opt, &bwd);
    if (st != FGX_OK) return st;
    *bytes = params_layout(bwd, B * D * H * W).total;
    return FGX_OK;
}

int fgx_geodesic_bwd_params(int ndim, const float* grad_dist, const float* image,
                            const float* mask, const void* saved, size_t saved_bytes,
                            float* grad_image, float* grad_mask, float* lambda_terms,
                            float* v_terms, double* grad_lambda, double* grad_v, int64_t B,
                            int64_t C, int64_t D, int64_t H, int64_t W, const float spacing[3],
                            float v, float lambda, int iterations, void* workspace,
                            size_t workspace_bytes, const fgx_options* opt, void* stream) {
    if (ndim != 2 && ndim != 3) return FGX_ERR_ARG;
    if (ndim == 2) D = 1;
    size_t bwd = 0;
    int st = fgx_backward_workspace_size(ndim, B, C, D, H, W, iterations, opt, &bwd);
    if (st != FGX_OK) return st;
    const int64_t n = B * D * H * W;
    const ParamsLayout l = params_layout(bwd, n);
    if (!workspace || workspace_bytes < l.total) return FGX_ERR_WORKSPACE;
    if (!mask && n > 0) return FGX_ERR_ARG;
    if (!is_device_ptr(workspace) || (n > 0 && !is_device_ptr(mask)))
        return FGX_ERR_NOT_DEVICE_PTR;
    for (void* p : {(void*)lambda_terms, (void*)v_terms, (void*)grad_lambda, (void*)grad_v})
        if (p && !is_device_ptr(p)) return FGX_ERR_NOT_DEVICE_PTR;
    char* w = (char*)workspace;
    float* g0 = (float*)(w + l.g0_off);
    float* lt = lambda_terms ? lambda_terms : (float*)(w + l.lt_off);
    float* vt = v_terms ? v_terms : (float*)(w + l.vt_off);
    st = run_backward(ndim, grad_dist, image, saved, saved_bytes, grad_image, grad_mask, B, C, D,
                      H, W, spacing, v, lambda, iterations, workspace, bwd, opt, stream, g0, lt);
    if (st != FGX_OK) return st;
    DeviceInfo dev;
    if ((st = current_device(&dev)) != FGX_OK) return st;
    return run_param_sums(mask, g0, vt, lt, grad_lambda, grad_v, (double*)(w + l.part_off), n,
                          dev.sms, stream);
}


}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free forward.  Some callers cannot allocate device memory at the
// point where they need a transform: code running inside a custom allocator's
// callback, real-time loops with a fixed memory budget, or plugins whose host
// framework owns every allocation.  This entry
// point runs the same sweep kernel as fgx_geodesic2d / fgx_geodesic3d, but
// its scratch (status word, barrier counter, tile progress tags) lives in the
// static device array below instead of a caller workspace.  Every GPU that
// loads the library holds the array until the process exits.
namespace {

constexpr size_t kNoAllocScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the kernel must be given
// this address, never the name.  The address is looked up again on every
// call made outside stream capture (a device reset reloads the module and
// may move the array); while `stream` is capturing, the last address found
// on this device is used.
int noalloc_scratch_address(cudaStream_t stream, void** out) {
    static std::mutex mu;
    static void* addr[64];
    static bool done[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FGX_ERR_DEVICE;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        return FGX_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!done[dev] || cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return FGX_ERR_CUDA;
        }
        addr[dev] = p;
        done[dev] = true;
    }
    *out = addr[dev];
    return FGX_OK;
}

}  // namespace

extern "C" int fgx_geodesic_noalloc(int ndim, const float* image, const float* mask, float* dist,
                                    int64_t B, int64_t C, int64_t D, int64_t H, int64_t W,
                                    const float spacing[3], float v, float lambda, int iterations,
                                    const fgx_options* opt, void* stream) {
    if (ndim != 2 && ndim != 3) return FGX_ERR_ARG;
    if (ndim == 2 && D != 1) return FGX_ERR_SHAPE;
    const float unit[3] = {1.f, 1.f, 1.f};
    Plan pl;
    int st = plan_forward(ndim, B, C, D, H, W, ndim == 3 && spacing ? spacing : unit, lambda,
                          iterations, opt, &pl);
    if (st != FGX_OK) return st;
    if (pl.ws_bytes > kNoAllocScratchBytes) return FGX_ERR_WORKSPACE;  // beyond the static limit
    void* scratch = nullptr;
    st = noalloc_scratch_address((cudaStream_t)stream, &scratch);
    if (st != FGX_OK) return st;
    return run_forward(ndim, image, mask, dist, B, C, D, H, W, spacing, v, lambda, iterations,
                       nullptr, 0, scratch, kNoAllocScratchBytes, opt, stream);
}

// Status word of the static scratch (its first int), read back on `stream`
// after the calls queued before it.  A plain copy from the symbol: nothing is
// allocated.
extern "C" int fgx_noalloc_status(void* stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FGX_ERR_DEVICE;
    int word = 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyFromSymbolAsync(&word, g_noalloc_scratch, sizeof(int), 0,
                                  cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return FGX_ERR_CUDA;
    }
    return word == 0 ? FGX_OK : word;
}
