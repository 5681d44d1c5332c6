// Reverse sweep through the recorded parent codes (the adjoint of the raster
// scan of FastGeodis, Implementation section).
//
// The forward pass is a composition of min and + of smooth edge costs, so
// away from ties it is differentiable along the recorded argmin parents.  For
// every pass application in reverse order and every line in reverse sweep
// order, with A = the total adjoint of an element in this pass:
//   A[e] = G_in[e] + sum over the children x that chose e (offset order) of A[x]
//   dI[e] -= (A[x] lambda / c(e,x)) (I(x) - I(e))      for each such child x
//   dI[e] += (A[e] lambda / c(p,e)) (I(e) - I(p))       for e's own parent p
// (image terms taken as 0 where c = 0), and the adjoint that reaches the
// previous pass is A[e] if e kept its value (code 0), else 0.  Finally
// dL/dM = v * (adjoint of D0).
//
// Decomposition: the same cooperative tile scheme as the forward sweep (tiles
// of a line, ring halo of K elements, tagged neighbour waits every K lines,
// grid barrier between passes).  The ring is recomputed redundantly from the
// same inputs; because sums are not idempotent, the adjoint lives in two
// ping-pong buffers so that a ring element always reads the previous pass's
// value, never one a neighbour already updated in this pass.
#include <cuda_runtime.h>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;

// Progress tag of a tile: passes are processed in decreasing order, so the
// tag counts processed passes (seq = T-1-t_app) to stay increasing.
__device__ __forceinline__ unsigned long long atag(int seq, int blk) {
    return ((unsigned long long)(seq + 1) << 32) | (unsigned int)blk;
}

// Cost of the edge (x, y) in the fixed order of the forward pass.
__device__ __forceinline__ float cost_of(const float* Ix, int64_t sx, const float* Iy, int64_t sy,
                                         int64_t C, float t, float lam) {
    float di2 = 0.0f;
    for (int64_t ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(Ix[ch * sx], Iy[ch * sy]);
        di2 = __fadd_rn(di2, __fmul_rn(d, d));
    }
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// One tile of one instance for pass application t_app (T in total).
__device__ bool adjoint_tile(const AdjointArgs& a, const PassGeom& g, int t_app, int T,
                             int64_t b, int tile, float* smem) {
    __shared__ int ok;
    const int jp = tile / g.ntq, jq = tile % g.ntq;
    const int64_t p0 = (int64_t)jp * g.tp, p1 = mn64(g.P, p0 + g.tp);
    const int64_t q0 = (int64_t)jq * g.tq, q1 = mn64(g.Q, q0 + g.tq);
    const int64_t L = g.L, P = g.P, Q = g.Q, N = a.N, C = a.C;
    const float* img = a.image + b * C * N;
    const uint8_t* cd = a.codes + ((int64_t)t_app * a.B + b) * N;
    const uint8_t* cd_next = (t_app + 1 < T) ? a.codes + ((int64_t)(t_app + 1) * a.B + b) * N
                                             : nullptr;
    const float* Gin = a.G[(T - 1 - t_app) & 1] + b * N;
    float* Gout = a.G[(T - t_app) & 1] + b * N;
    float* gi = a.grad_image ? a.grad_image + b * C * N : nullptr;
    unsigned long long* myflag = a.flags + b * a.max_tiles + tile;
    const int region = a.smem_region;
    float* bufA[2] = {smem, smem + region};
    float* bufC[2] = {smem + 2 * region, smem + 3 * region};
    float* bufI[2] = {smem + 4 * region, smem + (4 + C) * region};
    const float lam = a.lambda;
    const int dpmin = (a.ndim == 3) ? -1 : 0, dpmax = (a.ndim == 3) ? 1 : 0;

    const int nblk = (int)((L + g.K - 1) / g.K);
    for (int blk = 0; blk < nblk; ++blk) {
        const int64_t u0 = (int64_t)blk * g.K;  // reverse-sweep index of the block's first line
        const int nb = (int)mn64(g.K, L - u0);
        if (blk > 0) {
            if (threadIdx.x == 0) {
                ok = 1;
                const unsigned long long want = atag(T - 1 - t_app, blk);
                for (int dj = -1; dj <= 1 && ok; ++dj)
                    for (int di = -1; di <= 1 && ok; ++di) {
                        if (dj == 0 && di == 0) continue;
                        const int np = jp + dj, nq = jq + di;
                        if (np < 0 || np >= g.ntp || nq < 0 || nq >= g.ntq) continue;
                        if (!wait_tag(a.flags + b * a.max_tiles + np * g.ntq + nq, want,
                                      a.status, a.timeout_ns))
                            ok = 0;
                    }
            }
            __syncthreads();
            if (!ok) return false;
        }
        const int64_t rp0 = mx64(0, p0 - nb), rp1 = mn64(P, p1 + nb);
        const int64_t rq0 = mx64(0, q0 - nb), rq1 = mn64(Q, q1 + nb);
        const int64_t rw = rq1 - rq0;
        if (u0 > 0) {
            // the line after the block's first one in forward order: its
            // adjoints (written by the owning tiles), codes and intensities
            const int64_t l = L - u0;  // forward sweep index
            const int64_t ya = (g.dir > 0) ? l : (L - 1 - l);
            const int64_t n = (rp1 - rp0) * rw;
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                const int64_t p = rp0 + e / rw, q = rq0 + e % rw;
                const int64_t yi = ya * g.sl + p * g.sp + q * g.sq;
                bufA[0][e] = __ldcg(Gout + yi);
                bufC[0][e] = (float)cd[yi];
                for (int64_t ch = 0; ch < C; ++ch) bufI[0][ch * region + e] = __ldg(img + ch * N + yi);
            }
        }
        __syncthreads();
        int cur = 0;
        for (int i = 0; i < nb; ++i) {
            const int64_t u = u0 + i;
            const int64_t l = L - 1 - u;  // forward sweep index of this line
            const int64_t xa = (g.dir > 0) ? l : (L - 1 - l);
            const bool children = u > 0;
            const int r = nb - 1 - i;
            const int64_t cp0 = mx64(0, p0 - r), cp1 = mn64(P, p1 + r);
            const int64_t cq0 = mx64(0, q0 - r), cq1 = mn64(Q, q1 + r);
            const int64_t cw = cq1 - cq0, n = (cp1 - cp0) * cw;
            const float* pA = bufA[cur];
            const float* pC = bufC[cur];
            const float* pI = bufI[cur];
            float* nA = bufA[cur ^ 1];
            float* nC = bufC[cur ^ 1];
            float* nI = bufI[cur ^ 1];
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                const int64_t p = cp0 + e / cw, q = cq0 + e % cw;
                const int64_t xi = xa * g.sl + p * g.sp + q * g.sq;
                const int64_t s = (p - rp0) * rw + (q - rq0);
                for (int64_t ch = 0; ch < C; ++ch) nI[ch * region + s] = __ldg(img + ch * N + xi);
                const int code = cd[xi];
                nC[s] = (float)code;
                const bool owned = p >= p0 && p < p1 && q >= q0 && q < q1;
                const bool do_img = owned && gi != nullptr;
                float gin = __ldcg(Gin + xi);
                if (cd_next && cd_next[xi] != 0) gin = 0.0f;
                float acc = gin;
                int k = 0;
                for (int dp = dpmin; dp <= dpmax; ++dp) {
                    for (int dq = -1; dq <= 1; ++dq, ++k) {
                        if (!children) continue;
                        // the child that reaches this element through offset k
                        const int64_t xp = p - dp, xq = q - dq;
                        if (xp < 0 || xp >= P || xq < 0 || xq >= Q) continue;
                        const int64_t ys = (xp - rp0) * rw + (xq - rq0);
                        if ((int)pC[ys] != k + 1) continue;
                        const float Ax = pA[ys];
                        acc = __fadd_rn(acc, Ax);
                        if (do_img) {
                            const float c = cost_of(pI + ys, region, nI + s, region, C, g.t[k], lam);
                            if (c > 0.0f) {
                                const float w = __fdiv_rn(__fmul_rn(Ax, lam), c);
                                for (int64_t ch = 0; ch < C; ++ch) {
                                    const float d = __fsub_rn(pI[ch * region + ys], nI[ch * region + s]);
                                    float* gp = gi + ch * N + xi;
                                    *gp = __fsub_rn(*gp, __fmul_rn(w, d));
                                }
                            }
                        }
                    }
                }
                nA[s] = acc;
                if (owned) Gout[xi] = acc;
                if (do_img && code != 0 && l >= 1) {
                    // own parent in the previous line of the forward sweep
                    const int kk = code - 1;
                    const int dp = (a.ndim == 3) ? (kk / 3 - 1) : 0, dq = kk % 3 - 1;
                    const int64_t ya = xa - g.dir;
                    const int64_t yi = ya * g.sl + (p + dp) * g.sp + (q + dq) * g.sq;
                    const float c = cost_of(nI + s, region, img + yi, N, C, g.t[kk], lam);
                    if (c > 0.0f) {
                        const float w = __fdiv_rn(__fmul_rn(acc, lam), c);
                        for (int64_t ch = 0; ch < C; ++ch) {
                            const float d = __fsub_rn(nI[ch * region + s], __ldg(img + ch * N + yi));
                            float* gp = gi + ch * N + xi;
                            *gp = __fadd_rn(*gp, __fmul_rn(w, d));
                        }
                    }
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u64(myflag, atag(T - 1 - t_app, blk + 1));
        }
    }
    return true;
}

__global__ void __launch_bounds__(kThreads, 2) adjoint_kernel(const AdjointArgs a) {
    extern __shared__ float smem[];
    const int T = a.iterations * a.npass;
    const int64_t total = a.B * a.N;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < total; i += nth) a.G[0][i] = a.grad_dist[i];
    if (a.grad_image)
        for (int64_t i = tid; i < total * a.C; i += nth) a.grad_image[i] = 0.0f;
    unsigned int epoch = 1;
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    for (int t_app = T - 1; t_app >= 0; --t_app) {
        const PassGeom& g = a.pass[t_app % a.npass];
        const int ntiles = g.ntp * g.ntq;
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        bool alive = true;
        for (int64_t w = 0; w < nwaves && alive; ++w) {
            if ((int)blockIdx.x < per_wave * ntiles) {
                const int64_t b = w * per_wave + blockIdx.x / ntiles;
                if (b < a.B) alive = adjoint_tile(a, g, t_app, T, b, blockIdx.x % ntiles, smem);
            }
        }
        if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    }
    // dL/dM = v * (adjoint of D0): elements whose first-pass value came from
    // a parent pass their adjoint on and keep none
    if (a.grad_mask) {
        const float* A0 = a.G[T & 1];
        for (int64_t i = tid; i < total; i += nth) {
            float gv = A0[i];
            if (T > 0) {
                if (a.codes[i] != 0) gv = 0.0f;  // codes of pass application 0: [0][b][r]
            }
            a.grad_mask[i] = __fmul_rn(a.v, gv);
        }
    }
}

}  // namespace

int adjoint_max_blocks_per_sm(size_t smem, int* blocks) {
    if (cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, adjoint_kernel, kThreads, smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    return FGX_OK;
}

int launch_adjoint(const AdjointArgs& a, int grid, size_t smem, void* stream) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, adjoint_kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
