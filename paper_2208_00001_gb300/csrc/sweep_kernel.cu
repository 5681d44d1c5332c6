// Forward raster-scan sweep (FastGeodis, Implementation section): every pass
// updates the elements of one line from the already-updated previous line;
// the schedule of 4 (2D) or 6 (3D) passes repeats `iterations` times.
//
// Decomposition on the GPU.  One cooperative persistent launch runs the whole
// schedule.  For each pass the line domain (P x Q elements) is cut into tiles;
// each thread block owns one tile of one instance and sweeps the pass in
// blocks of K lines.  Within a block the thread block computes its tile plus
// a ring of K elements on every side from a copy of the previous line held in
// shared memory; the ring shrinks by one element per line (the dependency
// cone), so after K lines the tile's own values are exact without any
// exchange.  Between blocks, tiles publish a progress tag in global memory
// and wait (bounded) for their neighbours' tags before reloading the ring.
// Ring elements are recomputed with the same operations, so results stay
// bit-exact.  Passes are separated by a grid barrier.
#include <cuda_runtime.h>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;

__device__ __forceinline__ unsigned long long tag(int t_app, int blk) {
    return ((unsigned long long)(t_app + 1) << 32) | (unsigned int)blk;
}

// One tile of one instance for one pass application.  Returns false if a
// neighbour wait failed.
__device__ bool sweep_tile(const SweepArgs& a, const PassGeom& g, int t_app, int64_t b,
                           int tile, float* smem) {
    __shared__ int ok;
    const int jp = tile / g.ntq, jq = tile % g.ntq;
    const int64_t p0 = (int64_t)jp * g.tp, p1 = mn64(g.P, p0 + g.tp);
    const int64_t q0 = (int64_t)jq * g.tq, q1 = mn64(g.Q, q0 + g.tq);
    const int64_t L = g.L, P = g.P, Q = g.Q, N = a.N, C = a.C;
    const float* img = a.image + b * C * N;
    float* dist = a.dist + b * N;
    uint8_t* codes = a.codes ? a.codes + ((int64_t)t_app * a.B + b) * N : nullptr;
    unsigned long long* myflag = a.flags + b * a.max_tiles + tile;
    const int region = a.smem_region;
    float* bufD[2] = {smem, smem + region};
    float* bufI[2] = {smem + 2 * region, smem + (2 + C) * region};
    const float lam = a.lambda;
    const int dpmin = (a.ndim == 3) ? -1 : 0, dpmax = (a.ndim == 3) ? 1 : 0;

    if (L <= 1) return true;
    const int nblk = (int)((L - 1 + g.K - 1) / g.K);
    for (int blk = 0; blk < nblk; ++blk) {
        const int64_t l0 = 1 + (int64_t)blk * g.K;
        const int nb = (int)mn64(g.K, L - l0);
        if (blk > 0) {
            if (threadIdx.x == 0) {
                ok = 1;
                const unsigned long long want = tag(t_app, blk);
                for (int dj = -1; dj <= 1 && ok; ++dj) {
                    for (int di = -1; di <= 1 && ok; ++di) {
                        if (dj == 0 && di == 0) continue;
                        const int np = jp + dj, nq = jq + di;
                        if (np < 0 || np >= g.ntp || nq < 0 || nq >= g.ntq) continue;
                        if (!wait_tag(a.flags + b * a.max_tiles + np * g.ntq + nq, want,
                                      a.status, a.timeout_ns))
                            ok = 0;
                    }
                }
            }
            __syncthreads();
            if (!ok) return false;
        }
        // region of the previous line needed by this block: tile + ring of nb
        const int64_t rp0 = mx64(0, p0 - nb), rp1 = mn64(P, p1 + nb);
        const int64_t rq0 = mx64(0, q0 - nb), rq1 = mn64(Q, q1 + nb);
        const int64_t rw = rq1 - rq0;
        {
            const int64_t ya = (g.dir > 0) ? (l0 - 1) : (L - l0);
            const int64_t n = (rp1 - rp0) * rw;
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                const int64_t p = rp0 + e / rw, q = rq0 + e % rw;
                const int64_t yi = ya * g.sl + p * g.sp + q * g.sq;
                bufD[0][e] = __ldcg(dist + yi);
                for (int64_t ch = 0; ch < C; ++ch) bufI[0][ch * region + e] = __ldg(img + ch * N + yi);
            }
        }
        __syncthreads();
        int cur = 0;
        for (int i = 0; i < nb; ++i) {
            const int r = nb - 1 - i;
            const int64_t cp0 = mx64(0, p0 - r), cp1 = mn64(P, p1 + r);
            const int64_t cq0 = mx64(0, q0 - r), cq1 = mn64(Q, q1 + r);
            const int64_t cw = cq1 - cq0, n = (cp1 - cp0) * cw;
            const int64_t l = l0 + i;
            const int64_t xa = (g.dir > 0) ? l : (L - 1 - l);
            const float* pD = bufD[cur];
            const float* pI = bufI[cur];
            float* nD = bufD[cur ^ 1];
            float* nI = bufI[cur ^ 1];
            for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
                const int64_t p = cp0 + e / cw, q = cq0 + e % cw;
                const int64_t xi = xa * g.sl + p * g.sp + q * g.sq;
                const int64_t s = (p - rp0) * rw + (q - rq0);  // slot in region buffers
                for (int64_t ch = 0; ch < C; ++ch) nI[ch * region + s] = __ldg(img + ch * N + xi);
                float best = __ldcg(dist + xi);
                int code = 0;
                int k = 0;
                for (int dp = dpmin; dp <= dpmax; ++dp) {
                    for (int dq = -1; dq <= 1; ++dq, ++k) {
                        const int64_t yp = p + dp, yq = q + dq;
                        if (yp < 0 || yp >= P || yq < 0 || yq >= Q) continue;
                        const int64_t ys = (yp - rp0) * rw + (yq - rq0);
                        float di2 = 0.0f;
                        for (int64_t ch = 0; ch < C; ++ch) {
                            const float d = __fsub_rn(nI[ch * region + s], pI[ch * region + ys]);
                            di2 = __fadd_rn(di2, __fmul_rn(d, d));
                        }
                        const float c = __fsqrt_rn(__fadd_rn(g.t[k], __fmul_rn(lam, di2)));
                        const float cand = __fadd_rn(pD[ys], c);
                        if (cand < best) code = k + 1;
                        best = fminf(best, cand);
                    }
                }
                nD[s] = best;
                if (p >= p0 && p < p1 && q >= q0 && q < q1) {
                    dist[xi] = best;
                    if (codes) codes[xi] = (uint8_t)code;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u64(myflag, tag(t_app, blk + 1));
        }
    }
    return true;
}

__global__ void __launch_bounds__(kThreads) sweep_kernel(const SweepArgs a) {
    extern __shared__ float smem[];
    // D0 = v * M (generalised GDT with soft seeds)
    const int64_t total = a.B * a.N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        a.dist[i] = __fmul_rn(a.v, a.mask[i]);
    unsigned int epoch = 1;
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    const int napps = a.iterations * a.npass;
    for (int t_app = 0; t_app < napps; ++t_app) {
        const PassGeom& g = a.pass[t_app % a.npass];
        const int ntiles = g.ntp * g.ntq;
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        for (int64_t w = 0; w < nwaves; ++w) {
            if ((int)blockIdx.x < per_wave * ntiles) {
                const int64_t b = w * per_wave + blockIdx.x / ntiles;
                if (b < a.B && !sweep_tile(a, g, t_app, b, blockIdx.x % ntiles, smem)) return;
            }
        }
        if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    }
}

}  // namespace

int sweep_max_blocks_per_sm(size_t smem, int* blocks) {
    if (cudaFuncSetAttribute(sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, sweep_kernel, kThreads, smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    return FGX_OK;
}

int launch_sweep(const SweepArgs& a, int grid, size_t smem, void* stream) {
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
    if (cudaLaunchKernelEx(&cfg, sweep_kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
