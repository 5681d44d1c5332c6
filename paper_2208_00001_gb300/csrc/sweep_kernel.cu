// Forward raster-scan sweep on line tiles (FastGeodis, Implementation
// section): every pass updates the elements of one line from the
// already-updated previous line; the schedule of 4 (2D) or 6 (3D) passes
// repeats `iterations` times.  This engine serves every shape (2D and 3D,
// several instances, optional parent-code recording) and the batched launch.
//
// Decomposition.  One cooperative persistent launch runs the whole schedule.
// For each pass the line domain (P x Q elements) is cut into tiles; a thread
// block owns one tile of one instance and sweeps the pass in blocks of K
// lines.  Within a block it computes its tile plus a ring of K elements on
// every side from the previous line held in shared memory; the ring shrinks
// by one element per line (the dependency cone), so after K lines the tile's
// own values are exact without any exchange.  Between blocks, tiles publish a
// progress tag and wait (bounded) for their neighbours' tags before reloading
// the ring part of the previous line.  Ring elements are recomputed with the
// same operations, so results stay bit-exact.  The old distances and the
// intensities of the next block's K lines are prefetched into shared memory
// with cp.async while the current block computes.  Passes are separated by a
// grid barrier.
#include <cuda_runtime.h>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;

constexpr int kMaxSlots = (kMaxRegion + kThreads - 1) / kThreads;

__device__ __forceinline__ unsigned long long tag(int seq, int blk) {
    return ((unsigned long long)(seq + 1) << 32) | (unsigned int)blk;
}

__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Cost modes of the tiled engine, fixed per call on the host:
//  kCostGeneral: c = sqrt(t_k + lambda * sum_ch (I(x)-I(y))^2)
//  kCostAbs:     lambda = 1 and one channel: c = sqrt_rn(fl(d*d)) = |d| exactly
//                for 2^-63 <= |d| <= 2^63 and d = 0 (square root elsewhere)
//  kCostConst:   lambda = 0: c = sqrt_rn(t_k), the pass's constant per offset
//  kCostFast:    the general formula with fused multiply-adds and the
//                approximate square root (fast-math option)
// Offsets are unrolled at compile time; the shared previous-line buffers carry
// a one-element border of +inf so that neighbours outside the domain never
// win the min and need no bounds test.
template <int NDIM, int MODE, bool CODES>
__device__ bool sweep_tile(const TileJob& j, const PassGeom& g, float* smem) {
    __shared__ int ok;
    constexpr int DPMIN = (NDIM == 3) ? -1 : 0, DPMAX = (NDIM == 3) ? 1 : 0;
    constexpr int PADP = (NDIM == 3) ? 1 : 0;
    const int jp = j.tile / g.ntq, jq = j.tile % g.ntq;
    const int P = (int)g.P, Q = (int)g.Q, L = (int)g.L, K = g.K;
    const int p0 = jp * g.tp, p1 = min(P, p0 + g.tp);
    const int q0 = jq * g.tq, q1 = min(Q, q0 + g.tq);
    const int C = j.C, R = j.region, KM = j.kmax;
    const int CI = (MODE == kCostConst) ? 0 : C;  // intensity planes kept in shared memory
    const int64_t N = j.N;
    const float lam = j.lambda;
    if (L <= 1) return true;

    // fixed tile region: tile + ring of K (clipped to the domain), padded by 1
    const int rp0 = max(0, p0 - K), rp1 = min(P, p1 + K);
    const int rq0 = max(0, q0 - K), rq1 = min(Q, q1 + K);
    const int rw = rq1 - rq0, rn = (rp1 - rp0) * rw;
    const int pw = rw + 2, ph = (rp1 - rp0) + 2 * PADP;

    float* prevD[2] = {smem, smem + R};
    float* prevI[2] = {smem + 2 * R, smem + (2 + CI) * R};
    float* slab = smem + (2 + 2 * CI) * R;  // [2 bufs][1 + CI planes][KM lines][R]
    auto slab_at = [&](int buf, int plane, int line) {
        return slab + ((size_t)(buf * (1 + CI) + plane) * KM + line) * R;
    };

    // borders: +inf distances (and zero intensities) around the region
    for (int idx = threadIdx.x; idx < ph * pw; idx += kThreads) {
        const int pr = idx / pw, pc = idx % pw;
        const bool border = pc == 0 || pc == pw - 1 || (PADP && (pr == 0 || pr == ph - 1));
        if (border) {
            prevD[0][idx] = __int_as_float(0x7f800000);
            prevD[1][idx] = __int_as_float(0x7f800000);
            for (int ch = 0; ch < CI; ++ch) {
                prevI[0][ch * R + idx] = 0.0f;
                prevI[1][ch * R + idx] = 0.0f;
            }
        }
    }

    // per-thread slots: padded index, distance outside the tile, line offset
    int sl_e[kMaxSlots], sl_ring[kMaxSlots];
    int64_t sl_off[kMaxSlots];
#pragma unroll
    for (int k = 0; k < kMaxSlots; ++k) {
        const int e = threadIdx.x + k * kThreads;
        const int pr = e < rn ? e / rw : 0, pc = e < rn ? e % rw : 0;
        sl_e[k] = e < rn ? (pr + PADP) * pw + pc + 1 : -1;
        const int p = rp0 + pr, q = rq0 + pc;
        sl_off[k] = (int64_t)p * g.sp + (int64_t)q * g.sq;
        sl_ring[k] = max(max(max(p0 - p, p - (p1 - 1)), max(q0 - q, q - (q1 - 1))), 0);
    }
    auto line_off = [&](int l) -> int64_t {
        return (int64_t)((g.dir > 0) ? l : (L - 1 - l)) * g.sl;
    };
    // prefetch the old distances (and intensities) of lines l0 .. l0+nb-1
    auto fill = [&](int buf, int l0, int nb) {
        for (int i = 0; i < nb; ++i) {
            const int64_t lo = line_off(l0 + i);
#pragma unroll
            for (int k = 0; k < kMaxSlots; ++k) {
                if (sl_e[k] < 0) continue;
                cp_async4(slab_at(buf, 0, i) + sl_e[k], j.dist + lo + sl_off[k]);
                for (int ch = 0; ch < CI; ++ch)
                    cp_async4(slab_at(buf, 1 + ch, i) + sl_e[k], j.img + ch * N + lo + sl_off[k]);
            }
        }
        cp_commit();
    };

    const int nblk = (L - 1 + K - 1) / K;
    int cur = 0;
    fill(0, 1, min(K, L - 1));
    for (int blk = 0; blk < nblk; ++blk) {
        const int l0 = 1 + blk * K;
        const int nb = min(K, L - l0);
        const bool more = blk + 1 < nblk;
        if (more) fill((blk + 1) & 1, l0 + K, min(K, L - l0 - K));
        // previous line: all of it for the first block; afterwards only the
        // ring, once the neighbouring tiles have published it
        if (blk > 0) {
            // threads 0..8 each wait for one of the (up to 8) neighbouring tiles
            if (threadIdx.x == 0) ok = 1;
            __syncthreads();
            if (threadIdx.x < 9 && threadIdx.x != 4) {
                const int np = jp + (int)threadIdx.x / 3 - 1, nq = jq + (int)threadIdx.x % 3 - 1;
                if (np >= 0 && np < g.ntp && nq >= 0 && nq < g.ntq &&
                    !wait_tag(j.flags + np * g.ntq + nq, tag(j.seq, blk), j.status, j.timeout_ns))
                    ok = 0;
            }
            __syncthreads();
            if (!ok) {
                cp_wait_all();
                return false;
            }
        }
        {
            const int64_t lo = line_off(l0 - 1);
#pragma unroll
            for (int k = 0; k < kMaxSlots; ++k) {
                const int e = sl_e[k];
                if (e < 0 || (blk > 0 && sl_ring[k] == 0)) continue;
                prevD[cur][e] = __ldcg(j.dist + lo + sl_off[k]);
                for (int ch = 0; ch < CI; ++ch)
                    prevI[cur][ch * R + e] = __ldg(j.img + ch * N + lo + sl_off[k]);
            }
        }
        if (more) cp_wait_all_but_one(); else cp_wait_all();
        __syncthreads();
        const int buf = blk & 1;
        for (int i = 0; i < nb; ++i) {
            const int r = K - 1 - i;  // valid radius of the ring on this line
            const int64_t lo = line_off(l0 + i);
            const float* pD = prevD[cur];
            const float* pI = prevI[cur];
            float* nD = prevD[cur ^ 1];
            float* nI = prevI[cur ^ 1];
            const float* sD = slab_at(buf, 0, i);
            const float* sI = slab_at(buf, 1, i);
#pragma unroll
            for (int k = 0; k < kMaxSlots; ++k) {
                const int e = sl_e[k];
                if (e < 0 || sl_ring[k] > r) continue;
                float best = sD[e];
                int code = 0;
                float Ix0 = 0.0f;
                if (MODE == kCostAbs) Ix0 = sI[e];
#pragma unroll
                for (int dp = DPMIN; dp <= DPMAX; ++dp) {
#pragma unroll
                    for (int dq = -1; dq <= 1; ++dq) {
                        const int bit = (dp - DPMIN) * 3 + (dq + 1);
                        const int ys = e + dp * pw + dq;
                        float c;
                        if (MODE == kCostConst) {
                            c = g.c[bit];
                        } else if (MODE == kCostAbs) {
                            const float d = __fsub_rn(Ix0, pI[ys]);
                            const float ad = fabsf(d);
                            const unsigned int ub = __float_as_uint(ad);
                            if ((ub - 0x20000000u) <= 0x3F000000u || ub == 0u) c = ad;
                            else c = __fsqrt_rn(__fmul_rn(d, d));
                        } else if (MODE == kCostFast) {
                            float di2 = 0.0f;
                            for (int ch = 0; ch < C; ++ch) {
                                const float d = __fsub_rn(sI[(size_t)ch * KM * R + e],
                                                          pI[ch * R + ys]);
                                di2 = __fmaf_rn(d, d, di2);
                            }
                            c = fast_sqrt(__fmaf_rn(lam, di2, g.t[bit]));
                        } else {
                            float di2 = 0.0f;
                            for (int ch = 0; ch < C; ++ch) {
                                const float d = __fsub_rn(sI[(size_t)ch * KM * R + e],
                                                          pI[ch * R + ys]);
                                di2 = __fadd_rn(di2, __fmul_rn(d, d));
                            }
                            c = __fsqrt_rn(__fadd_rn(g.t[bit], __fmul_rn(lam, di2)));
                        }
                        const float cand = __fadd_rn(pD[ys], c);
                        if (CODES && cand < best) code = bit + 1;
                        best = fminf(best, cand);
                    }
                }
                nD[e] = best;
                for (int ch = 0; ch < CI; ++ch) nI[ch * R + e] = sI[(size_t)ch * KM * R + e];
                if (sl_ring[k] == 0) {
                    j.dist[lo + sl_off[k]] = best;
                    if (CODES) j.codes[lo + sl_off[k]] = (uint8_t)code;
                }
            }
            __syncthreads();
            cur ^= 1;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u64(j.flags + j.tile, tag(j.seq, blk + 1));
        }
    }
    return true;
}

// Picks the compiled variant for the call's dimensionality, cost mode and
// whether parent codes are recorded.
__device__ bool run_tile(int ndim, int mode, const TileJob& j, const PassGeom& g, float* smem) {
    const bool codes = j.codes != nullptr;
#define FGX_TILE(N, M)                                                   \
    return codes ? sweep_tile<N, M, true>(j, g, smem) : sweep_tile<N, M, false>(j, g, smem)
    if (ndim == 3) {
        if (mode == kCostAbs) FGX_TILE(3, kCostAbs);
        if (mode == kCostConst) FGX_TILE(3, kCostConst);
        if (mode == kCostFast) FGX_TILE(3, kCostFast);
        FGX_TILE(3, kCostGeneral);
    }
    if (mode == kCostAbs) FGX_TILE(2, kCostAbs);
    if (mode == kCostConst) FGX_TILE(2, kCostConst);
    if (mode == kCostFast) FGX_TILE(2, kCostFast);
    FGX_TILE(2, kCostGeneral);
#undef FGX_TILE
}

__global__ void __launch_bounds__(kThreads, 2) sweep_kernel(const SweepArgs a) {
    extern __shared__ float smem[];
    // D0 = v * M (generalised GDT with soft seeds)
    const int64_t total = a.B * a.N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        a.dist[i] = __fmul_rn(a.v, a.mask[i]);
    unsigned int epoch = 1;
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[0] = (unsigned long long)gtimer();
    const int napps = a.iterations * a.npass;
    for (int t_app = 0; t_app < napps; ++t_app) {
        const PassGeom& g = a.pass[t_app % a.npass];
        const int ntiles = g.ntp * g.ntq;
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        bool alive = true;
        for (int64_t w = 0; w < nwaves && alive; ++w) {
            if ((int)blockIdx.x < per_wave * ntiles) {
                const int64_t b = w * per_wave + blockIdx.x / ntiles;
                if (b < a.B) {
                    TileJob j;
                    j.img = a.image + (b % a.nimg) * a.C * a.N;
                    j.dist = a.dist + b * a.N;
                    j.codes = a.codes ? a.codes + ((int64_t)t_app * a.B + b) * a.N : nullptr;
                    j.flags = a.flags + b * a.max_tiles;
                    j.N = a.N;
                    j.C = (int)a.C;
                    j.ndim = a.ndim;
                    j.lambda = a.lambda;
                    j.seq = t_app;
                    j.tile = blockIdx.x % ntiles;
                    j.region = a.smem_region;
                    j.kmax = a.kmax;
                    j.status = a.status;
                    j.timeout_ns = a.timeout_ns;
                    alive = run_tile(a.ndim, a.cost_mode, j, g, smem);
                }
            }
        }
        if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 1 < 16)
            timeline[t_app + 1] = (unsigned long long)gtimer();
    }
}

// Batched launch: every instance's D0 = v * M, then rounds of one pass
// application per active instance, waves of whole instances per round, and a
// grid barrier between rounds.
__global__ void __launch_bounds__(kThreads, 2) batched_kernel(const BatchedArgs a) {
    extern __shared__ float smem[];
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    for (int i = 0; i < a.n; ++i) {
        const InstDesc& d = a.desc[i];
        for (int64_t e = tid; e < d.N; e += nth) d.dist[e] = __fmul_rn(d.v, d.mask[e]);
    }
    unsigned int epoch = 1;
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    for (int r = 0; r < a.rounds; ++r) {
        bool alive = true;
        for (int w = a.round_waves[r]; w < a.round_waves[r + 1] && alive; ++w) {
            const int item = a.wave_items[(int64_t)w * gridDim.x + blockIdx.x];
            if (item < 0) continue;
            const InstDesc& d = a.desc[item >> 16];
            const PassGeom& g = d.pass[r % d.npass];
            TileJob j;
            j.img = d.image;
            j.dist = d.dist;
            j.codes = nullptr;
            j.flags = a.flags + d.flags_off;
            j.N = d.N;
            j.C = d.C;
            j.ndim = d.ndim;
            j.lambda = d.lambda;
            j.seq = r;
            j.tile = item & 0xffff;
            j.region = d.region;
            j.kmax = d.kmax;
            j.status = a.status;
            j.timeout_ns = a.timeout_ns;
            alive = run_tile(d.ndim, d.cost_mode, j, g, smem);
        }
        if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return;
    }
}

}  // namespace

size_t sweep_smem_bytes(int64_t C, int region, int kmax) {
    return (size_t)(2 + 2 * C) * (size_t)(1 + kmax) * (size_t)region * sizeof(float);
}

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

int batched_max_blocks_per_sm(size_t smem, int* blocks) {
    if (cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, batched_kernel, kThreads, smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    return FGX_OK;
}

int launch_batched(const BatchedArgs& a, int grid, size_t smem, void* stream) {
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
    if (cudaLaunchKernelEx(&cfg, batched_kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
