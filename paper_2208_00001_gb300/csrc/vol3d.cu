// 3D forward on register-blocked plane tiles (FastGeodis, Implementation
// section: six passes per iteration, every voxel of a plane updated from the
// nine voxels of the already-updated previous plane).
//
// Decomposition.  One cooperative persistent launch runs all passes.  For a
// pass along one axis the plane (P x Q voxels) is cut into tiles of
// kTP x kTQ owned voxels; one thread block per tile computes a region of
// kRP x kRQ = 32 x 32 voxels: the tile plus a ring of kRing voxels on every
// side.  Eight compute warps each hold four region rows: lane q owns column q
// of the region and keeps the four distances of its rows in registers.  A
// plane step needs the 3 x 3 parents of every voxel: the own column's rows
// come from registers plus the two boundary rows of the warps above and below
// (shared memory, one named barrier of the compute warps per step), the
// neighbouring columns by warp shuffles.  Old distances and intensities of
// upcoming planes are staged in shared memory by four producer warps with
// cp.async (chunks of kChunk planes, one mbarrier per chunk).  The dependency
// cone shrinks the exact part of the region by one voxel per side and step,
// so the owned voxels stay exact for kRing steps; then every block publishes
// its owned voxels as 64-bit (value, tag) words and refreshes its ring from
// the owners' words (bounded polling, no fences: every word carries its own
// tag).  Passes are separated by a grid barrier.  Ring voxels are recomputed
// with exactly the operations of their owners, so results stay bit-exact.
//
// Edge costs are evaluated on the fly in the fixed order of the method:
//  constant (lambda = 0): sqrt(t_k), one constant per stencil offset;
//  absolute (lambda = 1, one channel): |I(x) - I(y)|, which equals
//    sqrt_rn(fl(d*d)) for d = 0 and 2^-63 <= |d| <= 2^63; a first kernel
//    checks that every intensity is 0 or has magnitude in [2^-40, 2^62],
//    which bounds every difference to that range; otherwise each candidate
//    is checked and falls back to the square root;
//  general: sqrt_rn(t_k + lambda * sum_ch (I(x)-I(y))^2).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;

constexpr int kRows = 4;                  // region rows per compute thread
constexpr int kCW = 8;                    // compute warps
constexpr int kPW = 4;                    // producer warps
constexpr int kRP = kRows * kCW;          // region rows
constexpr int kRQ = 32;                   // region columns (one per lane)
constexpr int kRing = 4;                  // ring width = steps between refreshes
constexpr int kTP = kRP - 2 * kRing;      // owned rows of a tile
constexpr int kTQ = kRQ - 2 * kRing;      // owned columns of a tile
constexpr int kPlane = kRP * kRQ;         // region voxels
constexpr int kChunk = kRing;             // planes per staging chunk
constexpr int kNst = 3;                   // chunks in the staging ring
constexpr int kMaxCI = 3;                 // intensity channels the stage holds
constexpr int kBlock3 = (kCW + kPW) * 32;
constexpr int kXWords = kTP * kTQ;        // published words per tile and parity
constexpr int kRangeFlagOffset = 32;      // workspace header: intensity range flag
constexpr int kTransposeWarps = 8;        // warps of a block that transpose (8 shared tiles)
#define kInf3 __int_as_float(0x7f800000)

enum { kModeConst = 0, kModeAbs = 1, kModeGeneral = 2 };

struct Vol3DArgs {
    const float* image;  // [B][C][N]
    const float* mask;   // [B][N]
    float* dist;         // [B][N]
    uint8_t* codes;      // [iterations * 6][B][N] parent codes, or null
    int64_t B, C, N;
    float v, lambda;
    int iterations;
    int mode;
    PassGeom pass[kMaxPasses];
    int ntp[kMaxPasses], ntq[kMaxPasses];
    int max_tiles;
    unsigned long long* xbuf;  // [B][max_tiles][2 parities][kXWords]
    unsigned int* barrier;
    int* status;
    const int* range_flag;     // nonzero: some intensity outside the |d| range
    long long timeout_ns;
    // W passes on transposed copies (planes of those passes have H as their
    // contiguous axis, so staging loads and result stores are coalesced):
    float* distT;              // [B][W][D][H], or null (W passes on dist itself)
    float* imageT;             // [B][C][W][D][H] (cost modes that read intensities)
    int64_t D, H, W;
};

struct Head3 {
    unsigned long long full[kNst], empty[kNst];
    float rowtop[2][kCW][kRQ];  // first row of each warp, per step parity
    float rowbot[2][kCW][kRQ];  // last row of each warp
};
static_assert(sizeof(Head3) % 16 == 0, "stage must stay 16-byte aligned");

__device__ __align__(16) unsigned int g_inf4[4] = {0x7f800000u, 0x7f800000u, 0x7f800000u,
                                                  0x7f800000u};
__device__ __align__(16) unsigned int g_zero4v[4] = {0u, 0u, 0u, 0u};

__device__ __forceinline__ unsigned int saddr3(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr3(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_arrive_noinc(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr3(b))
                 : "memory");
}
__device__ __forceinline__ void cp_wait_all3() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void mbar_init3(unsigned long long* b, unsigned int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr3(b)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive3(unsigned long long* b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(saddr3(b))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try3(unsigned long long* b, unsigned int parity) {
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr3(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of parity `parity` of *b (false on timeout or
// an earlier failure recorded in the status word).
__device__ __noinline__ bool mbar_wait3(unsigned long long* b, unsigned int parity, int* status,
                                        long long timeout_ns) {
    if (mbar_try3(b, parity)) return true;
    const long long t0 = gtimer();
    for (;;) {
        if (mbar_try3(b, parity)) return true;
        if (status_of(status) != 0) return false;
        if (gtimer() - t0 > timeout_ns) {
            record_timeout(status);
            return false;
        }
    }
}
// Compute-warp barrier (the producer warps never join it).
__device__ __forceinline__ void compute_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory");
}

// Position of one tile of one pass application.
struct Tile3 {
    const PassGeom* g;
    float* dist;       // distances of this instance in the pass's layout
    const float* img;  // intensities of this instance in the pass's layout
    int64_t csl, csp, csq;  // strides of line, p and q in the image order of the codes
    int jp, jq, ntq, tile;
    int64_t b;
    int L, nch;
    int64_t p0, q0;  // plane coordinates of region row 0 and column 0
};

__device__ __forceinline__ float* stage_plane(float* stage, int slot, int j, int arr, int CI) {
    return stage + ((size_t)(slot * kChunk + j) * (1 + CI) + arr) * kPlane;
}

// Producer warps: planes of old distances and intensities into the staging
// ring, chunk after chunk, once the compute warps have released the slot.
// Voxels outside the volume are staged with distance +inf and intensity 0
// (finite costs: a square root never sees an infinite argument).
template <int CI>
__device__ bool producer3(const Vol3DArgs& a, const Tile3& t, Head3& h, float* stage,
                          unsigned int cb) {
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31, pw = (threadIdx.x >> 5) - kCW;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const float* img = t.img;
    const float* dist = t.dist;
    for (int c = 0; c < t.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = (int)(gc % kNst);
        if (gc >= (unsigned)kNst &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.empty[slot], ((gc / kNst) & 1u) ^ 1u,
                                                a.status, a.timeout_ns))) {
            cp_wait_all3();
            return false;
        }
        const int jn = min(kChunk, t.L - c * kChunk);
        for (int j = 0; j < jn; ++j) {
            const int s = c * kChunk + j;
            const int64_t line = g.dir > 0 ? s : (t.L - 1 - s);
#pragma unroll
            for (int rr = 0; rr < kRP / kPW; ++rr) {
                const int r = pw + kPW * rr;
                const int64_t p = t.p0 + r;
                const bool in = qin && p >= 0 && p < g.P;
                const int64_t off = line * g.sl + p * g.sp + q * g.sq;
                float* dst = stage_plane(stage, slot, j, 0, CI) + r * kRQ + lane;
                cp_async4(dst, in ? (const void*)(dist + off) : (const void*)g_inf4);
#pragma unroll
                for (int ch = 0; ch < CI; ++ch)
                    cp_async4(dst + (ch + 1) * kPlane,
                              in ? (const void*)(img + ch * a.N + off) : (const void*)g_zero4v);
            }
        }
        cp_arrive_noinc(&h.full[slot]);
    }
    return true;
}

// Exchange area and failure reporting of one launch.
struct XLink3 {
    unsigned long long* xbuf;  // [B][max_tiles][2 parities][kXWords]
    int max_tiles;
    int* status;
    long long timeout_ns;
};

// Ring refresh after step s: publish the owned voxels of plane s, then take
// every ring voxel inside the volume from the tile that owns it.
__device__ bool exchange3(const XLink3& a, const Tile3& t, int w, unsigned int tg, int par,
                          float (&d)[kRows]) {
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31;
    unsigned long long* base = a.xbuf + (size_t)t.b * a.max_tiles * 2 * kXWords;
    unsigned long long* mine = base + ((size_t)t.tile * 2 + par) * kXWords;
    const bool qown = lane >= kRing && lane < kRing + kTQ;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const unsigned long long* src[kRows];
    bool need[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = w * kRows + i;
        const bool pown = r >= kRing && r < kRing + kTP;
        const unsigned long long word =
            ((unsigned long long)tg << 32) | (unsigned int)__float_as_uint(d[i]);
        if (pown && qown) st_relaxed_u64(mine + (r - kRing) * kTQ + (lane - kRing), word);
        const int64_t p = t.p0 + r;
        need[i] = !(pown && qown) && qin && p >= 0 && p < g.P;
        src[i] = nullptr;
        if (need[i]) {
            const int op = (int)(p / kTP), oq = (int)(q / kTQ);
            const int lr = (int)(p - (int64_t)op * kTP), lq = (int)(q - (int64_t)oq * kTQ);
            src[i] = base + ((size_t)(op * t.ntq + oq) * 2 + par) * kXWords + lr * kTQ + lq;
        }
    }
    long long t0 = 0;
    for (unsigned int it = 0;; ++it) {
        bool done = true;
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            if (!need[i]) continue;
            const unsigned long long wv = ld_relaxed_u64(src[i]);
            if ((unsigned int)(wv >> 32) == tg) {
                d[i] = __uint_as_float((unsigned int)wv);
                need[i] = false;
            } else {
                done = false;
            }
        }
        if (__all_sync(0xffffffffu, done)) return true;
        // the status word and the clock are read every 16th poll only
        if ((it & 15u) == 15u) {
            int fail = 0;
            if (lane == 0) {
                const long long now = gtimer();
                if (t0 == 0) t0 = now;
                if (status_of(a.status) != 0) fail = 1;
                else if (now - t0 > a.timeout_ns) {
                    record_timeout(a.status);
                    fail = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, fail, 0)) return false;
        }
    }
}

// Edge cost of one parent, in the fixed arithmetic order of the method.
template <int MODE, int CI, bool CHECKED>
__device__ __forceinline__ float cost3(const float (&ix)[CI > 0 ? CI : 1],
                                       const float (&iy)[CI > 0 ? CI : 1], float t, float c0,
                                       float lam) {
    if (MODE == kModeConst) return c0;
    if (MODE == kModeAbs) {
        const float d = __fsub_rn(ix[0], iy[0]);
        const float ad = fabsf(d);
        if (!CHECKED) return ad;
        const unsigned int ub = __float_as_uint(ad);
        if ((ub - 0x20000000u) <= 0x3F000000u || ub == 0u) return ad;
        return __fsqrt_rn(__fmul_rn(d, d));
    }
    float di2 = 0.0f;
#pragma unroll
    for (int ch = 0; ch < CI; ++ch) {
        const float d = __fsub_rn(ix[ch], iy[ch]);
        di2 = ch == 0 ? __fmul_rn(d, d) : __fadd_rn(di2, __fmul_rn(d, d));
    }
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// Compute warps of one tile: plane steps 1 .. L-1, ring refresh every kRing
// steps, owned voxels written to the distance map (and with CODES their
// parent codes: 0 if the voxel kept its value, else 1 + the lowest stencil
// offset whose candidate is the strictly smaller minimum).
template <int MODE, int CI, bool CHECKED, bool CODES>
__device__ bool compute3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h, float* stage,
                         unsigned int cb) {
    constexpr int NI = CI > 0 ? CI : 1;
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const bool qown = lane >= kRing && lane < kRing + kTQ;
    bool valid[kRows], own[kRows];
    int64_t goff[kRows], goffc[CODES ? kRows : 1];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = w * kRows + i;
        const int64_t p = t.p0 + r;
        valid[i] = qin && p >= 0 && p < g.P;
        own[i] = valid[i] && qown && r >= kRing && r < kRing + kTP;
        goff[i] = p * g.sp + q * g.sq;
        if (CODES) goffc[i] = p * t.csp + q * t.csq;
    }
    float* dist = t.dist;
    uint8_t* codes = CODES ? a.codes + ((int64_t)t_app * a.B + t.b) * a.N : nullptr;
    const float lam = a.lambda;
    float tk[9], ck[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        tk[k] = g.t[k];
        ck[k] = g.c[k];
    }
    // clamped stage columns of the left and right neighbours (their parent
    // distances are +inf where the clamp applies)
    const int cl = max(lane - 1, 0), cr = min(lane + 1, kRQ - 1);
    const int rows0 = w * kRows;

    // After a failure (timeout, or one reported by another block) the warps
    // keep stepping through the named barriers with every wait skipped, so
    // that no compute warp is left waiting for one that gave up.
    bool failed = !__all_sync(0xffffffffu, mbar_wait3(&h.full[cb % kNst], (cb / kNst) & 1u,
                                                      a.status, a.timeout_ns));
    float d[kRows];
    {
        const float* S0 = stage_plane(stage, (int)(cb % kNst), 0, 0, CI);
#pragma unroll
        for (int i = 0; i < kRows; ++i) d[i] = S0[(rows0 + i) * kRQ + lane];
    }
    const unsigned int tag_base = ((unsigned int)(t_app + 1)) << 16;
    int xi = 0;
    for (int s = 1; s < t.L; ++s) {
        const unsigned int gc = cb + s / kChunk;
        const int j = s % kChunk;
        const int slot = (int)(gc % kNst);
        if (j == 0 && !failed &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.full[slot], (gc / kNst) & 1u, a.status,
                                                a.timeout_ns)))
            failed = true;
        // boundary rows of plane s-1 for the warps above and below
        const int rb = s & 1;
        h.rowtop[rb][w][lane] = d[0];
        h.rowbot[rb][w][lane] = d[kRows - 1];
        compute_sync();
        // plane s-2 is no longer read by any compute warp: free its chunk if
        // it was the chunk's last plane
        if (threadIdx.x == 0 && s >= 2 && (s - 2) % kChunk == kChunk - 1)
            mbar_arrive3(&h.empty[(cb + (s - 2) / kChunk) % kNst]);
        float col[kRows + 2], lft[kRows + 2], rgt[kRows + 2];
        col[0] = w > 0 ? h.rowbot[rb][w - 1][lane] : kInf3;
#pragma unroll
        for (int i = 0; i < kRows; ++i) col[i + 1] = d[i];
        col[kRows + 1] = w < kCW - 1 ? h.rowtop[rb][w + 1][lane] : kInf3;
#pragma unroll
        for (int k = 0; k < kRows + 2; ++k) {
            lft[k] = __shfl_up_sync(0xffffffffu, col[k], 1);
            rgt[k] = __shfl_down_sync(0xffffffffu, col[k], 1);
            if (lane == 0) lft[k] = kInf3;
            if (lane == 31) rgt[k] = kInf3;
        }
        // old distances and intensities of plane s, intensities of plane s-1
        const float* Sd = stage_plane(stage, slot, j, 0, CI);
        const unsigned int gcp = cb + (s - 1) / kChunk;
        const int slotp = (int)(gcp % kNst), jp = (s - 1) % kChunk;
        float ip[kRows + 2][3][NI], ix[kRows][NI];
        if (CI > 0) {
#pragma unroll
            for (int k = 0; k < kRows + 2; ++k) {
                const int rr = min(max(rows0 + k - 1, 0), kRP - 1);
#pragma unroll
                for (int ch = 0; ch < CI; ++ch) {
                    const float* Pi = stage_plane(stage, slotp, jp, 1 + ch, CI) + rr * kRQ;
                    ip[k][0][ch] = Pi[cl];
                    ip[k][1][ch] = Pi[lane];
                    ip[k][2][ch] = Pi[cr];
                }
            }
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int ch = 0; ch < CI; ++ch)
                    ix[i][ch] = stage_plane(stage, slot, j, 1 + ch, CI)[(rows0 + i) * kRQ + lane];
        }
        const int64_t line = g.dir > 0 ? s : (t.L - 1 - s);
        const int64_t lo = line * g.sl;
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            float best = Sd[(rows0 + i) * kRQ + lane];
            unsigned int code = 0;
#pragma unroll
            for (int dp = -1; dp <= 1; ++dp) {
#pragma unroll
                for (int dq = -1; dq <= 1; ++dq) {
                    const int k = (dp + 1) * 3 + (dq + 1);
                    const int rk = i + 1 + dp;
                    const float pd = dq < 0 ? lft[rk] : (dq == 0 ? col[rk] : rgt[rk]);
                    const float c = cost3<MODE, CI, CHECKED>(ix[i], ip[rk][dq + 1], tk[k], ck[k],
                                                             lam);
                    const float cand = __fadd_rn(pd, c);
                    if (CODES && cand < best) code = (unsigned int)(k + 1);
                    best = fminf(best, cand);
                }
            }
            d[i] = valid[i] ? best : kInf3;
            if (own[i]) {
                dist[lo + goff[i]] = d[i];
                if (CODES) codes[line * t.csl + goffc[i]] = (uint8_t)code;
            }
        }
        if (s % kRing == 0 && s + 1 < t.L) {
            if (!failed && !exchange3(XLink3{a.xbuf, a.max_tiles, a.status, a.timeout_ns}, t, w,
                                      tag_base | (unsigned int)(xi + 1), xi & 1, d))
                failed = true;
            ++xi;
        }
    }
    // free the chunks still held (those whose last plane is one of the last two)
    compute_sync();
    if (threadIdx.x == 0) {
        const int nch = t.nch;
        for (int c = max(0, nch - 2); c < nch; ++c) {
            const int last = min(c * kChunk + kChunk - 1, t.L - 1);
            if (last >= t.L - 2) mbar_arrive3(&h.empty[(cb + c) % kNst]);
        }
    }
    return !failed;
}

// D0 = v * M, and the intensity range test that allows |d| as the cost.
__global__ void __launch_bounds__(256) init3d_kernel(const float* mask, float* dist, float v,
                                                     int64_t n, const float* image, int64_t ni,
                                                     int* range_flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        dist[i] = __fmul_rn(v, mask[i]);
    if (!range_flag) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += stride) {
        const float x = fabsf(image[i]);
        // 0, or a magnitude in [2^-40, 2^62] (false for NaN and infinity)
        const bool ok = x == 0.0f || (x >= 0x1p-40f && x <= 0x1p62f);
        if (!ok && *(volatile int*)range_flag == 0) atomicOr(range_flag, 1);
    }
}

// Transposes `count` arrays of R x W floats (R = D*H) into W x R (back:
// W x R into R x W).  Each of `nwarps` warps of a block moves whole 32 x 32
// tiles through its own 32 x 33 shared tile (32 loads in flight per lane);
// tiles are spread over all warps of the grid.  The sources may have been
// written by other blocks of the same launch: read through L2.
__device__ void transpose_rw(const float* src, float* dst, int64_t count, int64_t R, int64_t W,
                             bool back, float* smem, int nwarps) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < nwarps) {
        float* tile = smem + warp * (32 * 33);
        const int64_t rows = back ? W : R, cols = back ? R : W;  // of the source
        const int64_t tr = (rows + 31) / 32, tc = (cols + 31) / 32;
        const int64_t ntile = count * tr * tc;
        for (int64_t ti = (int64_t)blockIdx.x * nwarps + warp; ti < ntile;
             ti += (int64_t)gridDim.x * nwarps) {
            const int64_t c = ti / (tr * tc), rem = ti - c * (tr * tc);
            const int64_t r0 = (rem / tc) * 32, c0 = (rem % tc) * 32;
            const float* S = src + c * R * W;
            float* Dd = dst + c * R * W;
            float v[32];
#pragma unroll
            for (int y = 0; y < 32; ++y) {
                const int64_t r = r0 + y, cc = c0 + lane;
                v[y] = (r < rows && cc < cols) ? __ldcg(S + r * cols + cc) : 0.0f;
            }
            __syncwarp();
#pragma unroll
            for (int y = 0; y < 32; ++y) tile[y * 33 + lane] = v[y];
            __syncwarp();
#pragma unroll
            for (int y = 0; y < 32; ++y) {
                const int64_t cc = c0 + y, r = r0 + lane;
                if (cc < cols && r < rows) Dd[cc * rows + r] = tile[lane * 33 + y];
            }
        }
    }
    __syncthreads();
}

// The image in the W passes' layout, once per call (all SMs, before the
// persistent launch).
__global__ void __launch_bounds__(256) transpose_image3d_kernel(const float* image, float* imageT,
                                                                int64_t count, int64_t R,
                                                                int64_t W) {
    __shared__ float smem[8 * 32 * 33];
    transpose_rw(image, imageT, count, R, W, false, smem, 8);
}

template <int MODE, int CI, bool CODES = false>
__device__ __forceinline__ bool run_tile3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h,
                                          float* stage, unsigned int cb, bool checked) {
    if ((int)(threadIdx.x >> 5) >= kCW) return producer3<CI>(a, t, h, stage, cb);
    if (MODE == kModeAbs && checked)
        return compute3<MODE, CI, true, CODES>(a, t, t_app, h, stage, cb);
    return compute3<MODE, CI, false, CODES>(a, t, t_app, h, stage, cb);
}

template <int MODE, int CI, bool CODES>
__global__ void __launch_bounds__(kBlock3, 1) vol3d_kernel(const Vol3DArgs a) {
    extern __shared__ __align__(16) unsigned char smem3[];
    Head3& h = *reinterpret_cast<Head3*>(smem3);
    float* stage = reinterpret_cast<float*>(smem3 + sizeof(Head3));
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNst; ++i) {
            mbar_init3(&h.full[i], kPW * 32);  // one asynchronous arrival per producer lane
            mbar_init3(&h.empty[i], 1);
        }
    }
    __syncthreads();
    const bool checked = MODE == kModeAbs && *a.range_flag != 0;
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[0] = (unsigned long long)gtimer();
    unsigned int epoch = 1;
    unsigned int cb = 0;  // staging chunks handed over so far in this block
    const int napps = a.iterations * kMaxPasses;
    bool alive = true;
    const bool tw = a.distT != nullptr;
    const int64_t R = a.D * a.H;

    for (int t_app = 0; t_app < napps && alive; ++t_app) {
        const int pass = t_app % kMaxPasses;
        const PassGeom& g = a.pass[pass];
        const bool on_t = tw && pass >= 4;  // this pass runs on the transposed copies
        if (tw && pass == 4) {
            transpose_rw(a.dist, a.distT, a.B, R, a.W, false, stage, kTransposeWarps);
            if (!(alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns))) break;
        }
        const int ntiles = a.ntp[pass] * a.ntq[pass];
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        const int L = (int)g.L;
        const int nch = L > 1 ? (L + kChunk - 1) / kChunk : 0;
        for (int64_t wv = 0; wv < nwaves; ++wv) {
            if ((int)blockIdx.x >= per_wave * ntiles) continue;
            const int64_t b = wv * per_wave + blockIdx.x / ntiles;
            if (b >= a.B) continue;
            Tile3 t;
            t.g = &g;
            t.tile = blockIdx.x % ntiles;
            t.jp = t.tile / a.ntq[pass];
            t.jq = t.tile % a.ntq[pass];
            t.ntq = a.ntq[pass];
            t.b = b;
            t.dist = (on_t ? a.distT : a.dist) + b * a.N;
            t.img = (on_t ? a.imageT : a.image) + b * a.C * a.N;
            t.csl = on_t ? 1 : g.sl;
            t.csp = on_t ? a.H * a.W : g.sp;
            t.csq = on_t ? a.W : g.sq;
            t.L = L;
            t.nch = nch;
            t.p0 = (int64_t)t.jp * kTP - kRing;
            t.q0 = (int64_t)t.jq * kTQ - kRing;
            if (nch > 0) run_tile3<MODE, CI, CODES>(a, t, t_app, h, stage, cb, checked);
            cb += (unsigned int)nch;
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        if (alive && tw && pass == 5) {
            transpose_rw(a.distT, a.dist, a.B, R, a.W, true, stage, kTransposeWarps);
            alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 1 < 16)
            timeline[t_app + 1] = (unsigned long long)gtimer();
    }
}

// Batched launch: work list of (instance, tile) items per round, one round
// per pass application, grid barrier between rounds; every instance has its
// own arguments (cost mode, planes, exchange words, range flag).
struct Vol3DBatch {
    const Vol3DArgs* desc;
    int rounds;
    const int* round_waves;   // [rounds + 1]
    const int* wave_items;    // [waves][gridDim.x]: (instance << 16) | tile, or -1
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
};

// D0 = v * M and the intensity range test of instance blockIdx.y.
__global__ void __launch_bounds__(256) init3d_batched_kernel(const Vol3DArgs* desc) {
    const Vol3DArgs& a = desc[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += stride)
        a.dist[i] = __fmul_rn(a.v, a.mask[i]);
    if (a.mode != kModeAbs) return;
    int* flag = const_cast<int*>(a.range_flag);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.C * a.N; i += stride) {
        const float x = fabsf(a.image[i]);
        const bool ok = x == 0.0f || (x >= 0x1p-40f && x <= 0x1p62f);
        if (!ok && *(volatile int*)flag == 0) atomicOr(flag, 1);
    }
}

__device__ bool run_item3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h, float* stage,
                          unsigned int cb) {
    if (a.mode == kModeConst) return run_tile3<kModeConst, 0>(a, t, t_app, h, stage, cb, false);
    if (a.mode == kModeAbs)
        return run_tile3<kModeAbs, 1>(a, t, t_app, h, stage, cb, *a.range_flag != 0);
    if (a.C == 1) return run_tile3<kModeGeneral, 1>(a, t, t_app, h, stage, cb, false);
    if (a.C == 2) return run_tile3<kModeGeneral, 2>(a, t, t_app, h, stage, cb, false);
    return run_tile3<kModeGeneral, 3>(a, t, t_app, h, stage, cb, false);
}

__global__ void __launch_bounds__(kBlock3, 1) vol3d_batched_kernel(const Vol3DBatch bt) {
    extern __shared__ __align__(16) unsigned char smem3[];
    Head3& h = *reinterpret_cast<Head3*>(smem3);
    float* stage = reinterpret_cast<float*>(smem3 + sizeof(Head3));
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNst; ++i) {
            mbar_init3(&h.full[i], kPW * 32);
            mbar_init3(&h.empty[i], 1);
        }
    }
    __syncthreads();
    unsigned int epoch = 1;
    unsigned int cb = 0;
    bool alive = true;
    for (int r = 0; r < bt.rounds && alive; ++r) {
        for (int wv = bt.round_waves[r]; wv < bt.round_waves[r + 1]; ++wv) {
            const int item = bt.wave_items[(int64_t)wv * gridDim.x + blockIdx.x];
            if (item < 0) continue;
            const Vol3DArgs& a = bt.desc[item >> 16];
            const int pass = r % kMaxPasses;
            const PassGeom& g = a.pass[pass];
            Tile3 t;
            t.g = &g;
            t.tile = item & 0xffff;
            t.jp = t.tile / a.ntq[pass];
            t.jq = t.tile % a.ntq[pass];
            t.ntq = a.ntq[pass];
            t.b = 0;
            t.dist = a.dist;
            t.img = a.image;
            t.csl = g.sl;
            t.csp = g.sp;
            t.csq = g.sq;
            t.L = (int)g.L;
            t.nch = t.L > 1 ? (t.L + kChunk - 1) / kChunk : 0;
            t.p0 = (int64_t)t.jp * kTP - kRing;
            t.q0 = (int64_t)t.jq * kTQ - kRing;
            if (t.nch > 0) run_item3(a, t, r, h, stage, cb);
            cb += (unsigned int)t.nch;
        }
        alive = grid_barrier(bt.barrier, epoch++, bt.status, bt.timeout_ns);
    }
}

size_t stage_bytes(int CI) {
    return sizeof(Head3) + (size_t)kNst * kChunk * (1 + CI) * kPlane * sizeof(float);
}

using Vol3DKernel = void (*)(Vol3DArgs);

template <bool CODES>
Vol3DKernel pick_kernel_t(int mode, int CI) {
    if (mode == kModeConst) return vol3d_kernel<kModeConst, 0, CODES>;
    if (mode == kModeAbs) return vol3d_kernel<kModeAbs, 1, CODES>;
    if (CI == 1) return vol3d_kernel<kModeGeneral, 1, CODES>;
    if (CI == 2) return vol3d_kernel<kModeGeneral, 2, CODES>;
    return vol3d_kernel<kModeGeneral, 3, CODES>;
}
Vol3DKernel pick_kernel(int mode, int CI, bool codes = false) {
    return codes ? pick_kernel_t<true>(mode, CI) : pick_kernel_t<false>(mode, CI);
}

struct Vol3DPlan {
    int mode = 0, CI = 0, grid = 0, max_tiles = 0;
    int ntp[kMaxPasses] = {}, ntq[kMaxPasses] = {};
    size_t smem = 0, ws_bytes = 0;
    size_t zero_bytes = 0;             // header and exchange words (cleared per call)
    size_t distT_off = 0, imageT_off = 0;  // transposed copies for the W passes
};

// Whether the 3D call fits this kernel (at most kMaxCI channels in the
// general cost, every tile of a pass co-resident, no tile-shape options),
// and its launch geometry.
bool plan_vol3d(const SweepArgs& f, const fgx_options* opt, int sms, Vol3DPlan* vp,
                bool any_mode = false) {
    if (f.ndim != 3) return false;
    if (opt && (opt->tile_lines || opt->tile_width || opt->tile_height)) return false;
    vp->mode = f.cost_mode == kCostConst ? kModeConst
               : f.cost_mode == kCostAbs ? kModeAbs : kModeGeneral;
    vp->CI = vp->mode == kModeConst ? 0 : (int)f.C;
    // a workspace-size query covers every cost mode: plan the cheapest one
    if (any_mode) {
        vp->mode = kModeConst;
        vp->CI = 0;
    }
    if (vp->CI > kMaxCI) return false;
    int max_tiles = 1;
    for (int i = 0; i < kMaxPasses; ++i) {
        const PassGeom& g = f.pass[i];
        vp->ntp[i] = (int)std::max<int64_t>(1, (g.P + kTP - 1) / kTP);
        vp->ntq[i] = (int)std::max<int64_t>(1, (g.Q + kTQ - 1) / kTQ);
        if ((int64_t)vp->ntp[i] * vp->ntq[i] > (1 << 20)) return false;
        max_tiles = std::max(max_tiles, vp->ntp[i] * vp->ntq[i]);
    }
    vp->max_tiles = max_tiles;
    vp->smem = stage_bytes(vp->CI);
    Vol3DKernel k = pick_kernel(vp->mode, vp->CI);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vp->smem) !=
        cudaSuccess)
        return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock3, vp->smem) !=
            cudaSuccess ||
        per_sm < 1)
        return false;
    int64_t grid = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, f.B * max_tiles));
    if (grid < max_tiles) return false;
    vp->grid = (int)grid;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    vp->zero_bytes = kHeaderBytes + (size_t)std::max<int64_t>(f.B, 1) * max_tiles * 2 * kXWords * 8;
    vp->distT_off = al(vp->zero_bytes);
    vp->imageT_off = vp->distT_off + al((size_t)f.B * f.N * 4);
    vp->ws_bytes = vp->imageT_off + al((size_t)f.B * f.C * f.N * 4);
    return true;
}

}  // namespace

bool vol3d_supports(const SweepArgs& f, const fgx_options* opt, int sms) {
    Vol3DPlan vp;
    return plan_vol3d(f, opt, sms, &vp);
}

size_t vol3d_workspace_bytes(const SweepArgs& f, const fgx_options* opt, int sms) {
    Vol3DPlan vp;
    return plan_vol3d(f, opt, sms, &vp, true) ? vp.ws_bytes : 0;
}

int run_vol3d(const SweepArgs& f, const float* image, const float* mask, float* dist,
              uint8_t* codes, float v, void* workspace, size_t ws_bytes, const fgx_options* opt,
              int sms, void* stream) {
    Vol3DPlan vp;
    if (!plan_vol3d(f, opt, sms, &vp)) return FGX_ERR_UNSUPPORTED;
    if (ws_bytes < vp.ws_bytes) return FGX_ERR_WORKSPACE;
    Vol3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = image;
    a.mask = mask;
    a.dist = dist;
    a.codes = codes;
    a.B = f.B;
    a.C = f.C;
    a.N = f.N;
    a.v = v;
    a.lambda = f.lambda;
    a.iterations = f.iterations;
    a.mode = vp.mode;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = vp.ntp[i];
        a.ntq[i] = vp.ntq[i];
    }
    a.max_tiles = vp.max_tiles;
    char* w = (char*)workspace;
    a.status = (int*)w;
    a.barrier = (unsigned int*)(w + 64);
    int* range_flag = (int*)(w + kRangeFlagOffset);
    a.range_flag = range_flag;
    a.xbuf = (unsigned long long*)(w + kHeaderBytes);
    a.timeout_ns = f.timeout_ns;
    a.D = f.pass[0].L;
    a.H = f.pass[2].L;
    a.W = f.pass[4].L;
    if (a.W > 1) {
        // the W passes run on [W][D][H] copies: their planes' rows are contiguous
        a.distT = (float*)(w + vp.distT_off);
        a.imageT = vp.mode == kModeConst ? nullptr : (float*)(w + vp.imageT_off);
        for (int i = 4; i < 6; ++i) {
            a.pass[i].sl = a.D * a.H;
            a.pass[i].sp = a.H;
            a.pass[i].sq = 1;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, vp.zero_bytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    // codes of the first plane of every sweep stay 0 (it keeps its values)
    const size_t ncodes = (size_t)f.iterations * kMaxPasses * (size_t)(f.B * f.N);
    if (codes && ncodes && cudaMemsetAsync(codes, 0, ncodes, s) != cudaSuccess)
        return FGX_ERR_CUDA;
    const int64_t n = f.B * f.N;
    const int ig = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 16);
    init3d_kernel<<<std::max(ig, 1), 256, 0, s>>>(mask, dist, v, n, image, f.B * f.C * f.N,
                                                 vp.mode == kModeAbs ? range_flag : nullptr);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if (a.imageT && f.iterations > 0) {
        transpose_image3d_kernel<<<sms * 8, 256, 0, s>>>(image, a.imageT, f.B * f.C,
                                                          a.D * a.H, a.W);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    if (f.iterations == 0) return FGX_OK;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)vp.grid);
    cfg.blockDim = dim3(kBlock3);
    cfg.dynamicSmemBytes = vp.smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Vol3DKernel k = pick_kernel(vp.mode, vp.CI, codes != nullptr);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vp.smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaLaunchKernelEx(&cfg, k, a) != cudaSuccess)
        return FGX_ERR_CUDA;
    return FGX_OK;
}

// ---------------------------------------------------- batched 3D instances ----

size_t vol3d_desc_size() { return sizeof(Vol3DArgs); }

bool vol3d_instance_desc(void* desc, const fgx_instance& it, const SweepArgs& f,
                         const fgx_options* opt, int sms, char* hdr, int* range_flag, char* xb,
                         size_t* xbytes, int* ci, int* max_tiles, int tiles[kMaxPasses]) {
    Vol3DPlan vp;
    if (!plan_vol3d(f, opt, sms, &vp)) return false;
    *xbytes = (size_t)vp.max_tiles * 2 * kXWords * 8;
    *ci = vp.CI;
    *max_tiles = vp.max_tiles;
    for (int i = 0; i < kMaxPasses; ++i) tiles[i] = vp.ntp[i] * vp.ntq[i];
    if (!desc) return true;
    Vol3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = it.image;
    a.mask = it.mask;
    a.dist = it.dist;
    a.B = 1;
    a.C = f.C;
    a.N = f.N;
    a.v = it.v;
    a.lambda = f.lambda;
    a.iterations = it.iterations;
    a.mode = vp.mode;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = vp.ntp[i];
        a.ntq[i] = vp.ntq[i];
    }
    a.max_tiles = vp.max_tiles;
    a.xbuf = (unsigned long long*)xb;
    a.barrier = (unsigned int*)(hdr + 64);
    a.status = (int*)hdr;
    a.range_flag = range_flag;
    a.timeout_ns = f.timeout_ns;
    std::memcpy(desc, &a, sizeof(a));
    return true;
}

int vol3d_batched_geometry(int sms, int max_ci, const fgx_options* opt, int* grid, size_t* smem) {
    *smem = stage_bytes(max_ci);
    if (cudaFuncSetAttribute(vol3d_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)*smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vol3d_batched_kernel, kBlock3,
                                                      *smem) != cudaSuccess ||
        per_sm < 1)
        return FGX_ERR_CUDA;
    int64_t g = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) g = std::min<int64_t>(g, opt->max_blocks);
    *grid = (int)std::max<int64_t>(1, g);
    return FGX_OK;
}

int launch_vol3d_batched(const void* desc, int n, int rounds, const int* round_waves,
                         const int* wave_items, int grid, size_t smem, char* hdr,
                         long long timeout_ns, int sms, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const Vol3DArgs* d = (const Vol3DArgs*)desc;
    init3d_batched_kernel<<<dim3((unsigned)std::max(1, sms * 4), (unsigned)n), 256, 0, s>>>(d);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if (rounds == 0) return FGX_OK;
    Vol3DBatch bt;
    bt.desc = d;
    bt.rounds = rounds;
    bt.round_waves = round_waves;
    bt.wave_items = wave_items;
    bt.barrier = (unsigned int*)(hdr + 64);
    bt.status = (int*)hdr;
    bt.timeout_ns = timeout_ns;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlock3);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, vol3d_batched_kernel, bt) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx

// ---------------------------------------------------------- 3D reverse sweep --
//
// The adjoint of the 3D raster scan on the same plane tiles.  For the pass
// applications in reverse order and the planes of each in reverse sweep
// order, the adjoint of voxel e is A[e] = G_in[e] + sum over the nine stencil
// offsets k (in order) of A[x_k] for the child x_k of the next plane of the
// forward sweep that chose e (code k+1); a child that did not contributes
// -0.0 (an exact identity).  The adjoint handed to the previous application
// is A[e] if e kept its value (code 0), else 0; after the first application
// dL/dM = v * that adjoint.  A needs the 3 x 3 children exactly as the
// forward needs the 3 x 3 parents, so the tiles, warps, boundary-row
// exchange and ring refresh are the forward's.  The adjoint lives in two
// buffers (a pass never writes the one it reads: sums are not idempotent);
// with the image gradient wanted, A of every application is stored and a
// separate kernel adds the gradient terms per voxel in the fixed order.

namespace fgx {
namespace {

struct Adj3DArgs {
    const float* grad_dist;   // [B][N]
    const uint8_t* codes;     // [T][B][N]
    float* grad_mask;         // [B][N] or null
    float* g0;                // [B][N] adjoint of D0, or null
    float* G[2];              // [B][N] adjoint buffers
    float* Astore;            // [T][B][N] adjoint of every application, or null
    int64_t B, N;
    float v;
    int T;
    PassGeom pass[kMaxPasses];
    int ntp[kMaxPasses], ntq[kMaxPasses];
    int max_tiles;
    unsigned long long* xbuf;
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
};

struct AdjHead3 {
    unsigned long long full[kNst], empty[kNst];
    float rowtop[2][kCW][kRQ];
    float rowbot[2][kCW][kRQ];
};
static_assert(sizeof(AdjHead3) % 16 == 0, "stage must stay 16-byte aligned");

// followed by [kNst][kChunk][kPlane] adjoint values and as many code bytes
size_t adj3_smem_bytes() {
    return sizeof(AdjHead3) + (size_t)kNst * kChunk * kPlane * (sizeof(float) + 1);
}

// Producer warps: the incoming adjoint and the codes of the application,
// plane after plane in reverse sweep order (0 outside the volume).  Plain
// loads of a whole chunk first, then the stores and one release arrival per
// thread.
__device__ bool adj_producer3(const Adj3DArgs& a, const Tile3& t, const float* gsrc,
                              const uint8_t* csrc, AdjHead3& h, float* stg, uint8_t* stc,
                              unsigned int cb) {
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31, pw = (threadIdx.x >> 5) - kCW;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    for (int c = 0; c < t.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = (int)(gc % kNst);
        if (gc >= (unsigned)kNst &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.empty[slot], ((gc / kNst) & 1u) ^ 1u,
                                                a.status, a.timeout_ns)))
            return false;
        float gv[kChunk][kRP / kPW];
        unsigned int cv[kChunk][kRP / kPW];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int s = c * kChunk + j;
            const int64_t line = g.dir > 0 ? (t.L - 1 - s) : s;
#pragma unroll
            for (int rr = 0; rr < kRP / kPW; ++rr) {
                const int64_t p = t.p0 + pw + kPW * rr;
                const bool in = s < t.L && qin && p >= 0 && p < g.P;
                const int64_t off = line * g.sl + p * g.sp + q * g.sq;
                gv[j][rr] = in ? __ldcg(gsrc + off) : 0.0f;
                cv[j][rr] = in ? (unsigned int)__ldg(csrc + off) : 0u;
            }
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j)
#pragma unroll
            for (int rr = 0; rr < kRP / kPW; ++rr) {
                const int r = pw + kPW * rr;
                stg[((size_t)slot * kChunk + j) * kPlane + r * kRQ + lane] = gv[j][rr];
                stc[((size_t)slot * kChunk + j) * kPlane + r * kRQ + lane] = (uint8_t)cv[j][rr];
            }
        mbar_arrive3(&h.full[slot]);  // every lane releases its own stores
    }
    return true;
}

// Compute warps: planes 0 .. L-1 of the reverse sweep.
__device__ bool adj_compute3(const Adj3DArgs& a, const Tile3& t, int t_app, AdjHead3& h,
                             const float* stg, const uint8_t* stc, unsigned int cb, float* gdst,
                             float* gmask, float* adst, float* g0) {
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const bool qown = lane >= kRing && lane < kRing + kTQ;
    bool own[kRows];
    int64_t goff[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = w * kRows + i;
        const int64_t p = t.p0 + r;
        own[i] = qin && p >= 0 && p < g.P && qown && r >= kRing && r < kRing + kTP;
        goff[i] = p * g.sp + q * g.sq;
    }
    const int cl = max(lane - 1, 0), cr = min(lane + 1, kRQ - 1);
    const int rows0 = w * kRows;
    const float nz = __int_as_float(0x80000000);
    bool failed = false;
    float ap[kRows];  // adjoint of the previous plane of the reverse sweep
#pragma unroll
    for (int i = 0; i < kRows; ++i) ap[i] = nz;
    const unsigned int tag_base = ((unsigned int)(t_app + 1)) << 16;
    int xi = 0;
    for (int s = 0; s < t.L; ++s) {
        const unsigned int gc = cb + s / kChunk;
        const int j = s % kChunk;
        const int slot = (int)(gc % kNst);
        if (j == 0 && !failed &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.full[slot], (gc / kNst) & 1u, a.status,
                                                a.timeout_ns)))
            failed = true;
        const int rb = s & 1;
        h.rowtop[rb][w][lane] = ap[0];
        h.rowbot[rb][w][lane] = ap[kRows - 1];
        asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory");
        if (threadIdx.x == 0 && s >= 2 && (s - 2) % kChunk == kChunk - 1)
            mbar_arrive3(&h.empty[(cb + (s - 2) / kChunk) % kNst]);
        // children: adjoints of the previous plane (3 x 3 around each voxel)
        float col[kRows + 2], lft[kRows + 2], rgt[kRows + 2];
        col[0] = w > 0 ? h.rowbot[rb][w - 1][lane] : nz;
#pragma unroll
        for (int i = 0; i < kRows; ++i) col[i + 1] = ap[i];
        col[kRows + 1] = w < kCW - 1 ? h.rowtop[rb][w + 1][lane] : nz;
#pragma unroll
        for (int k = 0; k < kRows + 2; ++k) {
            lft[k] = __shfl_up_sync(0xffffffffu, col[k], 1);
            rgt[k] = __shfl_down_sync(0xffffffffu, col[k], 1);
            if (lane == 0) lft[k] = nz;
            if (lane == 31) rgt[k] = nz;
        }
        // their codes (plane s-1 of this application; none before the first)
        unsigned int cc[kRows + 2][3];
        if (s > 0) {
            const unsigned int gcp = cb + (s - 1) / kChunk;
            const uint8_t* Pc = stc + ((size_t)(gcp % kNst) * kChunk + (s - 1) % kChunk) * kPlane;
#pragma unroll
            for (int k = 0; k < kRows + 2; ++k) {
                const int rr = min(max(rows0 + k - 1, 0), kRP - 1);
                cc[k][0] = Pc[rr * kRQ + cl];
                cc[k][1] = Pc[rr * kRQ + lane];
                cc[k][2] = Pc[rr * kRQ + cr];
            }
        } else {
#pragma unroll
            for (int k = 0; k < kRows + 2; ++k) cc[k][0] = cc[k][1] = cc[k][2] = 0u;
        }
        const float* Sg = stg + ((size_t)slot * kChunk + j) * kPlane;
        const uint8_t* Sc = stc + ((size_t)slot * kChunk + j) * kPlane;
        const int64_t lo = (int64_t)(g.dir > 0 ? (t.L - 1 - s) : s) * g.sl;
        float na[kRows];
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            float acc = Sg[(rows0 + i) * kRQ + lane];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                // child of offset k = (dp, dq) sits at (row - dp, column - dq)
                const int dp = k / 3 - 1, dq = k % 3 - 1;
                const int rk = i + 1 - dp;
                const float ax = dq > 0 ? lft[rk] : (dq == 0 ? col[rk] : rgt[rk]);
                const unsigned int cx = cc[rk][1 - dq];
                acc = __fadd_rn(acc, cx == (unsigned int)(k + 1) ? ax : nz);
            }
            na[i] = acc;
            if (own[i]) {
                const float gout = Sc[(rows0 + i) * kRQ + lane] != 0 ? 0.0f : acc;
                if (gmask) gmask[lo + goff[i]] = __fmul_rn(a.v, gout);
                if (g0) g0[lo + goff[i]] = gout;
                if (gdst) gdst[lo + goff[i]] = gout;
                if (adst) adst[lo + goff[i]] = acc;
            }
        }
#pragma unroll
        for (int i = 0; i < kRows; ++i) ap[i] = na[i];
        if (s >= kRing && s % kRing == 0 && s + 1 < t.L) {
            if (!failed && !exchange3(XLink3{a.xbuf, a.max_tiles, a.status, a.timeout_ns}, t, w,
                                      tag_base | (unsigned int)(xi + 1), xi & 1, ap))
                failed = true;
            ++xi;
        }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory");
    if (threadIdx.x == 0) {
        for (int c = max(0, t.nch - 2); c < t.nch; ++c) {
            const int last = min(c * kChunk + kChunk - 1, t.L - 1);
            if (last >= t.L - 2) mbar_arrive3(&h.empty[(cb + c) % kNst]);
        }
    }
    return !failed;
}

template <bool STORE_A>
__global__ void __launch_bounds__(kBlock3, 1) adj3d_kernel(const Adj3DArgs a) {
    extern __shared__ __align__(16) unsigned char smem3[];
    AdjHead3& h = *reinterpret_cast<AdjHead3*>(smem3);
    float* stg = reinterpret_cast<float*>(smem3 + sizeof(AdjHead3));
    uint8_t* stc = reinterpret_cast<uint8_t*>(stg + (size_t)kNst * kChunk * kPlane);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNst; ++i) {
            mbar_init3(&h.full[i], kPW * 32);  // one arrival per producer thread
            mbar_init3(&h.empty[i], 1);
        }
    }
    __syncthreads();
    unsigned int epoch = 1;
    unsigned int cb = 0;
    int in_idx = -1;  // the first application reads the caller's dL/dD
    bool alive = true;
    for (int t_app = a.T - 1; t_app >= 0 && alive; --t_app) {
        const int pass = t_app % kMaxPasses;
        const PassGeom& g = a.pass[pass];
        const int ntiles = a.ntp[pass] * a.ntq[pass];
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        const int L = (int)g.L;
        const int nch = (L + kChunk - 1) / kChunk;
        const int out_idx = in_idx == 0 ? 1 : 0;
        for (int64_t wv = 0; wv < nwaves; ++wv) {
            if ((int)blockIdx.x >= per_wave * ntiles) continue;
            const int64_t b = wv * per_wave + blockIdx.x / ntiles;
            if (b >= a.B) continue;
            Tile3 t;
            t.g = &g;
            t.tile = blockIdx.x % ntiles;
            t.jp = t.tile / a.ntq[pass];
            t.jq = t.tile % a.ntq[pass];
            t.ntq = a.ntq[pass];
            t.b = b;
            t.L = L;
            t.nch = nch;
            t.p0 = (int64_t)t.jp * kTP - kRing;
            t.q0 = (int64_t)t.jq * kTQ - kRing;
            const float* gsrc = (in_idx < 0 ? a.grad_dist : a.G[in_idx]) + b * a.N;
            if ((int)(threadIdx.x >> 5) >= kCW) {
                adj_producer3(a, t, gsrc, a.codes + ((int64_t)t_app * a.B + b) * a.N, h, stg,
                              stc, cb);
            } else {
                float* gdst = t_app > 0 ? a.G[out_idx] + b * a.N : nullptr;
                float* gmask = (t_app == 0 && a.grad_mask) ? a.grad_mask + b * a.N : nullptr;
                float* adst = STORE_A ? a.Astore + ((int64_t)t_app * a.B + b) * a.N : nullptr;
                float* g0 = (t_app == 0 && a.g0) ? a.g0 + b * a.N : nullptr;
                adj_compute3(a, t, a.T - 1 - t_app, h, stg, stc, cb, gdst, gmask, adst, g0);
            }
            cb += (unsigned int)nch;
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        in_idx = out_idx;
    }
}

struct Grad3DArgs {
    const float* image;       // [B][C][N]
    const uint8_t* codes;     // [T][B][N]
    const float* Astore;      // [T][B][N]
    float* grad_image;        // [B][C][N], or null
    float* lambda_terms;      // [B][N] per-voxel terms of dL/dlambda, or null
    int64_t B, C, N;
    int64_t D, H, W;
    float lambda;
    int T;
    PassGeom pass[kMaxPasses];
    float s2[kMaxPasses][9];  // |offset|^2 of every pass and stencil offset
};

__device__ __forceinline__ float grad_cost3(const float* img, int64_t x, int64_t y, int C,
                                            int64_t n, float t, float lam,
                                            float* di2_out = nullptr) {
    float di2 = 0.0f;
    for (int ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(img[ch * n + x], img[ch * n + y]);
        di2 = __fadd_rn(di2, __fmul_rn(d, d));
    }
    if (di2_out) *di2_out = di2;
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// Image gradient of the 3D reverse sweep, one thread per voxel, pass
// applications in reverse order: per application the terms of the children
// that chose the voxel (offset order), then the term of its own parent.
// The gradient accumulates in the output array (each voxel is touched by its
// own thread only).  With lambda_terms, each voxel also sums, over the
// applications in the same order, its adjoint times d c / d lambda of its own
// parent edge, (di2 - s2) / (c + c).
template <int CC, bool IMG, typename Idx>
__global__ void __launch_bounds__(256) grad3d_kernel(const Grad3DArgs a) {
    // CC > 0: the CC channel sums stay in registers (written once at the end);
    // CC == 0: any channel count, accumulated in the output array.  Idx: the
    // index type within one instance (32-bit when every offset fits)
    const float lam = a.lambda;
    const int C = CC > 0 ? CC : (int)a.C;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.B * a.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / a.N;
        const Idx e = (Idx)(i - b * a.N);
        const Idx HW = (Idx)(a.H * a.W), Wd = (Idx)a.W;
        const Idx dd = e / HW, rem = e - dd * HW;
        const Idx hh = rem / Wd, ww = rem - hh * Wd;
        const float* img = a.image + b * a.C * a.N;
        float* gout = IMG ? a.grad_image + b * a.C * a.N + e : nullptr;
        float lt = 0.0f;
        float gi[CC > 0 ? CC : 1];
#pragma unroll
        for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gi[ch] = 0.0f;
        if (IMG && CC == 0)
            for (int ch = 0; ch < C; ++ch) gout[ch * a.N] = 0.0f;
        // g -= wgt (I(x) - I(y))  or  g += wgt (I(x) - I(y)), per channel
        auto add_term = [&](float wgt, Idx x, Idx y, bool minus) {
            if (CC > 0) {
#pragma unroll
                for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) {
                    const float term =
                        __fmul_rn(wgt, __fsub_rn(img[ch * a.N + x], img[ch * a.N + y]));
                    gi[ch] = minus ? __fsub_rn(gi[ch], term) : __fadd_rn(gi[ch], term);
                }
            } else {
                for (int ch = 0; ch < C; ++ch) {
                    const float term =
                        __fmul_rn(wgt, __fsub_rn(img[ch * a.N + x], img[ch * a.N + y]));
                    gout[ch * a.N] = minus ? __fsub_rn(gout[ch * a.N], term)
                                           : __fadd_rn(gout[ch * a.N], term);
                }
            }
        };
        for (int t = a.T - 1; t >= 0; --t) {
            const PassGeom& g = a.pass[t % kMaxPasses];
            const Idx line = g.axis == 0 ? dd : (g.axis == 1 ? hh : ww);
            const Idx p = g.axis == 0 ? hh : dd;
            const Idx q = g.axis == 2 ? hh : ww;
            const Idx L = (Idx)g.L, P = (Idx)g.P, Q = (Idx)g.Q;
            const Idx sl = (Idx)g.sl, sp = (Idx)g.sp, sq = (Idx)g.sq;
            const float* A = a.Astore + ((int64_t)t * a.B + b) * a.N;
            const uint8_t* cd = a.codes + ((int64_t)t * a.B + b) * a.N;
            // children on the next plane of the forward sweep, offset order
            const Idx cl = line + g.dir;
            if (IMG && cl >= 0 && cl < L) {
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const Idx cp = p - (k / 3 - 1), cq = q - (k % 3 - 1);
                    if (cp < 0 || cp >= P || cq < 0 || cq >= Q) continue;
                    const Idx x = cl * sl + cp * sp + cq * sq;
                    if (cd[x] != k + 1) continue;
                    const float c = grad_cost3(img, x, e, C, a.N, g.t[k], lam);
                    if (c > 0.0f) add_term(__fdiv_rn(__fmul_rn(A[x], lam), c), x, e, true);
                }
            }
            // own parent on the previous plane of the forward sweep
            const int code = cd[e];
            const Idx pl = line - g.dir;
            if (code >= 1 && code <= 9 && pl >= 0 && pl < L) {
                const int k = code - 1;
                const Idx pp = p + (k / 3 - 1), pq = q + (k % 3 - 1);
                if (pp >= 0 && pp < P && pq >= 0 && pq < Q) {
                    const Idx y = pl * sl + pp * sp + pq * sq;
                    float di2;
                    const float c = grad_cost3(img, e, y, C, a.N, g.t[k], lam, &di2);
                    if (c > 0.0f) {
                        if (a.lambda_terms) {
                            const float s2 = a.s2[t % kMaxPasses][k];
                            lt = __fadd_rn(lt, __fmul_rn(A[e], __fdiv_rn(__fsub_rn(di2, s2),
                                                                         __fadd_rn(c, c))));
                        }
                        if (IMG) add_term(__fdiv_rn(__fmul_rn(A[e], lam), c), e, y, false);
                    }
                }
            }
        }
        if (IMG && CC > 0) {
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gout[ch * a.N] = gi[ch];
        }
        if (a.lambda_terms) a.lambda_terms[i] = lt;
    }
}

struct Adj3DPlan {
    int grid = 0, max_tiles = 0;
    int ntp[kMaxPasses] = {}, ntq[kMaxPasses] = {};
    size_t xbuf_off = 0, g_off[2] = {}, a_off = 0, total = 0;
};

bool plan_adj3d(const SweepArgs& f, int iterations, const fgx_options* opt, int sms,
                Adj3DPlan* p) {
    if (f.ndim != 3 || iterations <= 0) return false;
    if (opt && (opt->tile_lines || opt->tile_width || opt->tile_height)) return false;
    int max_tiles = 1;
    for (int i = 0; i < kMaxPasses; ++i) {
        const PassGeom& g = f.pass[i];
        p->ntp[i] = (int)std::max<int64_t>(1, (g.P + kTP - 1) / kTP);
        p->ntq[i] = (int)std::max<int64_t>(1, (g.Q + kTQ - 1) / kTQ);
        if ((int64_t)p->ntp[i] * p->ntq[i] > (1 << 20)) return false;
        max_tiles = std::max(max_tiles, p->ntp[i] * p->ntq[i]);
    }
    p->max_tiles = max_tiles;
    const size_t smem = adj3_smem_bytes();
    if (cudaFuncSetAttribute(adj3d_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(adj3d_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj3d_kernel<true>, kBlock3,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
        return false;
    int64_t grid = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    grid = std::min<int64_t>(grid, std::max<int64_t>(1, f.B * max_tiles));
    if (grid < max_tiles) return false;
    p->grid = (int)grid;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = kHeaderBytes;
    p->xbuf_off = off;
    off += al((size_t)std::max<int64_t>(f.B, 1) * max_tiles * 2 * kXWords * 8);
    for (int i = 0; i < 2; ++i) {
        p->g_off[i] = off;
        off += al((size_t)f.B * f.N * 4);
    }
    p->a_off = off;
    off += al((size_t)iterations * kMaxPasses * f.B * f.N * 4);
    p->total = off;
    return true;
}

}  // namespace

size_t adj3d_workspace_bytes(const SweepArgs& f, int iterations, const fgx_options* opt,
                             int sms) {
    Adj3DPlan p;
    return plan_adj3d(f, iterations, opt, sms, &p) ? p.total : 0;
}

int run_adj3d(const SweepArgs& f, const float* grad_dist, const float* image,
              const uint8_t* codes, float* grad_image, float* grad_mask, float v, int iterations,
              void* workspace, size_t ws_bytes, const fgx_options* opt, int sms, void* stream,
              float* g0, float* lambda_terms, const float* s2) {
    if (lambda_terms && !s2) return FGX_ERR_ARG;
    Adj3DPlan p;
    if (!plan_adj3d(f, iterations, opt, sms, &p)) return FGX_ERR_UNSUPPORTED;
    if (ws_bytes < p.total) return FGX_ERR_WORKSPACE;
    char* w = (char*)workspace;
    Adj3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.grad_dist = grad_dist;
    a.codes = codes;
    a.grad_mask = grad_mask;
    a.g0 = g0;
    a.G[0] = (float*)(w + p.g_off[0]);
    a.G[1] = (float*)(w + p.g_off[1]);
    const bool need_a = grad_image || lambda_terms;  // the per-voxel pass needs every A
    a.Astore = need_a ? (float*)(w + p.a_off) : nullptr;
    a.B = f.B;
    a.N = f.N;
    a.v = v;
    a.T = iterations * kMaxPasses;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = p.ntp[i];
        a.ntq[i] = p.ntq[i];
    }
    a.max_tiles = p.max_tiles;
    a.xbuf = (unsigned long long*)(w + p.xbuf_off);
    a.barrier = (unsigned int*)(w + 64);
    a.status = (int*)w;
    a.timeout_ns = f.timeout_ns;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, p.g_off[0], s) != cudaSuccess) return FGX_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)p.grid);
    cfg.blockDim = dim3(kBlock3);
    cfg.dynamicSmemBytes = adj3_smem_bytes();
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, need_a ? adj3d_kernel<true> : adj3d_kernel<false>, a) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    if (need_a) {
        Grad3DArgs g;
        std::memset(&g, 0, sizeof(g));
        g.image = image;
        g.codes = codes;
        g.Astore = a.Astore;
        g.grad_image = grad_image;
        g.lambda_terms = lambda_terms;
        if (s2)
            for (int i = 0; i < kMaxPasses; ++i)
                for (int k = 0; k < 9; ++k) g.s2[i][k] = s2[i * 9 + k];
        g.B = f.B;
        g.C = f.C;
        g.N = f.N;
        g.D = f.pass[0].L;        // extent of the axis of the first pass pair (D)
        g.H = f.pass[2].L;
        g.W = f.pass[4].L;
        g.lambda = f.lambda;
        g.T = a.T;
        for (int i = 0; i < kMaxPasses; ++i) g.pass[i] = f.pass[i];
        const int64_t n = f.B * f.N;
        const int gg = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
        const int gb = std::max(gg, 1);
        // 32-bit offsets within an instance when every one fits (C * N < 2^31)
        if (f.C * f.N < ((int64_t)1 << 31)) {
            if (!grad_image) grad3d_kernel<0, false, int><<<gb, 256, 0, s>>>(g);
            else if (f.C == 1) grad3d_kernel<1, true, int><<<gb, 256, 0, s>>>(g);
            else if (f.C == 2) grad3d_kernel<2, true, int><<<gb, 256, 0, s>>>(g);
            else if (f.C == 3) grad3d_kernel<3, true, int><<<gb, 256, 0, s>>>(g);
            else grad3d_kernel<0, true, int><<<gb, 256, 0, s>>>(g);
        } else {
            if (!grad_image) grad3d_kernel<0, false, int64_t><<<gb, 256, 0, s>>>(g);
            else grad3d_kernel<0, true, int64_t><<<gb, 256, 0, s>>>(g);
        }
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

}  // namespace fgx
