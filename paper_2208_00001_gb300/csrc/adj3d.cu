// 3D reverse sweep on register-blocked plane tiles (the adjoint of the
// Implementation section's six passes per iteration; tiles, warp roles and
// ring exchange as in the forward plane-tile kernel).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_sync.cuh"
#include "fgx_internal.h"

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

using namespace dev;

constexpr int kRows = 4;                  // region rows per compute thread
constexpr int kCW = 8;                    // compute warps
constexpr int kPW = 4;                    // producer warps
constexpr int kRP = kRows * kCW;          // region rows
constexpr int kRQ = 32;                   // region columns (one per lane)
constexpr int kRing = 4;                  // narrow ring width = steps between refreshes
constexpr int kRingWide = 8;              // wide ring width (fewer refreshes, more tiles)
constexpr int kTP = kRP - 2 * kRing;      // owned rows of a narrow-ring tile (the most)
constexpr int kTQ = kRQ - 2 * kRing;      // owned columns of a narrow-ring tile
constexpr int kPlane = kRP * kRQ;         // region voxels
constexpr int kChunk = kRing;             // planes per staging chunk
constexpr int kNst = 3;                   // chunks in the staging ring
constexpr int kBlock3 = (kCW + kPW) * 32;
constexpr int kXWords = kTP * kTQ;        // published words per tile and parity
#define kInf3 __int_as_float(0x7f800000)

__device__ __forceinline__ unsigned int saddr3(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}
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
    int K, tp, tq;     // ring width and owned extents (tp = tq = 32 - 2K)
    int64_t b;
    int L, nch;
    int64_t p0, q0;  // plane coordinates of region row 0 and column 0
};

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
    const int K = t.K, tp = t.tp, tq = t.tq;
    const bool qown = lane >= K && lane < K + tq;
    const int64_t q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const unsigned long long* src[kRows];
    bool need[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = w * kRows + i;
        const bool pown = r >= K && r < K + tp;
        const unsigned long long word =
            ((unsigned long long)tg << 32) | (unsigned int)__float_as_uint(d[i]);
        if (pown && qown) st_relaxed_u64(mine + (r - K) * tq + (lane - K), word);
        const int64_t p = t.p0 + r;
        need[i] = !(pown && qown) && qin && p >= 0 && p < g.P;
        src[i] = nullptr;
        if (need[i]) {
            const int op = (int)(p / tp), oq = (int)(q / tq);
            const int lr = (int)(p - (int64_t)op * tp), lq = (int)(q - (int64_t)oq * tq);
            src[i] = base + ((size_t)(op * t.ntq + oq) * 2 + par) * kXWords + lr * tq + lq;
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

struct Adj3DArgs {
    const float* grad_dist;   // [B][N]
    const uint8_t* codes;     // [t_hi - t_lo][B][N]: codes of applications t_lo .. t_hi-1
    float* grad_mask;         // [B][N] or null
    float* g0;                // [B][N] adjoint of D0, or null
    float* G[2];              // [B][N] adjoint buffers
    float* A;                 // [B][N] adjoint of the current application (gradient terms), or null
    int64_t B, N;
    float v;
    int T;                    // pass applications of the whole transform
    int t_lo, t_hi;           // applications of this launch
    int in_first;             // adjoint of application t_hi-1: -1 = grad_dist, else G[in_first]
    PassGeom pass[kMaxPasses];
    int ntp[kMaxPasses], ntq[kMaxPasses];
    int ring[kMaxPasses];     // ring width K of each pass (4 or 8)
    int max_tiles;
    unsigned long long* xbuf;
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
    // image-gradient and lambda terms, added per application
    const float* image;       // [B][C][N]
    float* grad_image;        // [B][C][N] accumulator (cleared by the host), or null
    float* lambda_terms;      // [B][N] accumulator (cleared by the host), or null
    int64_t C, D, H, W;
    float lambda;
    float s2[kMaxPasses][9];  // |offset|^2 of every pass and stencil offset
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
    // lines contiguous in memory (the W passes) with every chunk whole and
    // aligned: a chunk's planes come as one 16-byte load of adjoints and one
    // 4-byte load of codes per voxel instead of four of each, strided
    static_assert(kChunk == 4, "vector loads of four planes");
    const bool vec = g.sl == 1 && (t.L % kChunk) == 0 && (g.sp % kChunk) == 0 &&
                     (g.sq % kChunk) == 0 && ((uintptr_t)gsrc & 15u) == 0 &&
                     ((uintptr_t)csrc & 3u) == 0;
    for (int c = 0; c < t.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = (int)(gc % kNst);
        if (gc >= (unsigned)kNst &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.empty[slot], ((gc / kNst) & 1u) ^ 1u,
                                                a.status, a.timeout_ns)))
            return false;
        float gv[kChunk][kRP / kPW];
        unsigned int cv[kChunk][kRP / kPW];
        if (vec) {
            // the chunk's four planes are four consecutive elements of memory
            const int64_t lo = g.dir > 0 ? (int64_t)(t.L - kChunk - c * kChunk) : c * kChunk;
#pragma unroll
            for (int rr = 0; rr < kRP / kPW; ++rr) {
                const int64_t p = t.p0 + pw + kPW * rr;
                const bool in = qin && p >= 0 && p < g.P;
                const int64_t off = lo + p * g.sp + q * g.sq;
                const float4 v = in ? __ldcg(reinterpret_cast<const float4*>(gsrc + off))
                                    : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                const unsigned int cw =
                    in ? __ldg(reinterpret_cast<const unsigned int*>(csrc + off)) : 0u;
                const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int j = 0; j < kChunk; ++j) {
                    const int k = g.dir > 0 ? kChunk - 1 - j : j;
                    gv[j][rr] = f[k];
                    cv[j][rr] = (cw >> (8 * k)) & 0xffu;
                }
            }
        } else {
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
    const int K = t.K, tp = t.tp, tq = t.tq;
    const bool qown = lane >= K && lane < K + tq;
    bool own[kRows];
    int64_t goff[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = w * kRows + i;
        const int64_t p = t.p0 + r;
        own[i] = qin && p >= 0 && p < g.P && qown && r >= K && r < K + tp;
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
        compute_sync();
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
        if (s >= K && s % K == 0 && s + 1 < t.L) {
            if (!failed && !exchange3(XLink3{a.xbuf, a.max_tiles, a.status, a.timeout_ns}, t, w,
                                      tag_base | (unsigned int)(xi + 1), xi & 1, ap))
                failed = true;
            ++xi;
        }
    }
    compute_sync();
    if (threadIdx.x == 0) {
        for (int c = max(0, t.nch - 2); c < t.nch; ++c) {
            const int last = min(c * kChunk + kChunk - 1, t.L - 1);
            if (last >= t.L - 2) mbar_arrive3(&h.empty[(cb + c) % kNst]);
        }
    }
    return !failed;
}

__device__ __forceinline__ float grad_cost3(const float* img, int x, int y, int C, int n,
                                            float t, float lam, float* di2_out = nullptr) {
    float di2 = 0.0f;
    for (int ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(img[ch * n + x], img[ch * n + y]);
        di2 = __fadd_rn(di2, __fmul_rn(d, d));
    }
    if (di2_out) *di2_out = di2;
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// Image-gradient and lambda terms of pass application t, one thread per
// voxel (grid-stride), added to the accumulators in place: the terms of the
// children (next plane of the forward sweep) that chose the voxel, in
// offset order, then the term of its own parent.  Applications run in
// reverse order, so every voxel receives its terms in the order of the
// sequential reverse sweep.  CC > 0: exactly CC channels, summed in
// registers; CC == 0: any channel count, summed in the accumulator.
template <int CC>
__device__ void grad_app3(const Adj3DArgs& a, int t) {
    const float lam = a.lambda;
    const int C = CC > 0 ? CC : (int)a.C;
    const int n = (int)a.N;
    const PassGeom& g = a.pass[t % kMaxPasses];
    const int L = (int)g.L, P = (int)g.P, Q = (int)g.Q;
    const int sl = (int)g.sl, sp = (int)g.sp, sq = (int)g.sq;
    const int HW = (int)(a.H * a.W), Wd = (int)a.W;
    const float* s2t = a.s2[t % kMaxPasses];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.B * a.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / a.N;
        const int e = (int)(i - b * a.N);
        const int dd = e / HW, rem = e - dd * HW;
        const int hh = rem / Wd, ww = rem - hh * Wd;
        const float* img = a.image + b * a.C * a.N;
        float* gout = a.grad_image ? a.grad_image + b * a.C * a.N + e : nullptr;
        const float* A = a.A + b * a.N;
        const uint8_t* cd = a.codes + ((int64_t)(t - a.t_lo) * a.B + b) * a.N;
        float gi[CC > 0 ? CC : 1];
        if (CC > 0 && gout) {
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gi[ch] = gout[ch * a.N];
        }
        // g -= wgt (I(x) - I(y))  or  g += wgt (I(x) - I(y)), per channel
        auto add_term = [&](float wgt, int x, int y, bool minus) {
            if (CC > 0) {
#pragma unroll
                for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) {
                    const float term = __fmul_rn(wgt, __fsub_rn(img[ch * n + x], img[ch * n + y]));
                    gi[ch] = minus ? __fsub_rn(gi[ch], term) : __fadd_rn(gi[ch], term);
                }
            } else {
                for (int ch = 0; ch < C; ++ch) {
                    const float term = __fmul_rn(wgt, __fsub_rn(img[ch * n + x], img[ch * n + y]));
                    gout[ch * a.N] = minus ? __fsub_rn(gout[ch * a.N], term)
                                           : __fadd_rn(gout[ch * a.N], term);
                }
            }
        };
        const int line = g.axis == 0 ? dd : (g.axis == 1 ? hh : ww);
        const int p = g.axis == 0 ? hh : dd;
        const int q = g.axis == 2 ? hh : ww;
        // children on the next plane of the forward sweep, offset order: the
        // offsets whose child chose this voxel are collected first, then
        // visited in increasing order, so that a warp evaluates one cost per
        // step for all its lanes instead of one per offset any lane needs
        const int cl = line + g.dir;
        if (gout && cl >= 0 && cl < L) {
            unsigned int chose = 0u;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int cp = p - (k / 3 - 1), cq = q - (k % 3 - 1);
                if (cp < 0 || cp >= P || cq < 0 || cq >= Q) continue;
                if (cd[cl * sl + cp * sp + cq * sq] == k + 1) chose |= 1u << k;
            }
            while (chose) {
                const int k = __ffs(chose) - 1;
                chose &= chose - 1u;
                const int x = cl * sl + (p - (k / 3 - 1)) * sp + (q - (k % 3 - 1)) * sq;
                const float c = grad_cost3(img, x, e, C, n, g.t[k], lam);
                if (c > 0.0f) add_term(__fdiv_rn(__fmul_rn(A[x], lam), c), x, e, true);
            }
        }
        // own parent on the previous plane of the forward sweep
        const int code = cd[e];
        const int pl = line - g.dir;
        if (code >= 1 && code <= 9 && pl >= 0 && pl < L) {
            const int k = code - 1;
            const int pp = p + (k / 3 - 1), pq = q + (k % 3 - 1);
            if (pp >= 0 && pp < P && pq >= 0 && pq < Q) {
                const int y = pl * sl + pp * sp + pq * sq;
                float di2;
                const float c = grad_cost3(img, e, y, C, n, g.t[k], lam, &di2);
                if (c > 0.0f) {
                    if (a.lambda_terms)
                        a.lambda_terms[i] = __fadd_rn(
                            a.lambda_terms[i],
                            __fmul_rn(A[e], __fdiv_rn(__fsub_rn(di2, s2t[k]), __fadd_rn(c, c))));
                    if (gout) add_term(__fdiv_rn(__fmul_rn(A[e], lam), c), e, y, false);
                }
            }
        }
        if (CC > 0 && gout) {
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gout[ch * a.N] = gi[ch];
        }
    }
}

// The terms of one application as a launch of its own (full occupancy: the
// per-voxel gathers need many loads in flight).
template <int CC>
__global__ void __launch_bounds__(256) grad3d_kernel(const Adj3DArgs a, int t) {
    grad_app3<CC>(a, t);
}

// Pass applications t_hi-1 down to t_lo.  STORE_A: also write the adjoint of
// the (single) application into a.A for the gradient kernel.
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
    int in_idx = a.in_first;  // -1: the caller's dL/dD
    bool alive = true;
    for (int t_app = a.t_hi - 1; t_app >= a.t_lo && alive; --t_app) {
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
            t.K = a.ring[pass];
            t.tp = t.tq = kRP - 2 * t.K;
            t.p0 = (int64_t)t.jp * t.tp - t.K;
            t.q0 = (int64_t)t.jq * t.tq - t.K;
            const float* gsrc = (in_idx < 0 ? a.grad_dist : a.G[in_idx]) + b * a.N;
            if ((int)(threadIdx.x >> 5) >= kCW) {
                adj_producer3(a, t, gsrc,
                              a.codes + ((int64_t)(t_app - a.t_lo) * a.B + b) * a.N, h, stg, stc,
                              cb);
            } else {
                float* gdst = t_app > 0 ? a.G[out_idx] + b * a.N : nullptr;
                float* gmask = (t_app == 0 && a.grad_mask) ? a.grad_mask + b * a.N : nullptr;
                float* adst = STORE_A ? a.A + b * a.N : nullptr;
                float* g0 = (t_app == 0 && a.g0) ? a.g0 + b * a.N : nullptr;
                adj_compute3(a, t, a.T - 1 - t_app, h, stg, stc, cb, gdst, gmask, adst, g0);
            }
            cb += (unsigned int)nch;
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        in_idx = out_idx;
    }
}

struct Adj3DPlan {
    int grid = 0, max_tiles = 0;
    int ntp[kMaxPasses] = {}, ntq[kMaxPasses] = {}, ring[kMaxPasses] = {};
    size_t xbuf_off = 0, g_off[2] = {}, a_off = 0, total = 0;
};

using Adj3DKernel = void (*)(Adj3DArgs);
Adj3DKernel adj_kernel(bool store_a) {
    return store_a ? adj3d_kernel<true> : adj3d_kernel<false>;
}

bool plan_adj3d(const SweepArgs& f, int iterations, const fgx_options* opt, int sms,
                Adj3DPlan* p) {
    if (f.ndim != 3 || iterations <= 0) return false;
    // the forward's ring-width option (tile_lines 4 or 8 alone) does not
    // concern the reverse sweep's fixed ring; other tile options select the
    // tiled engine
    if (opt && (opt->tile_width || opt->tile_height)) return false;
    if (opt && opt->tile_lines && opt->tile_lines != 4 && opt->tile_lines != 8) return false;
    // offsets within one instance (image channels included) are int
    if (f.C * f.N >= ((int64_t)1 << 31)) return false;
    const size_t smem = adj3_smem_bytes();
    for (Adj3DKernel k : {adj_kernel(false), adj_kernel(true)})
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_kernel(true), kBlock3,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
        return false;
    int64_t cap = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) cap = std::min<int64_t>(cap, opt->max_blocks);
    // per pass the ring is 8 wide (16 x 16 owned, half the refreshes) where
    // its tiles still fit the grid in about as few waves as the narrow
    // ring's (the rule of the forward plane tiles)
    const int64_t B = std::max<int64_t>(f.B, 1);
    auto tiles = [](const PassGeom& g, int K) {
        const int64_t t = kRP - 2 * K;
        return std::max<int64_t>(1, (g.P + t - 1) / t) * std::max<int64_t>(1, (g.Q + t - 1) / t);
    };
    auto waves = [&](int64_t n) { return (B + cap / n - 1) / (cap / n); };
    int max_tiles = 1;
    for (int i = 0; i < kMaxPasses; ++i) {
        const PassGeom& g = f.pass[i];
        const int64_t n4 = tiles(g, kRing), n8 = tiles(g, kRingWide);
        if (n4 > (1 << 20) || n4 > cap) return false;
        int K = kRing;
        if (n8 <= cap && 3 * waves(n8) <= 4 * waves(n4)) K = kRingWide;
        const int t = kRP - 2 * K;
        p->ring[i] = K;
        p->ntp[i] = (int)std::max<int64_t>(1, (g.P + t - 1) / t);
        p->ntq[i] = (int)std::max<int64_t>(1, (g.Q + t - 1) / t);
        max_tiles = std::max(max_tiles, p->ntp[i] * p->ntq[i]);
    }
    p->max_tiles = max_tiles;
    int64_t grid = std::min<int64_t>(cap, B * max_tiles);
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
    // the adjoint of one pass application (the gradient terms use it
    // before the next application's sweep overwrites it)
    p->a_off = off;
    off += al((size_t)f.B * f.N * 4);
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
              float* g0, float* lambda_terms, const float* s2, int t_lo, int t_hi, int in_first,
              int* in_next, bool clear) {
    if (lambda_terms && !s2) return FGX_ERR_ARG;
    Adj3DPlan p;
    if (!plan_adj3d(f, iterations, opt, sms, &p)) return FGX_ERR_UNSUPPORTED;
    if (ws_bytes < p.total) return FGX_ERR_WORKSPACE;
    const int T = iterations * kMaxPasses;
    if (t_hi < 0) t_hi = T;
    if (t_lo < 0 || t_hi > T || t_lo >= t_hi) return FGX_ERR_ARG;
    char* w = (char*)workspace;
    Adj3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.grad_dist = grad_dist;
    a.codes = codes;
    a.grad_mask = grad_mask;
    a.g0 = g0;
    a.G[0] = (float*)(w + p.g_off[0]);
    a.G[1] = (float*)(w + p.g_off[1]);
    const bool grad = grad_image || lambda_terms;
    a.A = grad ? (float*)(w + p.a_off) : nullptr;
    a.B = f.B;
    a.N = f.N;
    a.v = v;
    a.T = T;
    a.t_lo = t_lo;
    a.t_hi = t_hi;
    a.in_first = in_first;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = p.ntp[i];
        a.ntq[i] = p.ntq[i];
        a.ring[i] = p.ring[i];
    }
    a.max_tiles = p.max_tiles;
    a.xbuf = (unsigned long long*)(w + p.xbuf_off);
    a.barrier = (unsigned int*)(w + 64);
    a.status = (int*)w;
    a.timeout_ns = f.timeout_ns;
    a.image = image;
    a.grad_image = grad_image;
    a.lambda_terms = lambda_terms;
    a.C = f.C;
    a.D = f.pass[0].L;  // extent of the axis of the first pass pair (D)
    a.H = f.pass[2].L;
    a.W = f.pass[4].L;
    a.lambda = f.lambda;
    if (s2)
        for (int i = 0; i < kMaxPasses; ++i)
            for (int k = 0; k < 9; ++k) a.s2[i][k] = s2[i * 9 + k];
    cudaStream_t s = (cudaStream_t)stream;
    // header and exchange words; a later range of the same call keeps the
    // status word (offset 0) that earlier ranges may have set
    const size_t from = clear ? 0 : 64;
    if (cudaMemsetAsync(w + from, 0, p.g_off[0] - from, s) != cudaSuccess) return FGX_ERR_CUDA;
    if (clear) {
        if (grad_image && cudaMemsetAsync(grad_image, 0, (size_t)(f.B * f.C * f.N) * 4, s) !=
                              cudaSuccess)
            return FGX_ERR_CUDA;
        if (lambda_terms &&
            cudaMemsetAsync(lambda_terms, 0, (size_t)(f.B * f.N) * 4, s) != cudaSuccess)
            return FGX_ERR_CUDA;
    }
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
    if (!grad) {
        if (cudaLaunchKernelEx(&cfg, adj_kernel(false), a) != cudaSuccess) return FGX_ERR_CUDA;
    } else {
        // one application per sweep launch, each followed by its gradient
        // terms (applications in reverse order, as the accumulation needs)
        const int64_t n = f.B * f.N;
        const int gg = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256,
                                                                   (int64_t)sms * 8));
        int idx = in_first;
        for (int t = t_hi - 1; t >= t_lo; --t) {
            a.t_lo = t;
            a.t_hi = t + 1;
            a.in_first = idx;
            // the codes of application t sit at (t - t_lo) of the caller's range
            a.codes = codes + (size_t)(t - t_lo) * (size_t)n;
            if (t != t_hi - 1 && cudaMemsetAsync(w + 64, 0, 4, s) != cudaSuccess)
                return FGX_ERR_CUDA;  // fresh grid-barrier counter
            if (cudaLaunchKernelEx(&cfg, adj_kernel(true), a) != cudaSuccess)
                return FGX_ERR_CUDA;
            if (f.C == 1) grad3d_kernel<1><<<gg, 256, 0, s>>>(a, t);
            else grad3d_kernel<0><<<gg, 256, 0, s>>>(a, t);
            if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
            idx = idx == 0 ? 1 : 0;
        }
    }
    if (in_next) {
        int idx = in_first;
        for (int t = t_hi - 1; t >= t_lo; --t) idx = idx == 0 ? 1 : 0;
        *in_next = idx;
    }
    return FGX_OK;
}

}  // namespace fgx
