// 3D forward on register-blocked plane tiles (FastGeodis, Implementation
// section: six passes per iteration, every voxel of a plane updated from the
// nine voxels of the already-updated previous plane).
//
// Decomposition.  One cooperative persistent launch runs all passes.  For a
// pass along one axis the plane (P x Q voxels) is cut into tiles of
// (32 - 2K) x (32 - 2K) owned voxels; one thread block per tile computes a
// region of kRP x kRQ = 32 x 32 voxels: the tile plus a ring of K voxels on
// every side, K = 4 or 8 per pass (the planner takes 8 where the larger tile
// count still fits the grid: half the ring refreshes for the same region).
// Sixteen compute warps each hold two region rows: lane q owns column q of
// the region and keeps the two distances of its rows in registers.  A
// plane step needs the 3 x 3 parents of every voxel: the own column's rows
// come from registers plus the two boundary rows of the warps above and below
// (shared memory, one named barrier of the compute warps per step), the
// neighbouring columns by warp shuffles.  The dependency cone shrinks the
// exact part of the region by one voxel per side and step, so the owned
// voxels stay exact for K steps; then every block publishes its owned
// voxels as 64-bit (value, tag) words and refreshes its ring from the
// owners' words (bounded polling, no fences: every word carries its own
// tag).  Passes are separated by a grid barrier.  Ring voxels are recomputed
// with exactly the operations of their owners, so results stay bit-exact.
// The outermost ring column of the region takes a neighbour value across the
// warp edge (the shuffle returns the lane's own value there); it lies outside
// the exact cone from the first step on, so no owned voxel depends on it.
//
// Staging.  Old distances and intensities (or cost tables) of upcoming
// planes sit in a shared ring of kNst chunks of kChunk planes (Ring3); each
// staged array has a spare row above and below the region, so every parent
// load of a lane is one base register plus a constant offset.  Rows of the
// pass layouts are padded to 16 bytes where needed (pitched working copies
// of the distances and image, transposed copies for the W passes).  Two
// ways to fill the ring:
//  * tensor memory accelerator (every volume with W > 1): one producer warp
//    copies the plane tiles of a chunk
//    as boxes (cp.async.bulk.tensor, one box per lane) as soon as the chunk
//    slot is free, completed on the slot's mbarrier by transaction count;
//    outside the volume the copy fills distances with NaN (a NaN candidate
//    never wins fminf, exactly like +inf) and intensities with 0.  Issuing
//    the copies from a compute thread put them on the plane steps' critical
//    path (about a quarter of the step time, measured);
//  * otherwise (W = 1, or no tensor-map encoder) four producer warps copy
//    the tile with per-lane 4-byte cp.async (voxels outside the volume:
//    distance +inf, intensity 0).
//
// Edge costs, in the fixed order of the method:
//  constant (lambda = 0): sqrt(t_k), one constant per stencil offset;
//  absolute (lambda = 1, one channel): |I(x) - I(y)|, which equals
//    sqrt_rn(fl(d*d)) for d = 0 and 2^-63 <= |d| <= 2^63; a first kernel
//    checks that every intensity is 0 or has magnitude in [2^-40, 2^62],
//    which bounds every difference to that range; otherwise each candidate
//    is checked and falls back to the square root;
//  general: sqrt_rn(t_k + lambda * sum_ch (I(x)-I(y))^2), read from tables
//    written once per call (nine per voxel and axis) on the tensor-copy
//    path, else evaluated in every pass;
//  fast (fast-math option, forward without codes): the general formula with
//    fused multiply-adds and the approximate square root.
#include <cuda.h>  // CUtensorMap and its encoder's signature (the encoder is looked up at run time)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;

constexpr int kRows = 2;                  // region rows per compute thread
constexpr int kCW = 16;                   // compute warps
constexpr int kPW = 4;                    // producer warps (cp.async staging)
constexpr int kTW = 1;                    // producer warps (tensor copies)
constexpr int kRP = kRows * kCW;          // region rows
constexpr int kRQ = 32;                   // region columns (one per lane)
constexpr int kRing = 4;                  // narrow ring width = steps between refreshes
constexpr int kRingWide = 8;              // wide ring width
constexpr int kTP = kRP - 2 * kRing;      // owned rows of a narrow-ring tile (the most)
constexpr int kTQ = kRQ - 2 * kRing;      // owned columns of a narrow-ring tile
constexpr int kArr = (kRP + 2) * kRQ;     // floats of one staged array (spare row above and below)
constexpr int kMaxCI = 3;                 // intensity channels the stage holds
constexpr int kTabArrays = 9;             // staged arrays of a cost-table pass (one per parent)
constexpr int kXWords = kTP * kTQ;        // published words per tile and parity (room for the most)
constexpr int kRangeFlagOffset = 32;      // workspace header: intensity range flag
constexpr int kTransposeWarps = 8;        // warps of a block that transpose (8 shared tiles)
constexpr int kMaps = 6;
#define kInf3 __int_as_float(0x7f800000)

// Staging ring geometry R: kNst chunks of kChunk planes.  R = 0: 12 planes
// of up to 1 + kMaxCI arrays; R = 1: 5 planes of 1 + kTabArrays arrays (the
// cost-table mode), a chunk a plane.
template <int R>
struct Ring3 {
    static constexpr int kChunk = R == 0 ? 4 : 1;
    static constexpr int kNst = R == 0 ? 3 : 5;
    static constexpr int kSlots = kNst * kChunk;
    static_assert(kRing % kChunk == 0 && kRingWide % kChunk == 0, "refreshes at chunk boundaries");
};
constexpr int kNstMax = 5;

// Edge-cost modes of the plane-tile kernel; kModeTable: the general cost read
// from tables written once per call (nine per voxel and axis).
enum { kModeConst = 0, kModeAbs = 1, kModeGeneral = 2, kModeFast = 3, kModeTable = 4 };
// Tensor maps of one call: distances and intensities in the layouts of the
// D passes ([D][H][W], box = one plane tile), the H passes (same arrays, box
// spanning D) and the W passes (the [W][D][H] copies).
enum { kMapDistD = 0, kMapDistH = 1, kMapDistW = 2, kMapImgD = 3, kMapImgH = 4, kMapImgW = 5 };

struct Vol3DArgs {  // aligned as CUtensorMap (the descriptor arrays of batched runs too)
    CUtensorMap tmap[kMaps];   // tensor-memory-accelerator launches only
    const float* image;  // [B][C][N]
    const float* mask;   // [B][N]
    float* dist;         // [B][N]
    uint8_t* codes;      // [iterations * 6][B][N] parent codes, or null
    int64_t B, C, N;
    int64_t nimg;        // distinct images: instance b reads image b % nimg
    float v, lambda;
    int iterations;
    int mode;
    PassGeom pass[kMaxPasses];
    int ntp[kMaxPasses], ntq[kMaxPasses];
    int ring[kMaxPasses];      // ring width K of each pass (4 or 8)
    int max_tiles;
    unsigned long long* xbuf;  // [B][max_tiles][2 parities][kXWords]
    unsigned int* barrier;
    int* status;
    const int* range_flag;     // nonzero: some intensity outside the |d| range
    long long timeout_ns;
    // W passes on transposed copies (planes of those passes have H as their
    // contiguous axis, so staging loads and result stores are coalesced):
    float* distT;              // [B][W][D][H], or null (W passes on dist itself)
    float* imageT;             // [nimg][C][W][D][H] (cost modes that read intensities)
    int64_t D, H, W;
    // batched instances: the passes run on pitched working copies (rows of
    // Wp floats in [D][H][Wp], of Hp floats in the W passes' [W][D][Hp]) so
    // that every staged row starts on a 16-byte boundary; `out` and
    // `image_src` are the caller's arrays when dist / image are such copies
    // (null when they are the caller's own)
    int64_t Wp, Hp;
    float* out;
    const float* image_src;
    float* tables;  // batched cost tables: D axis, H axis ([9][D][H][Wp] each), W axis ([9][W][D][Hp])
    // strides of line, p and q of every pass in the caller's [D][H][W] order
    // (the codes' layout)
    int64_t csl[kMaxPasses], csp[kMaxPasses], csq[kMaxPasses];
};

struct Head3 {
    unsigned long long full[kNstMax], empty[kNstMax];
    float rowtop[2][kCW][kRQ];  // first row of each warp, per step parity
    float rowbot[2][kCW][kRQ];  // last row of each warp
};

__device__ __align__(16) unsigned int g_inf4[4] = {0x7f800000u, 0x7f800000u, 0x7f800000u,
                                                  0x7f800000u};
__device__ __align__(16) unsigned int g_zero4v[4] = {0u, 0u, 0u, 0u};

__device__ __forceinline__ unsigned int saddr3(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async4(unsigned int dst, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(gmem) : "memory");
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
__device__ __forceinline__ void mbar_expect_tx3(unsigned long long* b, unsigned int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     saddr3(b)),
                 "r"(bytes)
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
// Bounded wait that ignores the status word: used after a failure to let
// this block's own tensor copies land before the block moves on.
__device__ __noinline__ void mbar_drain3(unsigned long long* b, unsigned int parity,
                                         long long timeout_ns) {
    const long long t0 = gtimer();
    while (!mbar_try3(b, parity) && gtimer() - t0 <= timeout_ns) {
    }
}
// One box of a 4D tensor map into shared memory, completed on `mbar`.
__device__ __forceinline__ void tma_load4(unsigned int dst, const CUtensorMap* m, int x, int y,
                                          int z, int w, unsigned int mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
        "l"(m), "r"(x), "r"(y), "r"(z), "r"(w), "r"(mbar)
        : "memory");
}
// Compute-warp barrier (producer warps never join it).
__device__ __forceinline__ void compute_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(kCW * 32) : "memory");
}

// One tile of one pass application.
struct Tile3 {
    const PassGeom* g;
    float* dist;       // distances of this instance in the pass's layout
    const float* img;  // intensities of this instance in the pass's layout (channel stride N)
    uint8_t* codes;    // this application's codes of the instance (image order), or null
    int64_t csl, csp, csq;  // strides of line, p and q in the image order of the codes
    int64_t cst;       // channel stride of the intensities in the pass's layout
    int tile, ntq, L, nch;
    int K, tp, tq;     // ring width and owned extents (tp = tq = 32 - 2K)
    int p0, q0;        // plane coordinates of region row 0 and column 0
    int64_t b;
    // tensor maps of the pass and the order of the box coordinates: the
    // plane tile's row axis is the box's z (H passes) or y (other passes)
    int map_d, map_i, rows_z;
};

// Stage geometry: floats of one staged plane (distances, then intensities).
template <int CI>
struct Stage3 {
    static constexpr int kPlaneF = (1 + CI) * kArr;
};

// TMA: chunk c of the tile (global chunk count gc) into its slot, issued by
// the lanes of one warp: lane l copies array l % (1 + CI) of plane l / (1 + CI)
// of the chunk (one box each), all completed on the slot's mbarrier.
template <int CI, int R>
__device__ void tma_chunk(const Vol3DArgs& a, const Tile3& t, Head3& h, float* stage,
                          unsigned int gc, int c) {
    constexpr int PF = Stage3<CI>::kPlaneF;
    constexpr int kNst = Ring3<R>::kNst, kChunk = Ring3<R>::kChunk;
    const int lane = threadIdx.x & 31;
    const int slot = (int)(gc % kNst);
    const int jn = min(kChunk, t.L - c * kChunk);
    const unsigned int mb = saddr3(&h.full[slot]);
    if (lane == 0) mbar_expect_tx3(&h.full[slot], (unsigned int)(jn * (1 + CI) * kRP * kRQ * 4));
    __syncwarp();
    if (lane < jn * (1 + CI)) {
        const int j = lane / (1 + CI), arr = lane - j * (1 + CI);
        const int s = c * kChunk + j;
        const int line = t.g->dir > 0 ? s : t.L - 1 - s;
        const unsigned int dst = saddr3(stage + (slot * kChunk + j) * PF + kRQ + arr * kArr);
        const int y = t.rows_z ? line : t.p0, z = t.rows_z ? t.p0 : line;
        const int w4 = arr == 0 ? (int)t.b : (int)((t.b % a.nimg) * CI) + arr - 1;
        tma_load4(dst, &a.tmap[arr == 0 ? t.map_d : t.map_i], t.q0, y, z, w4, mb);
    }
}

// Producer warp (tensor copies): every chunk of the tile into the ring once
// the compute warps have released its slot.  On a failure it stops issuing.
// Either way it waits (bounded) until its last copies have landed.
template <int CI, int R>
__device__ bool producer3_tma(const Vol3DArgs& a, const Tile3& t, Head3& h, float* stage,
                              unsigned int cb) {
    constexpr int kNst = Ring3<R>::kNst;
    // shared memory written by ordinary stores (transposes) is handed to the
    // tensor copies
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    int c = 0;
    bool ok = true;
    for (; c < t.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = (int)(gc % kNst);
        if (gc >= (unsigned)kNst &&
            !__all_sync(0xffffffffu, mbar_wait3(&h.empty[slot], ((gc / kNst) & 1u) ^ 1u,
                                                a.status, a.timeout_ns))) {
            ok = false;
            break;
        }
        tma_chunk<CI, R>(a, t, h, stage, gc, c);
    }
    // the last copies of the tile have landed before the warp moves on (after
    // a failure the compute warps may no longer wait for them)
    if ((threadIdx.x & 31) == 0)
        for (int k = max(0, c - kNst); k < c; ++k)
            mbar_drain3(&h.full[(cb + k) % kNst], ((cb + k) / kNst) & 1u, a.timeout_ns);
    __syncwarp();
    return ok;
}

// Producer warps (cp.async staging): planes of old distances and intensities
// into the ring, chunk after chunk, once the compute warps have released the
// slot.  Voxels outside the volume are staged with distance +inf and
// intensity 0 (finite costs: a square root never sees an infinite argument).
template <int CI, int R>
__device__ bool producer3(const Vol3DArgs& a, const Tile3& t, Head3& h, float* stage,
                          unsigned int cb) {
    constexpr int PF = Stage3<CI>::kPlaneF;
    constexpr int kNst = Ring3<R>::kNst, kChunk = Ring3<R>::kChunk;
    constexpr int NR = kRP / kPW;  // rows per producer lane
    const PassGeom& g = *t.g;
    const int lane = threadIdx.x & 31, pw = (threadIdx.x >> 5) - kCW;
    const int q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    int64_t roff[NR];
    unsigned int inm = 0;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
        const int p = t.p0 + pw + kPW * rr;
        if (qin && p >= 0 && p < g.P) inm |= 1u << rr;
        roff[rr] = (int64_t)p * g.sp + (int64_t)q * g.sq;
    }
    const int64_t dsl = g.dir > 0 ? g.sl : -g.sl;
    int64_t lo = g.dir > 0 ? 0 : (int64_t)(t.L - 1) * g.sl;
    const unsigned int sbase = saddr3(stage) + (unsigned int)(((1 + pw) * kRQ + lane) * 4);
    const float* dist = t.dist;
    const float* img = t.img;
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
            const unsigned int dst = sbase + (unsigned int)((slot * kChunk + j) * PF) * 4u;
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) {
                const bool in = (inm >> rr) & 1u;
                const int64_t off = lo + roff[rr];
                const unsigned int dr = dst + (unsigned int)(kPW * rr * kRQ) * 4u;
                cp_async4(dr, in ? (const void*)(dist + off) : (const void*)g_inf4);
#pragma unroll
                for (int ch = 0; ch < CI; ++ch)
                    cp_async4(dr + (unsigned int)((1 + ch) * kArr) * 4u,
                              in ? (const void*)(img + ch * t.cst + off) : (const void*)g_zero4v);
            }
            lo += dsl;
        }
        cp_arrive_noinc(&h.full[slot]);
    }
    return true;
}

// Ring refresh after step s: publish the owned voxels of plane s, then take
// every ring voxel inside the volume from the tile that owns it.  xmine /
// xsrc: this lane's word offsets (parity 0) of its own and its source words
// per row, -1 where none.
__device__ bool exchange3(const Vol3DArgs& a, int64_t b, int tile, unsigned int tg, int par,
                          float (&d)[kRows], const int (&xmine)[kRows],
                          const int (&xsrc)[kRows]) {
    const int lane = threadIdx.x & 31;
    unsigned long long* base = a.xbuf + (size_t)b * a.max_tiles * 2 * kXWords;
    unsigned long long* mine = base + ((size_t)tile * 2 + par) * kXWords;
    const unsigned long long* src = base + (size_t)par * kXWords;
    unsigned int need = 0;
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        if (xmine[i] >= 0)
            st_relaxed_u64(mine + xmine[i],
                           ((unsigned long long)tg << 32) | (unsigned int)__float_as_uint(d[i]));
        if (xsrc[i] >= 0) need |= 1u << i;
    }
    long long t0 = 0;
    for (unsigned int it = 0;; ++it) {
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            if (!((need >> i) & 1u)) continue;
            const unsigned long long wv = ld_relaxed_u64(src + xsrc[i]);
            if ((unsigned int)(wv >> 32) == tg) {
                d[i] = __uint_as_float((unsigned int)wv);
                need &= ~(1u << i);
            }
        }
        if (__all_sync(0xffffffffu, need == 0)) return true;
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
        di2 = ch == 0 ? __fmul_rn(d, d)
                      : (MODE == kModeFast ? __fmaf_rn(d, d, di2) : __fadd_rn(di2, __fmul_rn(d, d)));
    }
    return MODE == kModeFast ? fast_sqrt(__fmaf_rn(lam, di2, t))
                             : __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// Compute warps of one tile: plane steps 1 .. L-1, ring refresh every K
// steps, owned voxels written to the distance map (and with CODES their
// parent codes: 0 if the voxel kept its value, else 1 + the lowest stencil
// offset whose candidate is the strictly smaller minimum).  Thread 0 hands
// every chunk slot back once no compute warp reads it any more.
template <int MODE, int CI, bool CHECKED, bool CODES, bool TMA, int R>
__device__ bool compute3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h, float* stage,
                         unsigned int cb) {
    constexpr bool kTab = MODE == kModeTable;
    constexpr int NI = CI > 0 && !kTab ? CI : 1;
    constexpr int PF = Stage3<CI>::kPlaneF;
    constexpr int kNst = Ring3<R>::kNst, kChunk = Ring3<R>::kChunk, kSlots = Ring3<R>::kSlots;
    const PassGeom& g = *t.g;
    const bool early = kTab && g.dir > 0;  // the previous plane's slot is released a step early
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int rows0 = w * kRows;
    const int q = t.q0 + lane;
    const bool qin = q >= 0 && q < g.Q;
    const int K = t.K, tp = t.tp, tq = t.tq;
    const bool qown = lane >= K && lane < K + tq;
    const int64_t line0 = g.dir > 0 ? 0 : (int64_t)(t.L - 1);
    const int64_t dsl = g.dir > 0 ? g.sl : -g.sl;
    const int64_t dcl = g.dir > 0 ? t.csl : -t.csl;
    bool valid[kRows], own[kRows];
    float* dp[kRows];
    uint8_t* cp[CODES ? kRows : 1];
    int xmine[kRows], xsrc[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const int r = rows0 + i;
        const int p = t.p0 + r;
        valid[i] = qin && p >= 0 && p < g.P;
        const bool pown = r >= K && r < K + tp;
        own[i] = valid[i] && qown && pown;
        dp[i] = t.dist + line0 * g.sl + (int64_t)p * g.sp + (int64_t)q * g.sq;
        if (CODES) cp[i] = t.codes + line0 * t.csl + (int64_t)p * t.csp + (int64_t)q * t.csq;
        xmine[i] = own[i] ? (r - K) * tq + (lane - K) : -1;
        xsrc[i] = -1;
        if (valid[i] && !(pown && qown)) {
            const int op = p / tp, oq = q / tq;
            xsrc[i] = (op * t.ntq + oq) * 2 * kXWords + (p - op * tp) * tq + (q - oq * tq);
        }
    }
    const float lam = a.lambda;
    float tk[9], ck[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        tk[k] = g.t[k];
        ck[k] = g.c[k];
    }
    // this lane's element (region row rows0, column lane) of array 0 of ring plane 0
    const float* S = stage + (1 + rows0) * kRQ + lane;
    int cur = (int)(cb % kNst) * kChunk * PF;
    // After a failure (timeout, or one reported by another block) the warps
    // keep stepping through the named barriers with every wait skipped, so
    // that no compute warp is left waiting for one that gave up.
    bool failed = !__all_sync(0xffffffffu, mbar_wait3(&h.full[cb % kNst], (cb / kNst) & 1u,
                                                      a.status, a.timeout_ns));
    float d[kRows];
#pragma unroll
    for (int i = 0; i < kRows; ++i) d[i] = S[cur + i * kRQ];
    const unsigned int tag_base = ((unsigned int)(t_app + 1)) << 16;
    int xi = 0;
    unsigned int gc = cb;  // chunk of the current plane
    int j = 0;             // plane within the chunk
    for (int s = 1; s < t.L; ++s) {
        const int prev = cur;
        cur += PF;
        if (cur == kSlots * PF) cur = 0;
        if (++j == kChunk) {
            j = 0;
            ++gc;
            if (!failed && !__all_sync(0xffffffffu, mbar_wait3(&h.full[gc % kNst],
                                                               (gc / kNst) & 1u, a.status,
                                                               a.timeout_ns)))
                failed = true;
        }
        // boundary rows of plane s-1 for the warps above and below
        const int rb = s & 1;
        h.rowtop[rb][w][lane] = d[0];
        h.rowbot[rb][w][lane] = d[kRows - 1];
        compute_sync();
        // plane s-2 is no longer read by any compute warp (plane s-1 already,
        // in a forward sweep reading cost tables: its costs sit at the
        // voxel, so the previous plane's slot is not read): its chunk slot is
        // free once it was the chunk's last plane
        if (threadIdx.x == 0) {
            const int fp = s - (early ? 1 : 2);
            if (fp >= 0 && (fp & (kChunk - 1)) == kChunk - 1)
                mbar_arrive3(&h.empty[(cb + fp / kChunk) % kNst]);
        }
        float col[kRows + 2], lft[kRows + 2], rgt[kRows + 2];
        col[0] = w > 0 ? h.rowbot[rb][w - 1][lane] : kInf3;
#pragma unroll
        for (int i = 0; i < kRows; ++i) col[i + 1] = d[i];
        col[kRows + 1] = w < kCW - 1 ? h.rowtop[rb][w + 1][lane] : kInf3;
#pragma unroll
        for (int k = 0; k < kRows + 2; ++k) {
            lft[k] = __shfl_up_sync(0xffffffffu, col[k], 1);
            rgt[k] = __shfl_down_sync(0xffffffffu, col[k], 1);
        }
        // old distances and intensities of plane s, intensities of plane s-1
        const float* Sc = S + cur;
        const float* Sp = S + prev;
        float ip[kRows + 2][3][NI], ix[kRows][NI];
        // cost tables: the costs of the nine parents of every voxel of the
        // plane in sweep order; a forward sweep reads them at the voxel
        // (array 1 + k of plane s), a backward sweep at the parent, whose
        // table holds the same edge under the mirrored offset 8 - k (array
        // 9 - k of plane s-1, shifted by the offset)
        float tc[kTab ? kRows : 1][9];
        if (kTab) {
            if (g.dir > 0) {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 9; ++k) tc[i][k] = Sc[(1 + k) * kArr + i * kRQ];
            } else {
#pragma unroll
                for (int i = 0; i < kRows; ++i)
#pragma unroll
                    for (int k = 0; k < 9; ++k)
                        tc[i][k] = Sp[(9 - k) * kArr + (i + k / 3 - 1) * kRQ + (k % 3 - 1)];
            }
        }
        if (CI > 0 && !kTab) {
#pragma unroll
            for (int k = 0; k < kRows + 2; ++k)
#pragma unroll
                for (int ch = 0; ch < NI; ++ch) {
                    const float* Pi = Sp + (1 + ch) * kArr + (k - 1) * kRQ;
                    ip[k][0][ch] = Pi[-1];
                    ip[k][1][ch] = Pi[0];
                    ip[k][2][ch] = Pi[1];
                }
#pragma unroll
            for (int i = 0; i < kRows; ++i)
#pragma unroll
                for (int ch = 0; ch < NI; ++ch) ix[i][ch] = Sc[(1 + ch) * kArr + i * kRQ];
        }
#pragma unroll
        for (int i = 0; i < kRows; ++i) {
            float best = Sc[i * kRQ];
            unsigned int code = 0;
#pragma unroll
            for (int dpp = -1; dpp <= 1; ++dpp) {
#pragma unroll
                for (int dq = -1; dq <= 1; ++dq) {
                    const int k = (dpp + 1) * 3 + (dq + 1);
                    const int rk = i + 1 + dpp;
                    const float pd = dq < 0 ? lft[rk] : (dq == 0 ? col[rk] : rgt[rk]);
                    const float c = kTab ? tc[kTab ? i : 0][k]
                                         : cost3<MODE, NI, CHECKED>(ix[i], ip[rk][dq + 1], tk[k],
                                                                    ck[k], lam);
                    const float cand = __fadd_rn(pd, c);
                    if (CODES && cand < best) code = (unsigned int)(k + 1);
                    best = fminf(best, cand);
                }
            }
            d[i] = valid[i] ? best : kInf3;
            dp[i] += dsl;
            if (CODES) cp[i] += dcl;
            if (own[i]) {
                *dp[i] = d[i];
                if (CODES) *cp[i] = (uint8_t)code;
            }
        }
        if ((s & (K - 1)) == 0 && s + 1 < t.L) {
            if (!failed && !exchange3(a, t.b, t.tile, tag_base | (unsigned int)(xi + 1), xi & 1, d,
                                      xmine, xsrc))
                failed = true;
            ++xi;
        }
    }
    compute_sync();
    if (threadIdx.x == 0) {
        // free the chunks still held (those whose last plane is one of the
        // last two, or the last one)
        const int held = early ? 1 : 2;
        for (int c = max(0, t.nch - 2); c < t.nch; ++c) {
            const int last = min(c * kChunk + kChunk - 1, t.L - 1);
            if (last >= t.L - held) mbar_arrive3(&h.empty[(cb + c) % kNst]);
        }
    }
    return !failed;
}

// D0 = v * M (unless dist is null: a call that resumes from the distances
// already in place), and the intensity range test that allows |d| as the
// cost.
__global__ void __launch_bounds__(256) init3d_kernel(const float* mask, float* dist, float v,
                                                     int64_t n, const float* image, int64_t ni,
                                                     int* range_flag) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (dist)
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

// One 32 x 32 tile of a transpose between the two pitched layouts of an
// instance, by one warp: forward from [D][H][sp] to [W][D][dp] (sp, dp: row
// pitches), back the other way.  unit = (d, tile row, tile column) over the
// H x W plane of slice d.  `tile`: this warp's 32 x 33 floats of shared
// memory.  The sources may have been written by other blocks of the same
// launch: read through L2.
__device__ void transpose_unit(const float* src, float* dst, int64_t D, int64_t H, int64_t W,
                               int64_t sp, int64_t dp, bool back, int64_t unit, float* tile) {
    const int lane = threadIdx.x & 31;
    const int64_t th = (H + 31) / 32, tw = (W + 31) / 32;
    const int64_t d = unit / (th * tw), rem = unit - d * (th * tw);
    const int64_t h0 = (rem / tw) * 32, w0 = (rem % tw) * 32;
    float v[32];
    if (!back) {
        // rows h0 + y, columns w0 + lane of slice d
#pragma unroll
        for (int y = 0; y < 32; ++y) {
            const int64_t h = h0 + y, w = w0 + lane;
            v[y] = (h < H && w < W) ? __ldcg(src + (d * H + h) * sp + w) : 0.0f;
        }
    } else {
        // rows w0 + y, columns h0 + lane of the transposed slice d
#pragma unroll
        for (int y = 0; y < 32; ++y) {
            const int64_t w = w0 + y, h = h0 + lane;
            v[y] = (h < H && w < W) ? __ldcg(src + (w * D + d) * sp + h) : 0.0f;
        }
    }
#pragma unroll
    for (int y = 0; y < 32; ++y) tile[y * 33 + lane] = v[y];
    __syncwarp();
#pragma unroll
    for (int y = 0; y < 32; ++y) {
        const float x = tile[lane * 33 + y];
        if (!back) {
            const int64_t w = w0 + y, h = h0 + lane;
            if (w < W && h < H) dst[(w * D + d) * dp + h] = x;
        } else {
            const int64_t h = h0 + y, w = w0 + lane;
            if (w < W && h < H) dst[(d * H + h) * dp + w] = x;
        }
    }
    __syncwarp();
}

__device__ __forceinline__ int64_t transpose_units(const Vol3DArgs& a) {
    return a.D * ((a.H + 31) / 32) * ((a.W + 31) / 32);
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

// The distance transposes of a single call around the W passes: every
// instance between [D][H][Wp] (the working distances) and [W][D][Hp], 32 x 32
// tiles spread over kTransposeWarps warps of every block (dense layouts as
// one tall matrix per instance, which runs faster).
__device__ void transpose_single(const Vol3DArgs& a, bool back, float* smem) {
    if (a.Wp == a.W && a.Hp == a.H) {
        // dense layouts: one [D*H][W] matrix per instance
        transpose_rw(back ? a.distT : a.dist, back ? a.dist : a.distT, a.B, a.D * a.H, a.W, back,
                     smem, kTransposeWarps);
        return;
    }
    const int warp = threadIdx.x >> 5;
    if (warp < kTransposeWarps) {
        float* tile = smem + warp * (32 * 33);
        const int64_t nw = (int64_t)gridDim.x * kTransposeWarps;
        const int64_t per = transpose_units(a);
        const int64_t nd = a.D * a.H * a.Wp, nt = a.W * a.D * a.Hp;
        for (int64_t u = (int64_t)blockIdx.x * kTransposeWarps + warp; u < a.B * per; u += nw) {
            const int64_t b = u / per;
            const float* src = back ? a.distT + b * nt : a.dist + b * nd;
            float* dst = back ? a.dist + b * nd : a.distT + b * nt;
            transpose_unit(src, dst, a.D, a.H, a.W, back ? a.Hp : a.Wp, back ? a.Wp : a.Hp, back,
                           u - b * per, tile);
        }
    }
    __syncthreads();
}

// The image of a single call in the W passes' layout [nimg][C][W][D][Hp], once
// per call from the caller's [nimg][C][D][H][W] (all SMs, before the
// persistent launch).
__global__ void __launch_bounds__(256) transpose_image3d_kernel(const float* image, float* imageT,
                                                                int64_t count, int64_t D,
                                                                int64_t H, int64_t W,
                                                                int64_t Hp) {
    __shared__ float smem[8 * 32 * 33];
    if (Hp == H) {
        transpose_rw(image, imageT, count, D * H, W, false, smem, 8);
        return;
    }
    const int warp = threadIdx.x >> 5;
    const int64_t per = D * ((H + 31) / 32) * ((W + 31) / 32);
    for (int64_t u = (int64_t)blockIdx.x * 8 + warp; u < count * per; u += (int64_t)gridDim.x * 8) {
        const int64_t c = u / per;
        transpose_unit(image + c * D * H * W, imageT + c * W * D * Hp, D, H, W, W, Hp, false,
                       u - c * per, smem + warp * (32 * 33));
    }
}

// Pitched working copies of a single call (instance blockIdx.y): the
// distances [D][H][Wp] (D0 = v * M, or the caller's distances when the call
// resumes from them) and, for instances below nimg, the image; one warp per
// row of W voxels.
__global__ void __launch_bounds__(256) pitch3d_kernel(const Vol3DArgs a, bool resume) {
    const int64_t b = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t rows = a.D * a.H, nd = rows * a.Wp;
    for (int64_t r = w0; r < rows; r += nw)
        for (int64_t x = lane; x < a.W; x += 32) {
            const int64_t i = b * a.N + r * a.W + x;
            a.dist[b * nd + r * a.Wp + x] = resume ? a.out[i] : __fmul_rn(a.v, a.mask[i]);
        }
    if (a.image_src && b < a.nimg)
        for (int64_t r = w0; r < a.C * rows; r += nw)
            for (int64_t x = lane; x < a.W; x += 32)
                const_cast<float*>(a.image)[b * a.C * nd + r * a.Wp + x] =
                    a.image_src[b * a.C * a.N + r * a.W + x];
}

// The caller's distances from the pitched working copies (instance blockIdx.y).
__global__ void __launch_bounds__(256) unpitch3d_kernel(const Vol3DArgs a) {
    const int64_t b = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t rows = a.D * a.H, nd = rows * a.Wp;
    for (int64_t r = w0; r < rows; r += nw)
        for (int64_t x = lane; x < a.W; x += 32)
            a.out[b * a.N + r * a.W + x] = __ldcg(a.dist + b * nd + r * a.Wp + x);
}

// Edge-cost tables of one axis (the general cost, once per call instead of in
// every pass application): for every voxel x of line l >= 1 of the axis'
// forward sweep and every stencil offset k, the cost of the edge between x
// and its parent x - e + (k / 3 - 1, k % 3 - 1) (previous line, in-plane
// offset along p and q), in exactly the order of the on-the-fly general cost:
// sqrt_rn(t_k + lambda * sum_ch (I(x) - I(y))^2).  The cost is symmetric bit
// for bit ((a - b)^2 = (b - a)^2 in rounded arithmetic; t_k depends on the
// squared offset), so a backward sweep reads the same edge at the parent
// under the mirrored offset 8 - k.  A parent outside the volume gets the cost
// of a zero difference (never used: its distance is +inf or NaN).
// Layouts: the intensities and the table share the pass geometry g (strides
// sl, sp, sq); channel ch at img + ch * cstride, offset k at tab + k * kstride.
template <int C>
__device__ void cost_table_axis(const float* img, int cstride, float* tab, int kstride,
                                  const PassGeom& g, float lam, int64_t warp0, int64_t nwarps) {
    // one warp per line of the plane (lanes along q; no division per voxel),
    // the nine parent loads of a voxel independent of one another; offsets
    // within one image fit 32 bits (the planner checks 9 N < 2^31)
    const int lane = threadIdx.x & 31;
    const int P = (int)g.P, Q = (int)g.Q, sl = (int)g.sl, sp = (int)g.sp, sq = (int)g.sq;
    const int64_t rows = (g.L - 1) * g.P;
    for (int64_t row = warp0; row < rows; row += nwarps) {
        const int l = 1 + (int)(row / P), p = (int)(row - (int64_t)(l - 1) * P);
        const int bx = l * sl + p * sp, by = (l - 1) * sl + p * sp;
        for (int q = lane; q < Q; q += 32) {
            const int ox = bx + q * sq;
            float ix[C], iy[9][C];
#pragma unroll
            for (int ch = 0; ch < C; ++ch) ix[ch] = img[ch * cstride + ox];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int dp = k / 3 - 1, dq = k % 3 - 1;
                const bool in = p + dp >= 0 && p + dp < P && q + dq >= 0 && q + dq < Q;
                const int oy = by + dp * sp + (q + dq) * sq;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) iy[k][ch] = in ? img[ch * cstride + oy] : ix[ch];
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                float di2 = 0.0f;
#pragma unroll
                for (int ch = 0; ch < C; ++ch) {
                    const float d = __fsub_rn(ix[ch], iy[k][ch]);
                    di2 = ch == 0 ? __fmul_rn(d, d) : __fadd_rn(di2, __fmul_rn(d, d));
                }
                tab[k * kstride + ox] = __fsqrt_rn(__fadd_rn(g.t[k], __fmul_rn(lam, di2)));
            }
        }
    }
}
// Tables of the three axes of `count` images (blockIdx.y = axis): image i at
// image + i * istride (D and H axes) or imageT + i * istride (W axis), its
// tables at tabs[axis] + i * tstride.
struct CostTables {
    const float* img[3];
    float* tab[3];
    PassGeom g[3];
    int64_t cstride[3], kstride[3], istride[3], tstride[3];
    int64_t count;
    int C;
    float lam;
};
template <int C>
__global__ void __launch_bounds__(256) cost_table3d_kernel(const CostTables ct) {
    const int ax = blockIdx.y;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    for (int64_t i = 0; i < ct.count; ++i)
        cost_table_axis<C>(ct.img[ax] + i * ct.istride[ax], (int)ct.cstride[ax],
                           ct.tab[ax] + i * ct.tstride[ax], (int)ct.kstride[ax], ct.g[ax], ct.lam,
                           w0, nw);
}

template <int MODE, int CI, bool CODES, bool TMA, int R>
__device__ __forceinline__ bool run_tile3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h,
                                          float* stage, unsigned int cb, bool checked) {
    if ((int)(threadIdx.x >> 5) >= kCW)
        return TMA ? producer3_tma<CI, R>(a, t, h, stage, cb)
                   : producer3<CI, R>(a, t, h, stage, cb);
    if (MODE == kModeAbs && checked)
        return compute3<MODE, CI, true, CODES, TMA, R>(a, t, t_app, h, stage, cb);
    return compute3<MODE, CI, false, CODES, TMA, R>(a, t, t_app, h, stage, cb);
}

// Shared-memory layout of a block: the head, then the staging ring at the
// next 128-byte boundary (tensor copies land on 128-byte boundaries).
__device__ __forceinline__ float* stage_of(unsigned char* smem) {
    const unsigned int base = saddr3(smem);
    const unsigned int st = (base + (unsigned int)sizeof(Head3) + 127u) & ~127u;
    return reinterpret_cast<float*>(smem + (st - base));
}

__device__ __forceinline__ void init_barriers3(Head3& h, bool tma) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNstMax; ++i) {
            // one transaction-counted arrival (TMA) or one per producer lane
            mbar_init3(&h.full[i], tma ? 1u : (unsigned int)(kPW * 32));
            mbar_init3(&h.empty[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
}

template <int MODE, int CI, bool CODES, bool TMA>
__global__ void __launch_bounds__(TMA ? (kCW + kTW) * 32 : (kCW + kPW) * 32, 1)
    vol3d_kernel(const __grid_constant__ Vol3DArgs a) {
    extern __shared__ __align__(128) unsigned char smem3[];
    Head3& h = *reinterpret_cast<Head3*>(smem3);
    float* stage = stage_of(smem3);
    init_barriers3(h, TMA);
    const bool checked = MODE == kModeAbs && *a.range_flag != 0;
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[0] = (unsigned long long)gtimer();
    unsigned int epoch = 1;
    unsigned int cb = 0;  // staging chunks handed over so far in this block
    const int napps = a.iterations * kMaxPasses;
    bool alive = true;
    const bool tw = a.distT != nullptr;
    // instance strides of the working and transposed layouts
    const int64_t nd = a.D * a.H * a.Wp, nt = a.W * a.D * a.Hp;

    for (int t_app = 0; t_app < napps && alive; ++t_app) {
        const int pass = t_app % kMaxPasses;
        const PassGeom& g = a.pass[pass];
        const bool on_t = tw && pass >= 4;  // this pass runs on the transposed copies
        if (tw && pass == 4) {
            transpose_single(a, false, stage);
            if (!(alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns))) break;
        }
        const int ntiles = a.ntp[pass] * a.ntq[pass];
        const int per_wave = gridDim.x / ntiles;
        const int64_t nwaves = (a.B + per_wave - 1) / per_wave;
        const int L = (int)g.L;
        constexpr int RG = MODE == kModeTable ? 1 : 0;  // staging ring geometry
        const int nch = L > 1 ? (L + Ring3<RG>::kChunk - 1) / Ring3<RG>::kChunk : 0;
        for (int64_t wv = 0; wv < nwaves; ++wv) {
            if ((int)blockIdx.x >= per_wave * ntiles) continue;
            const int64_t b = wv * per_wave + blockIdx.x / ntiles;
            if (b >= a.B) continue;
            Tile3 t;
            t.g = &g;
            t.tile = blockIdx.x % ntiles;
            t.ntq = a.ntq[pass];
            t.b = b;
            t.dist = on_t ? a.distT + b * nt : a.dist + b * nd;
            t.img = on_t ? a.imageT + (b % a.nimg) * a.C * nt : a.image + (b % a.nimg) * a.C * nd;
            t.codes = CODES ? a.codes + ((int64_t)t_app * a.B + b) * a.N : nullptr;
            t.csl = a.csl[pass];
            t.csp = a.csp[pass];
            t.csq = a.csq[pass];
            t.cst = on_t ? nt : nd;
            t.L = L;
            t.nch = nch;
            t.K = a.ring[pass];
            t.tp = t.tq = kRP - 2 * t.K;
            t.p0 = (t.tile / t.ntq) * t.tp - t.K;
            t.q0 = (t.tile % t.ntq) * t.tq - t.K;
            t.map_d = pass < 2 ? kMapDistD : (pass < 4 ? kMapDistH : kMapDistW);
            t.map_i = t.map_d + 3;
            t.rows_z = pass == 2 || pass == 3;
            if (nch > 0) run_tile3<MODE, CI, CODES, TMA, RG>(a, t, t_app, h, stage, cb, checked);
            cb += (unsigned int)nch;
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        if (alive && tw && pass == 5) {
            transpose_single(a, true, stage);
            alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 1 < 16)
            timeline[t_app + 1] = (unsigned long long)gtimer();
    }
}

// Batched launch: work list of (instance, tile) items per round, one round
// per pass application, grid barrier between rounds; every instance has its
// own arguments (cost mode, planes, exchange words, range flag, tensor maps)
// and runs on pitched working copies, so every plane is staged by tensor
// copies.
struct Vol3DBatch {
    const Vol3DArgs* desc;
    int n;                    // instances
    int rounds;
    const int* round_waves;   // [rounds + 1]
    const int* wave_items;    // [waves][gridDim.x]: (instance << 16) | tile, or -1
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
};

// The distance transposes of round r of a batched launch: every instance
// that applies pass 4 in this round (forward) or applied pass 5 (back).
// Units are spread over kTransposeWarps warps of every block.
__device__ void transpose_round(const Vol3DBatch& bt, int r, bool back, float* smem) {
    const int warp = threadIdx.x >> 5;
    if (warp < kTransposeWarps) {
        float* tile = smem + warp * (32 * 33);
        const int64_t nw = (int64_t)gridDim.x * kTransposeWarps;
        const int64_t gw = (int64_t)blockIdx.x * kTransposeWarps + warp;
        int64_t base = 0;
        for (int k = 0; k < bt.n; ++k) {
            const Vol3DArgs& a = bt.desc[k];
            if (r >= a.iterations * kMaxPasses) continue;
            const int64_t nu = transpose_units(a);
            for (int64_t u = ((gw - base) % nw + nw) % nw; u < nu; u += nw)
                transpose_unit(back ? a.distT : a.dist, back ? a.dist : a.distT, a.D, a.H, a.W,
                               back ? a.Hp : a.Wp, back ? a.Wp : a.Hp, back, u, tile);
            base += nu;
        }
    }
    __syncthreads();
}

// D0 = v * M into the working distances of instance blockIdx.y, the pitched
// copy of its image when it has one, and the intensity range test.
__global__ void __launch_bounds__(256) init3d_batched_kernel(const Vol3DArgs* desc) {
    const Vol3DArgs& a = desc[blockIdx.y];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float* img = a.image_src ? a.image_src : a.image;
    // one warp per row of W voxels (rows of the caller's layout to rows of
    // the pitched copy), lanes along the row
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    const int64_t rows = a.D * a.H;
    for (int64_t r = w0; r < rows; r += nw)
        for (int64_t x = lane; x < a.W; x += 32)
            a.dist[r * a.Wp + x] = __fmul_rn(a.v, a.mask[r * a.W + x]);
    if (a.image_src && a.mode != kModeConst)
        for (int64_t r = w0; r < a.C * rows; r += nw)
            for (int64_t x = lane; x < a.W; x += 32)
                const_cast<float*>(a.image)[r * a.Wp + x] = a.image_src[r * a.W + x];
    if (a.mode != kModeAbs) return;
    int* flag = const_cast<int*>(a.range_flag);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.C * a.N; i += stride) {
        const float x = fabsf(img[i]);
        const bool ok = x == 0.0f || (x >= 0x1p-40f && x <= 0x1p62f);
        if (!ok && *(volatile int*)flag == 0) atomicOr(flag, 1);
    }
}

// The image of instance blockIdx.y in the W passes' layout [C][W][D][Hp],
// from the caller's image (channel slices stacked along D).
__global__ void __launch_bounds__(256) transpose_image3d_batched_kernel(const Vol3DArgs* desc) {
    __shared__ float smem[8 * 32 * 33];
    const Vol3DArgs& a = desc[blockIdx.y];
    if (a.mode == kModeConst || !a.imageT) return;
    const float* src = a.image_src ? a.image_src : a.image;
    const int warp = threadIdx.x >> 5;
    // channel c is slices c*D .. c*D + D - 1 of a [C*D][H][W] stack
    const int64_t nu = a.C * transpose_units(a);
    for (int64_t u = (int64_t)blockIdx.x * 8 + warp; u < nu; u += (int64_t)gridDim.x * 8) {
        const int64_t per = transpose_units(a);
        const int64_t c = u / per;
        transpose_unit(src + c * a.N, a.imageT + c * a.W * a.D * a.Hp, a.D, a.H, a.W, a.W, a.Hp,
                       false, u - c * per, smem + warp * (32 * 33));
    }
}

// The caller's distances of the instances that ran on pitched copies.
__global__ void __launch_bounds__(256) finish3d_batched_kernel(const Vol3DArgs* desc) {
    const Vol3DArgs& a = desc[blockIdx.y];
    if (!a.out) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = w0; r < a.D * a.H; r += nw)
        for (int64_t x = lane; x < a.W; x += 32) a.out[r * a.W + x] = __ldcg(a.dist + r * a.Wp + x);
}

// Cost tables of the batched instances with C channels that read them
// (blockIdx.y = instance).
template <int C>
__global__ void __launch_bounds__(256) cost_table3d_batched_kernel(const Vol3DArgs* desc) {
    const Vol3DArgs& a = desc[blockIdx.y];
    if (a.mode != kModeTable || a.C != C) return;
    const int pl = (int)(a.D * a.H * a.Wp), plT = (int)(a.W * a.D * a.Hp);
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x / 32);
    cost_table_axis<C>(a.image, pl, a.tables, pl, a.pass[0], a.lambda, w0, nw);
    cost_table_axis<C>(a.image, pl, a.tables + kTabArrays * pl, pl, a.pass[2], a.lambda, w0, nw);
    cost_table_axis<C>(a.imageT, plT, a.tables + 2 * kTabArrays * pl, plT, a.pass[4], a.lambda,
                       w0, nw);
}

// One batched item in ring geometry R (R = 1 when some instance of the
// launch reads cost tables: every item then stages planes one by one).
template <int R>
__device__ bool run_item3(const Vol3DArgs& a, const Tile3& t, int t_app, Head3& h, float* stage,
                          unsigned int cb) {
    if (a.mode == kModeConst)
        return run_tile3<kModeConst, 0, false, true, R>(a, t, t_app, h, stage, cb, false);
    if (a.mode == kModeAbs)
        return run_tile3<kModeAbs, 1, false, true, R>(a, t, t_app, h, stage, cb,
                                                      *a.range_flag != 0);
    if (R == 1 && a.mode == kModeTable)
        return run_tile3<kModeTable, kTabArrays, false, true, R>(a, t, t_app, h, stage, cb,
                                                                 false);
    if (a.mode == kModeFast) {
        if (a.C == 1)
            return run_tile3<kModeFast, 1, false, true, R>(a, t, t_app, h, stage, cb, false);
        if (a.C == 2)
            return run_tile3<kModeFast, 2, false, true, R>(a, t, t_app, h, stage, cb, false);
        return run_tile3<kModeFast, 3, false, true, R>(a, t, t_app, h, stage, cb, false);
    }
    if (a.C == 1)
        return run_tile3<kModeGeneral, 1, false, true, R>(a, t, t_app, h, stage, cb, false);
    if (a.C == 2)
        return run_tile3<kModeGeneral, 2, false, true, R>(a, t, t_app, h, stage, cb, false);
    return run_tile3<kModeGeneral, 3, false, true, R>(a, t, t_app, h, stage, cb, false);
}

constexpr int kBlockBatched3 = (kCW + kTW) * 32;

template <int R>
__global__ void __launch_bounds__(kBlockBatched3, 1) vol3d_batched_kernel(const Vol3DBatch bt) {
    extern __shared__ __align__(128) unsigned char smem3[];
    Head3& h = *reinterpret_cast<Head3*>(smem3);
    float* stage = stage_of(smem3);
    init_barriers3(h, true);
    unsigned int epoch = 1;
    unsigned int cb = 0;
    bool alive = true;
    for (int r = 0; r < bt.rounds && alive; ++r) {
        const int pass = r % kMaxPasses;
        if (pass == 4) {
            transpose_round(bt, r, false, stage);
            if (!(alive = grid_barrier(bt.barrier, epoch++, bt.status, bt.timeout_ns))) break;
        }
        for (int wv = bt.round_waves[r]; wv < bt.round_waves[r + 1]; ++wv) {
            const int item = bt.wave_items[(int64_t)wv * gridDim.x + blockIdx.x];
            if (item < 0) continue;
            const Vol3DArgs& a = bt.desc[item >> 16];
            const PassGeom& g = a.pass[pass];
            const bool on_t = pass >= 4;
            Tile3 t;
            t.g = &g;
            t.tile = item & 0xffff;
            t.ntq = a.ntq[pass];
            t.b = 0;
            t.dist = on_t ? a.distT : a.dist;
            t.img = on_t ? a.imageT : a.image;
            t.codes = nullptr;
            t.csl = t.csp = t.csq = 0;
            t.cst = on_t ? a.W * a.D * a.Hp : a.D * a.H * a.Wp;
            t.L = (int)g.L;
            t.nch = t.L > 1 ? (t.L + Ring3<R>::kChunk - 1) / Ring3<R>::kChunk : 0;
            t.K = a.ring[pass];
            t.tp = t.tq = kRP - 2 * t.K;
            t.p0 = (t.tile / t.ntq) * t.tp - t.K;
            t.q0 = (t.tile % t.ntq) * t.tq - t.K;
            t.map_d = pass < 2 ? kMapDistD : (pass < 4 ? kMapDistH : kMapDistW);
            t.map_i = t.map_d + 3;
            t.rows_z = pass == 2 || pass == 3;
            if (t.nch > 0) run_item3<R>(a, t, r, h, stage, cb);
            cb += (unsigned int)t.nch;
        }
        alive = grid_barrier(bt.barrier, epoch++, bt.status, bt.timeout_ns);
        if (alive && pass == 5) {
            transpose_round(bt, r, true, stage);
            alive = grid_barrier(bt.barrier, epoch++, bt.status, bt.timeout_ns);
        }
    }
}

// Dynamic shared memory of a block staging 1 + CI arrays a plane in ring
// geometry R (R = 1: the cost-table ring).
size_t stage_bytes(int CI, int R = 0) {
    const size_t head = (sizeof(Head3) + 127) & ~size_t(127);
    const int slots = R ? Ring3<1>::kSlots : Ring3<0>::kSlots;
    // the ring, plus one row of slack for the last lane's right-hand reads
    const size_t st = (size_t)(slots * (1 + CI) * kArr + kRQ) * sizeof(float);
    return head + st + 128;  // + up to 127 bytes of alignment
}

using Vol3DKernel = void (*)(Vol3DArgs);

template <bool CODES, bool TMA>
Vol3DKernel pick_kernel_t(int mode, int CI) {
    if (mode == kModeConst) return vol3d_kernel<kModeConst, 0, CODES, TMA>;
    if (mode == kModeAbs) return vol3d_kernel<kModeAbs, 1, CODES, TMA>;
    // the fast-math mode serves forwards without codes only
    if (mode == kModeFast && !CODES) {
        if (CI == 1) return vol3d_kernel<kModeFast, 1, false, TMA>;
        if (CI == 2) return vol3d_kernel<kModeFast, 2, false, TMA>;
        return vol3d_kernel<kModeFast, 3, false, TMA>;
    }
    if (CI == 1) return vol3d_kernel<kModeGeneral, 1, CODES, TMA>;
    if (CI == 2) return vol3d_kernel<kModeGeneral, 2, CODES, TMA>;
    return vol3d_kernel<kModeGeneral, 3, CODES, TMA>;
}
Vol3DKernel pick_kernel(int mode, int CI, bool codes, bool tma) {
    // cost tables are staged by tensor copies only
    if (mode == kModeTable)
        return !tma ? nullptr
                    : codes ? vol3d_kernel<kModeTable, kTabArrays, true, true>
                            : vol3d_kernel<kModeTable, kTabArrays, false, true>;
    if (tma)
        return codes ? pick_kernel_t<true, true>(mode, CI) : pick_kernel_t<false, true>(mode, CI);
    return codes ? pick_kernel_t<true, false>(mode, CI) : pick_kernel_t<false, false>(mode, CI);
}
int block_threads(bool tma) { return tma ? (kCW + kTW) * 32 : (kCW + kPW) * 32; }

// A float32 tensor map of dims (d0 innermost .. d3), rows of `pitch` floats
// (0: d0), with box (b0, b1, b2, 1); NaN fill outside the tensor for
// distances, zero for intensities.
bool make_map(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2,
              uint64_t d3, uint32_t b0, uint32_t b1, uint32_t b2, bool nan_fill,
              uint64_t pitch = 0) {
    const uint64_t dims[4] = {d0, d1, d2, d3};
    const uint32_t box[4] = {b0, b1, b2, 1};
    return encode_map_f32(m, base, 4, dims, box, nan_fill, pitch);
}

// Tensor maps of a call (false: stage with cp.async).  The rows of every
// staged plane must start on 16-byte boundaries: W (the D and H passes) and
// H (the W passes on the transposed copies) multiples of 4.
bool make_maps(Vol3DArgs& a) {
    const uint64_t D = (uint64_t)a.D, H = (uint64_t)a.H, W = (uint64_t)a.W;
    const uint64_t B = (uint64_t)a.B, BC = (uint64_t)(a.nimg * a.C);
    const uint64_t Wp = (uint64_t)a.Wp, Hp = (uint64_t)a.Hp;
    if (Wp % 4 || Hp % 4 || !a.distT) return false;
    if (D > (1u << 30) || H > (1u << 30) || W > (1u << 30) || BC > (1u << 30)) return false;
    bool ok = make_map(&a.tmap[kMapDistD], a.dist, W, H, D, B, kRQ, kRP, 1, true, Wp) &&
              make_map(&a.tmap[kMapDistH], a.dist, W, H, D, B, kRQ, 1, kRP, true, Wp) &&
              make_map(&a.tmap[kMapDistW], a.distT, H, D, W, B, kRQ, kRP, 1, true, Hp);
    if (ok && a.mode != kModeConst)
        ok = make_map(&a.tmap[kMapImgD], a.image, W, H, D, BC, kRQ, kRP, 1, false, Wp) &&
             make_map(&a.tmap[kMapImgH], a.image, W, H, D, BC, kRQ, 1, kRP, false, Wp) &&
             make_map(&a.tmap[kMapImgW], a.imageT, H, D, W, BC, kRQ, kRP, 1, false, Hp);
    return ok;
}

struct Vol3DPlan {
    int mode = 0, CI = 0, grid = 0, max_tiles = 0;
    int ntp[kMaxPasses] = {}, ntq[kMaxPasses] = {}, ring[kMaxPasses] = {};
    size_t smem = 0, ws_bytes = 0;
    size_t zero_bytes = 0;             // header and exchange words (cleared per call)
    size_t distT_off = 0, imageT_off = 0;  // transposed copies for the W passes
    // cost tables (general cost on tensor-copy layouts): [B][9][D][H][Wp] for
    // the D axis, then the H axis, then the W axis in its [W][D][Hp] layout;
    // ws_bytes includes them when tab_bytes > 0, ws_min_bytes does not
    size_t tab_off = 0, tab_bytes = 0, ws_min_bytes = 0;
    int64_t Wp = 0, Hp = 0;            // row pitches of the working and transposed layouts
    size_t pd_off = 0, pi_off = 0;     // pitched working copies of the distances and image (or 0)
};

int64_t tiles_of(const PassGeom& g, int K) {
    const int64_t t = kRP - 2 * K;
    return std::max<int64_t>(1, (g.P + t - 1) / t) * std::max<int64_t>(1, (g.Q + t - 1) / t);
}

// Whether the 3D call fits this kernel (at most kMaxCI channels in the
// general cost, every tile of a pass co-resident, no tile-shape options),
// and its launch geometry.  Per pass the ring is 8 wide where its tiles
// still fit the grid in about as few waves as the narrow ring's: a plane
// step with the narrow ring costs about two units (the step and a quarter of
// a refresh that takes as long as four steps' arithmetic), with the wide ring
// about 1.5.  `wide` = false keeps every pass narrow (batched launches).
bool plan_vol3d(const SweepArgs& f, const fgx_options* opt, int sms, Vol3DPlan* vp,
                bool any_mode = false, bool wide = true) {
    if (f.ndim != 3) return false;
    // tile_lines alone = 4 or 8 forces the ring width of every pass (8 where
    // the tiles fit the grid); any other tile option selects the tiled engine
    if (opt && (opt->tile_width || opt->tile_height)) return false;
    const int force = opt ? opt->tile_lines : 0;
    if (force && force != kRing && force != kRingWide) return false;
    vp->mode = f.cost_mode == kCostConst ? kModeConst
               : f.cost_mode == kCostAbs ? kModeAbs
               : f.cost_mode == kCostFast ? kModeFast : kModeGeneral;
    vp->CI = vp->mode == kModeConst ? 0 : (int)f.C;
    // a workspace-size query covers every cost mode: plan the cheapest one
    if (any_mode) {
        vp->mode = kModeConst;
        vp->CI = 0;
    }
    if (vp->CI > kMaxCI) return false;
    // plane coordinates are int: every extent below 2^30
    for (int i = 0; i < kMaxPasses; ++i)
        if (f.pass[i].L >= (1 << 30) || f.pass[i].P >= (1 << 30) || f.pass[i].Q >= (1 << 30))
            return false;
    vp->smem = stage_bytes(vp->CI);
    // occupancy of the cp.async variant (the larger block) bounds both
    Vol3DKernel k = pick_kernel(vp->mode, vp->CI, false, false);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)vp->smem) !=
        cudaSuccess)
        return false;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block_threads(false),
                                                      vp->smem) != cudaSuccess ||
        per_sm < 1)
        return false;
    int64_t cap = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) cap = std::min<int64_t>(cap, opt->max_blocks);
    const int64_t B = std::max<int64_t>(f.B, 1);
    auto waves = [&](int64_t n) { return (B + cap / n - 1) / (cap / n); };
    int64_t max_tiles = 1, xtiles = 1;
    for (int i = 0; i < kMaxPasses; ++i) {
        const PassGeom& g = f.pass[i];
        const int64_t n4 = tiles_of(g, kRing), n8 = tiles_of(g, kRingWide);
        if (n4 > (1 << 20) || n4 > cap) return false;
        int K = kRing;
        if (n8 <= cap) {
            xtiles = std::max(xtiles, n8);
            if (force ? force == kRingWide : wide && 3 * waves(n8) <= 4 * waves(n4))
                K = kRingWide;
        }
        xtiles = std::max(xtiles, n4);
        const int t = kRP - 2 * K;
        vp->ring[i] = K;
        vp->ntp[i] = (int)std::max<int64_t>(1, (g.P + t - 1) / t);
        vp->ntq[i] = (int)std::max<int64_t>(1, (g.Q + t - 1) / t);
        max_tiles = std::max<int64_t>(max_tiles, (int64_t)vp->ntp[i] * vp->ntq[i]);
    }
    // the exchange area has room for either ring choice of every pass, so a
    // workspace sized by the size query serves every call of that shape
    vp->max_tiles = (int)xtiles;
    vp->grid = (int)std::min<int64_t>(cap, B * max_tiles);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    vp->zero_bytes = kHeaderBytes + (size_t)B * xtiles * 2 * kXWords * 8;
    // rows padded to 16 bytes (pitches Wp, Hp) so that every plane stages by
    // tensor copies: the W passes' transposed copies always carry the pitch
    // Hp; with W not a multiple of 4 the distances and the image also get
    // pitched working copies (results copied back after the launch).  A
    // volume with W = 1 has no W passes and keeps the caller's arrays.
    const int64_t D = f.pass[0].L, H = f.pass[2].L, W = f.pass[4].L;
    vp->Wp = W > 1 ? (W + 3) / 4 * 4 : W;
    vp->Hp = W > 1 ? (H + 3) / 4 * 4 : H;
    const size_t nd = (size_t)D * H * vp->Wp, nt = (size_t)W * D * vp->Hp;
    vp->distT_off = al(vp->zero_bytes);
    vp->imageT_off = vp->distT_off + al((size_t)f.B * nt * 4);
    vp->ws_bytes = vp->imageT_off + al((size_t)f.B * f.C * nt * 4);
    vp->pd_off = vp->pi_off = 0;
    if (vp->Wp != W) {
        vp->pd_off = vp->ws_bytes;
        vp->pi_off = vp->pd_off + al((size_t)f.B * nd * 4);
        vp->ws_bytes = vp->pi_off + al((size_t)f.B * f.C * nd * 4);
    }
    vp->ws_min_bytes = vp->ws_bytes;
    // the general cost reads tables on the tensor-copy path (W > 1); a size
    // query (any_mode) covers them
    const bool tab = (any_mode || vp->mode == kModeGeneral) && W > 1 &&
                     !(opt && opt->no_cost_tables) &&
                     (int64_t)kTabArrays * (int64_t)std::max(nd, nt) < ((int64_t)1 << 31);
    if (tab) {
        vp->tab_off = vp->ws_bytes;
        vp->tab_bytes = al((size_t)f.B * 9 * (2 * nd + nt) * 4);
        vp->ws_bytes += vp->tab_bytes;
    }
    return true;
}

}  // namespace

// cuTensorMapEncodeTiled, looked up once through the runtime (no link-time
// dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn tensor_map_encoder() {
    static EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

bool encode_map_f32(void* map, const void* base, int rank, const uint64_t* dims,
                    const uint32_t* box, bool nan_fill, uint64_t row_pitch) {
    EncodeTiledFn enc = tensor_map_encoder();
    const uint64_t rp = row_pitch ? row_pitch : dims[0];
    if (!enc || rank < 1 || rank > 5 || ((uintptr_t)base & 15u) || ((rp * 4) & 15u) ||
        rp < dims[0])
        return false;
    cuuint64_t d[5], str[4];
    cuuint32_t b[5], e[5];
    uint64_t pitch = 4;
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        b[i] = box[i];
        e[i] = 1;
        if (i > 0) str[i - 1] = pitch;
        pitch *= i == 0 ? rp : dims[i];
    }
    return enc(static_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank,
               const_cast<void*>(base), d, str, b, e, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA
                        : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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
              int sms, void* stream, bool resume, int64_t nimg) {
    Vol3DPlan vp;
    if (!plan_vol3d(f, opt, sms, &vp)) return FGX_ERR_UNSUPPORTED;
    if (ws_bytes < vp.ws_min_bytes) return FGX_ERR_WORKSPACE;
    Vol3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = image;
    a.mask = mask;
    a.dist = dist;
    a.codes = codes;
    a.B = f.B;
    a.C = f.C;
    a.N = f.N;
    a.nimg = nimg > 0 ? nimg : std::max<int64_t>(f.B, 1);
    a.v = v;
    a.lambda = f.lambda;
    a.iterations = f.iterations;
    a.mode = vp.mode;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = vp.ntp[i];
        a.ntq[i] = vp.ntq[i];
        a.ring[i] = vp.ring[i];
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
    a.Wp = vp.Wp;
    a.Hp = vp.Hp;
    // the codes keep the caller's element order: (line, p, q) strides of
    // every pass in [D][H][W] (the W passes' lines are columns)
    for (int i = 0; i < kMaxPasses; ++i) {
        a.csl[i] = i < 4 ? f.pass[i].sl : 1;
        a.csp[i] = i < 4 ? f.pass[i].sp : a.H * a.W;
        a.csq[i] = i < 4 ? f.pass[i].sq : a.W;
    }
    if (a.W > 1) {
        // the W passes run on [W][D][Hp] copies: their planes' rows are contiguous
        a.distT = (float*)(w + vp.distT_off);
        a.imageT = vp.mode == kModeConst ? nullptr : (float*)(w + vp.imageT_off);
        for (int i = 4; i < 6; ++i) {
            a.pass[i].sl = a.D * a.Hp;
            a.pass[i].sp = a.Hp;
            a.pass[i].sq = 1;
        }
    }
    if (vp.pd_off) {
        // rows of W floats are not 16-byte aligned: the passes run on pitched
        // working copies [D][H][Wp] and the results are copied back
        a.dist = (float*)(w + vp.pd_off);
        a.out = dist;
        if (vp.mode != kModeConst) {
            a.image = (const float*)(w + vp.pi_off);
            a.image_src = image;
        }
        for (int i = 0; i < 4; ++i) {
            a.pass[i].sl = i < 2 ? a.H * a.Wp : a.Wp;
            a.pass[i].sp = i < 2 ? a.Wp : a.H * a.Wp;
            a.pass[i].sq = 1;
        }
    }
    const bool tma = make_maps(a);
    // the general cost from tables when the workspace holds them (tensor
    // copies only): the intensity maps then address the tables, nine
    // arrays per image and axis
    size_t smem = vp.smem;
    const bool tab = tma && vp.mode == kModeGeneral && vp.tab_bytes > 0 && ws_bytes >= vp.ws_bytes;
    float* tabs[3] = {nullptr, nullptr, nullptr};
    const int64_t nd = a.D * a.H * a.Wp, nt = a.W * a.D * a.Hp;
    if (tab) {
        const uint64_t D = (uint64_t)a.D, H = (uint64_t)a.H, W = (uint64_t)a.W;
        const uint64_t n9 = (uint64_t)a.nimg * kTabArrays;
        tabs[0] = (float*)(w + vp.tab_off);
        tabs[1] = tabs[0] + n9 * (uint64_t)nd;
        tabs[2] = tabs[1] + n9 * (uint64_t)nd;
        if (make_map(&a.tmap[kMapImgD], tabs[0], W, H, D, n9, kRQ, kRP, 1, false, a.Wp) &&
            make_map(&a.tmap[kMapImgH], tabs[1], W, H, D, n9, kRQ, 1, kRP, false, a.Wp) &&
            make_map(&a.tmap[kMapImgW], tabs[2], H, D, W, n9, kRQ, kRP, 1, false, a.Hp)) {
            a.mode = kModeTable;
            smem = stage_bytes(kTabArrays, 1);
        } else if (!make_maps(a)) {
            return FGX_ERR_CUDA;  // the intensity maps could be encoded a moment ago
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
    // D0 (into the caller's distances unless they are pitched or the call
    // resumes) and the intensity range test
    init3d_kernel<<<std::max(ig, 1), 256, 0, s>>>(mask, resume || a.out ? nullptr : dist, v, n,
                                                 image, a.nimg * f.C * f.N,
                                                 vp.mode == kModeAbs ? range_flag : nullptr);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if (a.out) {
        pitch3d_kernel<<<dim3((unsigned)std::max(1, sms * 4), (unsigned)f.B), 256, 0, s>>>(a,
                                                                                      resume);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    if (a.imageT && f.iterations > 0) {
        transpose_image3d_kernel<<<sms * 8, 256, 0, s>>>(image, a.imageT, a.nimg * f.C, a.D, a.H,
                                                          a.W, a.Hp);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    if (f.iterations == 0) return FGX_OK;
    if (a.mode == kModeTable) {
        CostTables ct;
        std::memset(&ct, 0, sizeof(ct));
        const int src_pass[3] = {0, 2, 4};
        for (int ax = 0; ax < 3; ++ax) {
            const int64_t pl = ax < 2 ? nd : nt;
            ct.img[ax] = ax < 2 ? a.image : a.imageT;
            ct.tab[ax] = tabs[ax];
            ct.g[ax] = a.pass[src_pass[ax]];
            ct.cstride[ax] = pl;
            ct.kstride[ax] = pl;
            ct.istride[ax] = f.C * pl;
            ct.tstride[ax] = kTabArrays * pl;
        }
        ct.count = a.nimg;
        ct.C = (int)f.C;
        ct.lam = f.lambda;
        const dim3 tg((unsigned)(sms * 4), 3);
        if (f.C == 1) cost_table3d_kernel<1><<<tg, 256, 0, s>>>(ct);
        else if (f.C == 2) cost_table3d_kernel<2><<<tg, 256, 0, s>>>(ct);
        else cost_table3d_kernel<3><<<tg, 256, 0, s>>>(ct);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)vp.grid);
    cfg.blockDim = dim3((unsigned)block_threads(tma));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    Vol3DKernel k = a.mode == kModeTable
                        ? pick_kernel(kModeTable, kTabArrays, codes != nullptr, true)
                        : pick_kernel(vp.mode, vp.CI, codes != nullptr, tma);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaLaunchKernelEx(&cfg, k, a) != cudaSuccess)
        return FGX_ERR_CUDA;
    if (a.out) {
        unpitch3d_kernel<<<dim3((unsigned)std::max(1, sms * 4), (unsigned)f.B), 256, 0, s>>>(a);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

// ---------------------------------------------------- batched 3D instances ----

size_t vol3d_desc_size() { return sizeof(Vol3DArgs); }

bool vol3d_instance_desc(void* desc, const fgx_instance& it, const SweepArgs& f,
                         const fgx_options* opt, int sms, char* hdr, int* range_flag, char* xb,
                         char* work, size_t* xbytes, size_t* wbytes, int* ci, int* max_tiles,
                         int tiles[kMaxPasses]) {
    Vol3DPlan vp;
    if (!plan_vol3d(f, opt, sms, &vp, false, false)) return false;
    const int64_t D = f.pass[0].L, H = f.pass[2].L, W = f.pass[4].L;
    const int64_t Wp = (W + 3) / 4 * 4, Hp = (H + 3) / 4 * 4;
    const bool pitched = Wp != W;
    const bool img = vp.mode != kModeConst;
    const bool tab = vp.mode == kModeGeneral && !(opt && opt->no_cost_tables) &&
                     (int64_t)kTabArrays * std::max(D * H * Wp, W * D * Hp) < ((int64_t)1 << 31);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    // working copies: [pitched dist | pitched image] | transposed dist |
    // transposed image | [cost tables of the D, H and W axes]
    const size_t pd = pitched ? al((size_t)D * H * Wp * 4) : 0;
    const size_t pi = pitched && img ? al((size_t)f.C * D * H * Wp * 4) : 0;
    const size_t td = al((size_t)W * D * Hp * 4);
    const size_t ti = img ? al((size_t)f.C * W * D * Hp * 4) : 0;
    const size_t tb =
        tab ? al((size_t)kTabArrays * (2 * (size_t)D * H * Wp + (size_t)W * D * Hp) * 4) : 0;
    *xbytes = (size_t)vp.max_tiles * 2 * kXWords * 8;
    *wbytes = pd + pi + td + ti + tb;
    *ci = tab ? kTabArrays : vp.CI;
    *max_tiles = vp.max_tiles;
    for (int i = 0; i < kMaxPasses; ++i) tiles[i] = vp.ntp[i] * vp.ntq[i];
    if (!desc) return true;
    Vol3DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.image = pitched && img ? (const float*)(work + pd) : it.image;
    a.image_src = pitched && img ? it.image : nullptr;
    a.mask = it.mask;
    a.dist = pitched ? (float*)work : it.dist;
    a.out = pitched ? it.dist : nullptr;
    a.distT = (float*)(work + pd + pi);
    a.imageT = img ? (float*)(work + pd + pi + td) : nullptr;
    a.B = 1;
    a.nimg = 1;
    a.C = f.C;
    a.N = f.N;
    a.D = D;
    a.H = H;
    a.W = W;
    a.Wp = Wp;
    a.Hp = Hp;
    a.v = it.v;
    a.lambda = f.lambda;
    a.iterations = it.iterations;
    a.mode = tab ? kModeTable : vp.mode;
    a.tables = tab ? (float*)(work + pd + pi + td + ti) : nullptr;
    for (int i = 0; i < kMaxPasses; ++i) {
        a.pass[i] = f.pass[i];
        a.ntp[i] = vp.ntp[i];
        a.ntq[i] = vp.ntq[i];
        a.ring[i] = vp.ring[i];
    }
    // strides of the working layouts: [D][H][Wp] for the D and H passes,
    // [W][D][Hp] for the W passes
    for (int i = 0; i < 2; ++i) {
        a.pass[i].sl = H * Wp;
        a.pass[i].sp = Wp;
        a.pass[i].sq = 1;
    }
    for (int i = 2; i < 4; ++i) {
        a.pass[i].sl = Wp;
        a.pass[i].sp = H * Wp;
        a.pass[i].sq = 1;
    }
    for (int i = 4; i < 6; ++i) {
        a.pass[i].sl = D * Hp;
        a.pass[i].sp = Hp;
        a.pass[i].sq = 1;
    }
    a.max_tiles = vp.max_tiles;
    a.xbuf = (unsigned long long*)xb;
    a.barrier = (unsigned int*)(hdr + 64);
    a.status = (int*)hdr;
    a.range_flag = range_flag;
    a.timeout_ns = f.timeout_ns;
    const uint64_t C = (uint64_t)f.C;
    bool ok = make_map(&a.tmap[kMapDistD], a.dist, W, H, D, 1, kRQ, kRP, 1, true, Wp) &&
              make_map(&a.tmap[kMapDistH], a.dist, W, H, D, 1, kRQ, 1, kRP, true, Wp) &&
              make_map(&a.tmap[kMapDistW], a.distT, H, D, W, 1, kRQ, kRP, 1, true, Hp);
    if (tab) {
        // the intensity maps address the tables: nine arrays per axis
        const uint64_t pl = (uint64_t)D * H * Wp;
        float* tD = a.tables;
        float* tH = tD + kTabArrays * pl;
        float* tW = tH + kTabArrays * pl;
        ok = ok && make_map(&a.tmap[kMapImgD], tD, W, H, D, kTabArrays, kRQ, kRP, 1, false, Wp) &&
             make_map(&a.tmap[kMapImgH], tH, W, H, D, kTabArrays, kRQ, 1, kRP, false, Wp) &&
             make_map(&a.tmap[kMapImgW], tW, H, D, W, kTabArrays, kRQ, kRP, 1, false, Hp);
    } else if (img) {
        ok = ok && make_map(&a.tmap[kMapImgD], a.image, W, H, D, C, kRQ, kRP, 1, false, Wp) &&
             make_map(&a.tmap[kMapImgH], a.image, W, H, D, C, kRQ, 1, kRP, false, Wp) &&
             make_map(&a.tmap[kMapImgW], a.imageT, H, D, W, C, kRQ, kRP, 1, false, Hp);
    }
    if (!ok) return false;
    std::memcpy(desc, &a, sizeof(a));
    return true;
}

int vol3d_batched_geometry(int sms, int max_ci, int tables, const fgx_options* opt, int* grid,
                           size_t* smem) {
    *smem = stage_bytes(max_ci, tables ? 1 : 0);
    auto k = tables ? vol3d_batched_kernel<1> : vol3d_batched_kernel<0>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlockBatched3, *smem) !=
            cudaSuccess ||
        per_sm < 1)
        return FGX_ERR_CUDA;
    int64_t g = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) g = std::min<int64_t>(g, opt->max_blocks);
    *grid = (int)std::max<int64_t>(1, g);
    return FGX_OK;
}

int launch_vol3d_batched(const void* desc, int n, int rounds, const int* round_waves,
                         const int* wave_items, int grid, size_t smem, int tables, char* hdr,
                         unsigned int* barrier, long long timeout_ns, int sms, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const Vol3DArgs* d = (const Vol3DArgs*)desc;
    const dim3 per_inst((unsigned)std::max(1, sms * 4), (unsigned)n);
    init3d_batched_kernel<<<per_inst, 256, 0, s>>>(d);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if (rounds == 0) return FGX_OK;
    transpose_image3d_batched_kernel<<<per_inst, 256, 0, s>>>(d);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    if (tables) {
        cost_table3d_batched_kernel<1><<<per_inst, 256, 0, s>>>(d);
        cost_table3d_batched_kernel<2><<<per_inst, 256, 0, s>>>(d);
        cost_table3d_batched_kernel<3><<<per_inst, 256, 0, s>>>(d);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    Vol3DBatch bt;
    bt.desc = d;
    bt.n = n;
    bt.rounds = rounds;
    bt.round_waves = round_waves;
    bt.wave_items = wave_items;
    bt.barrier = barrier;
    bt.status = (int*)hdr;
    bt.timeout_ns = timeout_ns;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlockBatched3);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    auto k = tables ? vol3d_batched_kernel<1> : vol3d_batched_kernel<0>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    if (cudaLaunchKernelEx(&cfg, k, bt) != cudaSuccess) return FGX_ERR_CUDA;
    finish3d_batched_kernel<<<per_inst, 256, 0, s>>>(d);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
