// 2D reverse sweep (the adjoint of the raster scan of FastGeodis,
// Implementation section) on warp chains.
//
// The forward is a composition of min and + of edge costs, so along the
// recorded argmin parents it is differentiable.  For the pass applications in
// reverse order, and the lines of each in reverse sweep order, the adjoint of
// an element e of line l is
//   A[e] = G_in[e] + sum over k = 0, 1, 2 of A[x_k]  where child x_k (line
//          l+1 of the forward sweep, in-line offset 1-k) chose e (code k+1),
// in that order; the adjoint handed to the previous pass application is A[e]
// if e kept its value (code 0), else 0; after the first pass application
// dL/dM = v * that adjoint.  The image gradient of e collects, per pass
// application, -(A[x_k] lambda / c(x_k,e)) (I(x_k) - I(e)) for each child
// that chose e (offset order) and then +(A[e] lambda / c(e,p)) (I(e) - I(p))
// for its own parent p (terms with c = 0 are zero).
//
// Three kernels:
//  * a layout kernel writes the incoming adjoint and the parent codes of
//    every pass application in the line layout of that pass (rows for the
//    top-bottom / bottom-top passes, transposed for left-right / right-left,
//    rows padded to a multiple of four with zeros);
//  * the chain kernel propagates A line after line with the warp-chain tiles
//    of the forward (chain warp, producer warp, flusher warp; ring refresh
//    every K lines).  Per line only the A recurrence is on the chain: three
//    additions per column in the fixed order, where a child that did not
//    choose the element contributes -0.0 (x + -0.0 = x for every x, signed
//    zeros included), so the code has no branches.  It writes the masked
//    adjoint for the next pass application into one of two buffers per line
//    layout (never the buffer it reads: ring columns recompute from the
//    previous application's values, and sums are not idempotent) and, when
//    the image gradient is wanted, the unmasked A of every pass application;
//  * the gradient kernel runs one thread per element over the pass
//    applications in reverse order and adds the terms above in the order
//    given, from the stored A, the codes and the image.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "chain_common.cuh"
#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

using namespace dev;
using namespace chain;

constexpr int kRegionA = 128;            // columns per tile region (4 per lane)
constexpr int kBlockA = 96;              // chain, producer and flusher warps
constexpr int kChA = 8;                  // lines per chunk
constexpr int kNciA = 5;                 // chunks in the input ring
constexpr int kNoA = 3;                  // chunks in the output ring
constexpr int kOutLdA = kRegionA + 4;    // floats per output row
// The flusher waits for chunks on the input ring's barriers by phase parity:
// the chain, at most kNoA chunks ahead of it, must not complete two phases
// of one input slot in between.
static_assert(kNoA <= kNciA, "output ring deeper than the input ring");
constexpr int kTileA = 32;               // layout kernel tile
#define kNegZero __int_as_float(0x80000000)

struct Adj2DArgs {
    const float* grad_dist;   // [B][H][W]
    const uint8_t* codes;     // [T][B][H][W], image order
    float* grad_mask;         // [B][H][W] or null
    float* g0;                // [B][H][W] adjoint of D0 (image order), or null
    int B, H, W, Wp, Hp, T;
    float v;
    float* Gw[2];             // [B][H][Wp] adjoint in row layout (two buffers)
    float* Gt[2];             // [B][W][Hp] adjoint in column layout (two buffers)
    uint8_t* Cv;              // [T][B][H][Wp] codes of vertical pass applications
    uint8_t* Ch;              // [T][B][W][Hp] codes of horizontal pass applications
    float* Astore;            // [T][B][slab] A of every application (pass layout) or null
    int64_t slab;             // floats per (application, image) in Astore
    unsigned long long* xbuf; // [B][max_tiles][2 parity][2 side][kMaxRing]
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
    int K, Tw;                // ring and owned widths of multi-tile passes
    int tiles_v, tiles_h, max_tiles;
};

struct AdjSmem {
    unsigned long long in_full[kNciA], done[kNciA], out_empty[kNoA];
    unsigned long long pad_[2 - (2 * kNciA + kNoA) % 2];  // keeps the rings 16-byte aligned
    float g[kNciA][kChA][kRegionA];      // incoming adjoint per line
    unsigned int c[kNciA][kChA][32];     // code bytes per line, four per lane
    float outg[kNoA][kChA][kOutLdA];     // masked adjoint per line (next application)
    float outa[kNoA][kChA][kOutLdA];     // unmasked adjoint per line (gradient)
};

// Zero source for lanes outside the line (adjoint 0, code 0).
__device__ __align__(16) unsigned int g_zero4[4] = {0u, 0u, 0u, 0u};

__device__ __forceinline__ bool vertical(int t) { return (t & 3) < 2; }

// Layout kernel: one 32 x 32 tile of one image, for the incoming adjoint
// (j == T, in the layout of application T-1) or the codes of application j.
__global__ void __launch_bounds__(256) adj2d_layout_kernel(const Adj2DArgs a) {
    __shared__ float tf[kTileA][kTileA + 1];
    __shared__ uint8_t tb[kTileA][kTileA + 4];
    const int z = blockIdx.z;
    const int b = z / (a.T + 1), j = z % (a.T + 1);
    const int w0 = blockIdx.x * kTileA, h0 = blockIdx.y * kTileA;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t N = (int64_t)a.H * a.W;
    const bool is_g = j == a.T;
    const bool vert = vertical(is_g ? a.T - 1 : j);
    const float* gsrc = a.grad_dist + (int64_t)b * N;
    const uint8_t* csrc = is_g ? nullptr : a.codes + ((int64_t)j * a.B + b) * N;
    if (vert) {
        // rows [H][Wp], padding columns zero
        for (int i = ty; i < kTileA; i += 8) {
            const int h = h0 + i, w = w0 + tx;
            if (h >= a.H || w >= a.Wp) continue;
            const bool in = w < a.W;
            if (is_g)
                a.Gw[0][((int64_t)b * a.H + h) * a.Wp + w] = in ? gsrc[(int64_t)h * a.W + w] : 0.0f;
            else
                a.Cv[(((int64_t)j * a.B + b) * a.H + h) * a.Wp + w] =
                    in ? csrc[(int64_t)h * a.W + w] : (uint8_t)0;
        }
        return;
    }
    // columns [W][Hp] through a shared-memory transpose, padding rows zero
    for (int i = ty; i < kTileA; i += 8) {
        const int h = h0 + i, w = w0 + tx;
        const bool in = h < a.H && w < a.W;
        if (is_g) tf[i][tx] = in ? gsrc[(int64_t)h * a.W + w] : 0.0f;
        else tb[i][tx] = in ? csrc[(int64_t)h * a.W + w] : (uint8_t)0;
    }
    __syncthreads();
    for (int i = ty; i < kTileA; i += 8) {
        const int w = w0 + i, h = h0 + tx;
        if (w >= a.W || h >= a.Hp) continue;
        if (is_g)
            a.Gt[0][((int64_t)b * a.W + w) * a.Hp + h] = tf[tx][i];
        else
            a.Ch[(((int64_t)j * a.B + b) * a.W + w) * a.Hp + h] = tb[tx][i];
    }
}

// Geometry and buffers of one tile of one pass application.
struct AdjGeo {
    int L, Q, ld, ntiles, K, T, q0, q1, r0, nch;
    bool multi, fwdpass;
    const float* gsrc;         // incoming adjoint rows of this application (pass layout)
    const uint8_t* csrc;       // code rows of this application (pass layout)
    float* gdst;               // masked adjoint for the next application, or null
    int gdst_ld;
    bool gdst_transposed;
    float* gmask;              // first application: dL/dM = v * adjoint of this image
                               // (image order), else null
    float* g0;                 // first application: the adjoint itself (image order), or null
    float* adst;               // A of this application (pass layout), or null
};

__device__ __forceinline__ int line_of(const AdjGeo& g, int s) {
    // reverse sweep: the last line of the forward sweep comes first
    return g.fwdpass ? g.L - 1 - s : s;
}

// Producer warp: incoming adjoint and code rows of chunk c into ring slot
// (cb + c) % kNciA once the chain has finished the chunk that held it.
__device__ bool adj_producer(const Adj2DArgs& a, const AdjGeo& g, AdjSmem& sm, unsigned int cb) {
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    const bool lane_loads = (c0 >= 0) && (c0 < g.Q);
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = slot_of(gc, kNciA);
        if (gc >= (unsigned)kNciA &&
            !__all_sync(0xffffffffu, mbar_wait(&sm.done[slot], empty_parity(gc, kNciA), a.status,
                                               a.timeout_ns))) {
            cp_async_wait_all();
            return false;
        }
        const int jn = min(kChA, g.L - c * kChA);
        for (int j = 0; j < jn; ++j) {
            const int64_t off = (int64_t)line_of(g, c * kChA + j) * g.ld + c0;
            cp_async16(&sm.g[slot][j][4 * lane],
                       lane_loads ? (const void*)(g.gsrc + off) : (const void*)g_zero4);
            cp_async4(&sm.c[slot][j][lane],
                      lane_loads ? (const void*)(g.csrc + off) : (const void*)g_zero4);
        }
        cp_async_arrive_noinc(&sm.in_full[slot]);
    }
    return true;
}

// Flusher warp: writes the owned columns of each finished chunk: the masked
// adjoint (rows, or transposed when the next application runs along the
// other axis; v times it into dL/dM after the first application) and A.
// The chunk goes to registers first and its output slot is handed back
// before the global stores, so the chain never waits for them.
__device__ bool adj_flusher(const Adj2DArgs& a, const AdjGeo& g, AdjSmem& sm, unsigned int cb) {
    static_assert(kChA == 8, "transposed stores: 8 lines x 4 column groups per warp");
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    bool owned[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) owned[i] = (c0 + i >= g.q0) && (c0 + i < g.q1);
    // rows of the padded pass layouts start on 16 bytes (K and T are
    // multiples of 4), image-order rows need not
    const bool all_owned = owned[0] && owned[3];
    const int ncol = g.q1 - g.q0;
    const int off = g.q0 - g.r0;
    const bool rows_g = g.gdst && !g.gdst_transposed;
    const bool cols_g = g.gdst && g.gdst_transposed;
    // transposed: lane (jj, cg) writes line jj of columns cg, cg + 4, ...
    const int jj = lane & (kChA - 1);
    const int cg = lane >> 3;
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = slot_of(gc, kNoA);
        if (!__all_sync(0xffffffffu, mbar_wait(&sm.done[slot_of(gc, kNciA)],
                                               full_parity(gc, kNciA), a.status, a.timeout_ns)))
            return false;
        const int s0 = c * kChA;
        const int nl = min(kChA, g.L - s0);
        float4 va[kChA], vg[kChA];
#pragma unroll
        for (int j = 0; j < kChA; ++j) {
            va[j] = *reinterpret_cast<const float4*>(&sm.outa[slot][j][4 * lane]);
            vg[j] = *reinterpret_cast<const float4*>(&sm.outg[slot][j][4 * lane]);
        }
        float vt[kRegionA / 4];
        if (cols_g) {
#pragma unroll
            for (int k = 0; k < kRegionA / 4; ++k) {
                const int col = cg + 4 * k;
                vt[k] = col < ncol ? sm.outg[slot][jj][off + col] : 0.0f;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.out_empty[slot]);
#pragma unroll
        for (int j = 0; j < kChA; ++j) {
            if (j >= nl) break;
            const int64_t row = (int64_t)line_of(g, s0 + j);
            const float a4[4] = {va[j].x, va[j].y, va[j].z, va[j].w};
            const float g4[4] = {vg[j].x, vg[j].y, vg[j].z, vg[j].w};
            if (g.adst) {
                float* p = g.adst + row * g.ld + c0;
                if (all_owned) {
                    *reinterpret_cast<float4*>(p) = va[j];
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (owned[i]) p[i] = a4[i];
                }
            }
            if (rows_g) {
                float* p = g.gdst + row * g.gdst_ld + c0;
                if (all_owned) {
                    *reinterpret_cast<float4*>(p) = vg[j];
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (owned[i]) p[i] = g4[i];
                }
            }
            if (g.gmask || g.g0) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (!owned[i]) continue;
                    if (g.gmask) g.gmask[row * a.W + c0 + i] = __fmul_rn(a.v, g4[i]);
                    if (g.g0) g.g0[row * a.W + c0 + i] = g4[i];
                }
            }
        }
        if (cols_g && jj < nl) {
            float* p = g.gdst + (int64_t)g.q0 * g.gdst_ld + line_of(g, s0 + jj);
#pragma unroll
            for (int k = 0; k < kRegionA / 4; ++k) {
                const int col = cg + 4 * k;
                if (col < ncol) p[(int64_t)col * g.gdst_ld] = vt[k];
            }
        }
    }
    return true;
}

// One line of the A recurrence.  ap / cp: A and code bytes of the previous
// line of the reverse sweep (the children), gin / cc: incoming adjoint and
// code bytes of this line.
__device__ __forceinline__ void adj_step(float (&ap)[4], unsigned int& cp, const float4 gin,
                                         unsigned int cc, int lane, float* outa, float* outg) {
    // a child contributes to the parent it chose: to column j-1 with code 1,
    // j with code 2, j+1 with code 3; the lane's first and last columns feed
    // the neighbouring lanes
    const float up = ((cp & 0xffu) == 1u) ? ap[0] : kNegZero;
    const float dn = ((cp >> 24) == 3u) ? ap[3] : kNegZero;
    float from_next = __shfl_down_sync(0xffffffffu, up, 1);
    float from_prev = __shfl_up_sync(0xffffffffu, dn, 1);
    if (lane == 31) from_next = kNegZero;
    if (lane == 0) from_prev = kNegZero;
    const float g[4] = {gin.x, gin.y, gin.z, gin.w};
    float na[4], ng[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float t0 = (i < 3) ? ((((cp >> (8 * (i + 1))) & 0xffu) == 1u) ? ap[i + 1] : kNegZero)
                                 : from_next;
        const float t1 = (((cp >> (8 * i)) & 0xffu) == 2u) ? ap[i] : kNegZero;
        const float t2 = (i > 0) ? ((((cp >> (8 * (i - 1))) & 0xffu) == 3u) ? ap[i - 1] : kNegZero)
                                 : from_prev;
        na[i] = __fadd_rn(__fadd_rn(__fadd_rn(g[i], t0), t1), t2);
        ng[i] = ((cc >> (8 * i)) & 0xffu) != 0u ? 0.0f : na[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) ap[i] = na[i];
    cp = cc;
    *reinterpret_cast<float4*>(outa) = make_float4(na[0], na[1], na[2], na[3]);
    *reinterpret_cast<float4*>(outg) = make_float4(ng[0], ng[1], ng[2], ng[3]);
}

// Chain warp of one tile: chunks of kChA lines, fully unrolled, with the
// next line's inputs read one line ahead; ring refresh every K lines.
__device__ bool adj_chain(const Adj2DArgs& a, const AdjGeo& g, int seq, int b, int tile,
                          AdjSmem& sm, unsigned int cb) {
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    bool valid[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) valid[i] = (c0 + i >= 0) && (c0 + i < g.Q);
    const unsigned int tag_base = ((unsigned int)(seq + 1)) << 16;
    const RingLink link{a.xbuf + (size_t)b * a.max_tiles * (4 * kMaxRing), a.status, a.timeout_ns};
    float ap[4] = {kNegZero, kNegZero, kNegZero, kNegZero};
    unsigned int cp = 0;  // the first line of the reverse sweep has no children
    RingPos i0(cb, kNciA), i1 = i0.next(kNciA), i2 = i1.next(kNciA);
    RingPos o0(cb, kNoA), o1 = o0.next(kNoA);
    if (!__all_sync(0xffffffffu, mbar_wait(&sm.in_full[i0.slot], i0.par, a.status, a.timeout_ns)))
        return false;
    float4 gbuf[2];
    unsigned int cbuf[2];
    gbuf[0] = *reinterpret_cast<const float4*>(&sm.g[i0.slot][0][4 * lane]);
    cbuf[0] = sm.c[i0.slot][0][lane];
    int next_refresh = g.multi ? g.K : 0x7fffffff;
    int blk = 0;
    bool in_ready = g.nch < 2 || mbar_peek(&sm.in_full[i1.slot], i1.par);
    bool out_ready = cb < (unsigned)kNoA || mbar_peek(&sm.out_empty[o0.slot], o0.par ^ 1u);
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = i0.slot, nslot = i1.slot, oslot = o0.slot;
        if (!__all_sync(0xffffffffu, in_ready) &&
            !__all_sync(0xffffffffu, mbar_wait(&sm.in_full[nslot], i1.par, a.status, a.timeout_ns)))
            return false;
        if (!__all_sync(0xffffffffu, out_ready) &&
            !__all_sync(0xffffffffu,
                        mbar_wait(&sm.out_empty[oslot], o0.par ^ 1u, a.status, a.timeout_ns)))
            return false;
        in_ready = c + 2 >= g.nch || mbar_peek(&sm.in_full[i2.slot], i2.par);
        out_ready = gc + 1 < (unsigned)kNoA || mbar_peek(&sm.out_empty[o1.slot], o1.par ^ 1u);
        i0 = i1;
        i1 = i2;
        i2 = i2.next(kNciA);
        o0 = o1;
        o1 = o1.next(kNoA);
        if (c * kChA == next_refresh) {
            if (!ring_exchange(link, tile, g.ntiles, g.q0, g.K, g.T, c0,
                               tag_base | (unsigned int)(blk + 1), blk & 1, ap, valid, 0.0f))
                return false;
            next_refresh += g.K;
            ++blk;
        }
#pragma unroll
        for (int j = 0; j < kChA; ++j) {
            const int nj = j + 1;
            const int sl = nj < kChA ? slot : nslot;
            const int jl = nj < kChA ? nj : 0;
            gbuf[nj & 1] = *reinterpret_cast<const float4*>(&sm.g[sl][jl][4 * lane]);
            cbuf[nj & 1] = sm.c[sl][jl][lane];
            adj_step(ap, cp, gbuf[j & 1], cbuf[j & 1], lane, &sm.outa[oslot][j][4 * lane],
                     &sm.outg[oslot][j][4 * lane]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.done[slot]);
    }
    return true;
}

template <bool store_a>
__global__ void __launch_bounds__(kBlockA, 1) adj2d_kernel(const Adj2DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjSmem& sm = *reinterpret_cast<AdjSmem*>(smem_raw);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNciA; ++i) {
            mbar_init(&sm.in_full[i], 32);  // one asynchronous arrival per producer lane
            mbar_init(&sm.done[i], 1);
        }
        for (int i = 0; i < kNoA; ++i) mbar_init(&sm.out_empty[i], 1);
    }
    __syncthreads();
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[0] = (unsigned long long)gtimer();
    unsigned int epoch = 1;
    unsigned int cb = 0;  // chunks handed over so far in this block
    const int warp = threadIdx.x >> 5;
    // the incoming adjoint of an application lives in one of two buffers of
    // its line layout
    bool in_vert = vertical(a.T - 1);
    int in_idx = 0;
    bool alive = true;
    for (int t = a.T - 1; t >= 0 && alive; --t) {
        const int pass = t & 3;
        const bool vert = pass < 2;
        const bool out_vert = t > 0 ? vertical(t - 1) : true;
        const int out_idx = (out_vert == in_vert) ? 1 - in_idx : 0;
        const int ntiles = vert ? a.tiles_v : a.tiles_h;
        const int L = vert ? a.H : a.W;
        const int nch = (L + kChA - 1) / kChA;
        const int per_wave = gridDim.x / ntiles;
        const int nwaves = (a.B + per_wave - 1) / per_wave;
        bool ok = true;
        for (int wv = 0; wv < nwaves && ok; ++wv) {
            if ((int)blockIdx.x >= per_wave * ntiles) continue;
            const int b = wv * per_wave + blockIdx.x / ntiles;
            if (b >= a.B) continue;
            const int tile = blockIdx.x % ntiles;
            AdjGeo g;
            g.L = L;
            g.Q = vert ? a.W : a.H;
            g.ld = vert ? a.Wp : a.Hp;
            g.ntiles = ntiles;
            g.multi = ntiles > 1;
            g.K = g.multi ? a.K : 0;
            g.T = g.multi ? a.Tw : g.Q;
            g.q0 = g.multi ? tile * g.T : 0;
            g.q1 = min(g.Q, g.q0 + g.T);
            g.r0 = g.q0 - g.K;
            g.nch = nch;
            g.fwdpass = pass == 0 || pass == 2;
            const int64_t plane = (int64_t)L * g.ld;
            g.gsrc = (in_vert ? a.Gw[in_idx] : a.Gt[in_idx]) + (int64_t)b * plane;
            g.csrc = (vert ? a.Cv : a.Ch) + ((int64_t)t * a.B + b) * plane;
            g.gmask = (t == 0 && a.grad_mask) ? a.grad_mask + (int64_t)b * a.H * a.W : nullptr;
            g.g0 = (t == 0 && a.g0) ? a.g0 + (int64_t)b * a.H * a.W : nullptr;
            g.gdst = nullptr;
            g.gdst_ld = 0;
            g.gdst_transposed = false;
            if (t > 0) {
                g.gdst = out_vert ? a.Gw[out_idx] + (int64_t)b * a.H * a.Wp
                                  : a.Gt[out_idx] + (int64_t)b * a.W * a.Hp;
                g.gdst_ld = out_vert ? a.Wp : a.Hp;
                g.gdst_transposed = out_vert != vert;
            }
            g.adst = store_a ? a.Astore + ((int64_t)t * a.B + b) * a.slab : nullptr;
            if (warp == 0) ok = adj_chain(a, g, a.T - 1 - t, b, tile, sm, cb);
            else if (warp == 1) ok = adj_producer(a, g, sm, cb);
            else ok = adj_flusher(a, g, sm, cb);
            cb += (unsigned int)nch;
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        in_vert = out_vert;
        in_idx = out_idx;
        if (blockIdx.x == 0 && threadIdx.x == 0 && a.T - t < 16)
            timeline[a.T - t] = (unsigned long long)gtimer();
    }
}

struct Grad2DArgs {
    const float* image;       // [B][C][H][W]
    const uint8_t* codes;     // [T][B][H][W]
    const float* Astore;      // [T][B][slab], pass layout
    float* grad_image;        // [B][C][H][W], or null
    float* lambda_terms;      // [B][H][W] per-element terms of dL/dlambda, or null
    int64_t slab;
    int B, C, H, W, Wp, Hp, T;
    float lambda;
    float tv[3], th[3];       // (1 - lambda) |offset|^2 of vertical / horizontal passes
    float sv[3], sh[3];       // |offset|^2 of vertical / horizontal passes
};

// Edge cost between image elements x and y, channel stride n, in the fixed
// order of the method: di2 = sum_ch (I(x)-I(y))^2, c = sqrt(t + lambda*di2).
__device__ __forceinline__ float grad_cost(const float* img, int64_t x, int64_t y, int C,
                                           int64_t n, float t, float lam, float* di2_out = nullptr) {
    float di2 = 0.0f;
    for (int ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(img[ch * n + x], img[ch * n + y]);
        di2 = __fadd_rn(di2, __fmul_rn(d, d));
    }
    if (di2_out) *di2_out = di2;
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// d c / d lambda of an edge (c^2 = (1 - lambda) s2 + lambda di2) times the
// child's adjoint, in the fixed order (di2 - s2) / (c + c), then the product.
__device__ __forceinline__ float lambda_term(float A, float di2, float s2, float c) {
    return __fmul_rn(A, __fdiv_rn(__fsub_rn(di2, s2), __fadd_rn(c, c)));
}

// Image gradient, one thread per element, pass applications in reverse
// order; CC > 0 keeps CC channels in registers, CC == 0 accumulates in the
// output array (each element is touched by its own thread only).
template <int CC, bool IMG>
__global__ void __launch_bounds__(256) grad2d_kernel(const Grad2DArgs a) {
    const int64_t N = (int64_t)a.H * a.W;
    const int C = CC > 0 ? CC : a.C;
    const float lam = a.lambda;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.B * N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / N);
        const int64_t e = i - (int64_t)b * N;
        const int h = (int)(e / a.W), w = (int)(e - (int64_t)h * a.W);
        const float* img = a.image + (int64_t)b * a.C * N;
        float* gout = IMG ? a.grad_image + (int64_t)b * a.C * N + e : nullptr;
        float lt = 0.0f;  // this element's terms of dL/dlambda
        float gi[CC > 0 ? CC : 1];
        if (CC > 0) {
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gi[ch] = 0.0f;
        } else if (IMG) {
            for (int ch = 0; ch < C; ++ch) gout[ch * N] = 0.0f;
        }
        auto add_term = [&](float wgt, int64_t x, int64_t y, bool minus) {
            // g -= wgt (I(x) - I(y))  or  g += wgt (I(x) - I(y)), per channel
            if (CC > 0) {
#pragma unroll
                for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) {
                    const float term = __fmul_rn(wgt, __fsub_rn(img[ch * N + x], img[ch * N + y]));
                    gi[ch] = minus ? __fsub_rn(gi[ch], term) : __fadd_rn(gi[ch], term);
                }
            } else {
                for (int ch = 0; ch < C; ++ch) {
                    const float term = __fmul_rn(wgt, __fsub_rn(img[ch * N + x], img[ch * N + y]));
                    gout[ch * N] = minus ? __fsub_rn(gout[ch * N], term)
                                         : __fadd_rn(gout[ch * N], term);
                }
            }
        };
        for (int t = a.T - 1; t >= 0; --t) {
            const int pass = t & 3;
            const bool vert = pass < 2;
            const int dir = (pass == 0 || pass == 2) ? 1 : -1;
            const int L = vert ? a.H : a.W, Q = vert ? a.W : a.H;
            const int line = vert ? h : w, q = vert ? w : h;
            const int ld = vert ? a.Wp : a.Hp;
            const float* A = a.Astore + ((int64_t)t * a.B + b) * a.slab;
            const uint8_t* cd = a.codes + ((int64_t)t * a.B + b) * N;
            const float* tk = vert ? a.tv : a.th;
            auto at = [&](int ln, int qq) -> int64_t {
                return vert ? (int64_t)ln * a.W + qq : (int64_t)qq * a.W + ln;
            };
            // children on the next line of the forward sweep, offset order:
            // the offsets whose child chose this element are collected first,
            // then visited in increasing order, so that a warp evaluates one
            // cost per step for all its lanes instead of one per offset any
            // lane needs
            const int cl = line + dir;
            if (IMG && cl >= 0 && cl < L) {
                unsigned int chose = 0u;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const int cq = q + 1 - k;
                    if (cq >= 0 && cq < Q && cd[at(cl, cq)] == k + 1) chose |= 1u << k;
                }
                while (chose) {
                    const int k = __ffs(chose) - 1;
                    chose &= chose - 1u;
                    const int cq = q + 1 - k;
                    const int64_t x = at(cl, cq);
                    const float c = grad_cost(img, x, e, C, N, tk[k], lam);
                    if (c > 0.0f) {
                        const float wgt =
                            __fdiv_rn(__fmul_rn(A[(int64_t)cl * ld + cq], lam), c);
                        add_term(wgt, x, e, true);
                    }
                }
            }
            // own parent on the previous line of the forward sweep
            const int code = cd[e];
            const int pl = line - dir, pq = q + code - 2;
            // (codes outside 1..3 or pointing outside the line are ignored)
            if (code >= 1 && code <= 3 && pl >= 0 && pl < L && pq >= 0 && pq < Q) {
                const int64_t p = at(pl, pq);
                float di2;
                const float c = grad_cost(img, e, p, C, N, tk[code - 1], lam, &di2);
                if (c > 0.0f) {
                    const float Ae = A[(int64_t)line * ld + q];
                    if (a.lambda_terms)
                        lt = __fadd_rn(lt, lambda_term(Ae, di2, (vert ? a.sv : a.sh)[code - 1], c));
                    if (IMG) add_term(__fdiv_rn(__fmul_rn(Ae, lam), c), e, p, false);
                }
            }
        }
        if (CC > 0 && IMG) {
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch) gout[ch * N] = gi[ch];
        }
        if (a.lambda_terms) a.lambda_terms[i] = lt;
    }
}

struct Adj2DLayout {
    int K, Tw, tv, th, max_tiles, Wp, Hp;
    int64_t slab;
    size_t xbuf_off, gw_off[2], gt_off[2], cv_off, ch_off, a_off, total;
};

size_t al256a(size_t x) { return (x + 255) & ~size_t(255); }

Adj2DLayout adj2d_layout(int64_t B, int64_t H, int64_t W, int T, const fgx_options* opt) {
    Adj2DLayout l;
    chain2d_geometry(H, W, opt, &l.K, &l.Tw, &l.tv, &l.th);
    l.max_tiles = std::max(l.tv, l.th);
    l.Wp = (int)((W + 3) & ~int64_t(3));
    l.Hp = (int)((H + 3) & ~int64_t(3));
    l.slab = std::max<int64_t>(H * l.Wp, W * l.Hp);
    size_t off = kHeaderBytes;
    l.xbuf_off = off;
    off += al256a((size_t)B * l.max_tiles * 4 * kMaxRing * 8);
    for (int i = 0; i < 2; ++i) {
        l.gw_off[i] = off;
        off += al256a((size_t)B * H * l.Wp * 4);
    }
    for (int i = 0; i < 2; ++i) {
        l.gt_off[i] = off;
        off += al256a((size_t)B * W * l.Hp * 4);
    }
    l.cv_off = off;
    off += al256a((size_t)T * B * H * l.Wp);
    l.ch_off = off;
    off += al256a((size_t)T * B * W * l.Hp);
    l.a_off = off;
    off += al256a((size_t)T * B * l.slab * 4);
    l.total = off;
    return l;
}

}  // namespace

size_t adj2d_workspace_bytes(int64_t B, int64_t H, int64_t W, int iterations,
                             const fgx_options* opt) {
    return adj2d_layout(B, H, W, iterations * 4, opt).total;
}

int run_adj2d(const float* grad_dist, const float* image, const uint8_t* codes,
              float* grad_image, float* grad_mask, int64_t B, int64_t C, int64_t H, int64_t W,
              float v, float lambda, int iterations, void* workspace, size_t ws_bytes,
              const fgx_options* opt, int sms, void* stream, float* g0, float* lambda_terms) {
    const int T = iterations * 4;
    if (T <= 0 || B * (T + 1) > 65535) return FGX_ERR_UNSUPPORTED;
    const Adj2DLayout l = adj2d_layout(B, H, W, T, opt);
    if (ws_bytes < l.total) return FGX_ERR_WORKSPACE;
    char* w = (char*)workspace;
    Adj2DArgs a;
    std::memset(&a, 0, sizeof(a));
    a.grad_dist = grad_dist;
    a.codes = codes;
    a.grad_mask = grad_mask;
    a.g0 = g0;
    a.B = (int)B;
    a.H = (int)H;
    a.W = (int)W;
    a.Wp = l.Wp;
    a.Hp = l.Hp;
    a.T = T;
    a.v = v;
    for (int i = 0; i < 2; ++i) {
        a.Gw[i] = (float*)(w + l.gw_off[i]);
        a.Gt[i] = (float*)(w + l.gt_off[i]);
    }
    a.Cv = (uint8_t*)(w + l.cv_off);
    a.Ch = (uint8_t*)(w + l.ch_off);
    const bool need_a = grad_image || lambda_terms;  // the per-element pass needs every A
    a.Astore = need_a ? (float*)(w + l.a_off) : nullptr;
    a.slab = l.slab;
    a.xbuf = (unsigned long long*)(w + l.xbuf_off);
    a.barrier = (unsigned int*)(w + 64);
    a.status = (int*)w;
    a.timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) * 1000000LL;
    a.K = l.K;
    a.Tw = l.Tw;
    a.tiles_v = l.tv;
    a.tiles_h = l.th;
    a.max_tiles = l.max_tiles;

    auto kernel = need_a ? adj2d_kernel<true> : adj2d_kernel<false>;
    const size_t smem = sizeof(AdjSmem);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlockA, smem) !=
            cudaSuccess ||
        per_sm < 1)
        return FGX_ERR_CUDA;
    int64_t grid = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, B * l.max_tiles));
    if (grid < l.max_tiles) return FGX_ERR_UNSUPPORTED;

    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, l.gw_off[0], s) != cudaSuccess) return FGX_ERR_CUDA;
    const dim3 lg((unsigned)((l.Wp + kTileA - 1) / kTileA), (unsigned)((l.Hp + kTileA - 1) / kTileA),
                  (unsigned)(B * (T + 1)));
    adj2d_layout_kernel<<<lg, dim3(32, 8), 0, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlockA);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    if (need_a) {
        Grad2DArgs g;
        std::memset(&g, 0, sizeof(g));
        g.image = image;
        g.codes = codes;
        g.Astore = a.Astore;
        g.grad_image = grad_image;
        g.lambda_terms = lambda_terms;
        g.slab = l.slab;
        g.B = (int)B;
        g.C = (int)C;
        g.H = (int)H;
        g.W = (int)W;
        g.Wp = l.Wp;
        g.Hp = l.Hp;
        g.T = T;
        g.lambda = lambda;
        const float unit[3] = {1.f, 1.f, 1.f};
        float t9[9];
        pass_offsets_t(2, 1, unit, lambda, t9);  // pass along H: offsets along W
        for (int k = 0; k < 3; ++k) g.tv[k] = t9[k];
        pass_offsets_t(2, 2, unit, lambda, t9);  // pass along W: offsets along H
        for (int k = 0; k < 3; ++k) g.th[k] = t9[k];
        pass_offsets_t(2, 1, unit, 0.0f, t9);    // (1 - 0) |offset|^2
        for (int k = 0; k < 3; ++k) g.sv[k] = t9[k];
        pass_offsets_t(2, 2, unit, 0.0f, t9);
        for (int k = 0; k < 3; ++k) g.sh[k] = t9[k];
        const int64_t n = B * H * W;
        const int gg = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
        if (grad_image) {
            if (C == 1) grad2d_kernel<1, true><<<gg, 256, 0, s>>>(g);
            else if (C == 2) grad2d_kernel<2, true><<<gg, 256, 0, s>>>(g);
            else if (C == 3) grad2d_kernel<3, true><<<gg, 256, 0, s>>>(g);
            else if (C == 4) grad2d_kernel<4, true><<<gg, 256, 0, s>>>(g);
            else grad2d_kernel<0, true><<<gg, 256, 0, s>>>(g);
        } else {
            grad2d_kernel<0, false><<<gg, 256, 0, s>>>(g);
        }
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

}  // namespace fgx
