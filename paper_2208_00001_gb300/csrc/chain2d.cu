// 2D forward on warp chains (FastGeodis, Implementation section: four passes
// per iteration, each row or column updated from the already-updated previous
// one).
//
// Layout and schedule.  The distance map lives in two padded workspace copies:
// Dw [H][Wp] (rows contiguous) for the top-bottom / bottom-top passes and
// Dt [W][Hp] (columns contiguous) for the left-right / right-left passes, so
// every pass streams contiguous rows.  Bottom-top writes its result straight
// into Dt and right-left straight back into Dw (or into the caller's output in
// the last iteration) through a shared-memory transpose, so no separate
// transpose phase exists.  Edge costs do not depend on D: a first phase
// evaluates the cost of every undirected grid edge once per call (the cost is
// symmetric and the same in every pass and iteration) into two tables,
// Ev[3][H][Wp] for the edges between rows h and h+1 and Eh[3][W][Hp] for the
// edges between columns w and w+1.  With lambda = 0 the costs are the
// constants sqrt(t_k) and no table is built.
//
// Work decomposition.  One cooperative persistent launch; each thread block
// owns a tile of T columns of one line plus a ring of K columns on each side
// (T + 2K = 128, four columns per lane of the chain warp).  Three warps per
// block: the chain warp applies the min-plus update line after line, getting
// the two neighbouring columns across lanes by shuffle; a producer warp
// copies old values and edge costs into a shared-memory ring of 8-line
// chunks ahead of it; a flusher warp writes finished chunks out.  The
// dependency cone shrinks the valid part of the ring by one column per line,
// so after K lines the owned columns are exact; every K lines (a whole number
// of chunks) the chain warp publishes the 2K owned columns its neighbours
// need as 64-bit words (value, tag) and polls the neighbours' words until the
// tags match (bounded wait); the ring is then refreshed.  Passes are
// separated by a grid barrier.
#include <cuda.h>  // CUtensorMap and its encoder's signature (the encoder is looked up at run time)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "chain_common.cuh"
#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {

namespace {

constexpr int kRegion = 128;           // columns per tile region (4 per lane)
constexpr int kMaxSeg = 8;             // speculative segments per pass at most
constexpr int kMinSegLines = 256;      // shortest segment worth a separate chain
constexpr int kMaxSegImages = 128;     // images of one call that segments are used for
constexpr int kMaxCk = 64;             // checkpoints of one re-run at most
constexpr int kBlockThreads = 96;      // chain, producer and flusher warps
#define kInf __int_as_float(0x7f800000)

struct Chain2DArgs {
    const float* image;  // [B][C][H][W]
    const float* mask;   // [B][H][W]
    float* dist;         // [B][H][W]
    uint8_t* codes;      // [iterations * 4][B][H][W] parent codes, or null
    int B, C, H, W, Wp, Hp;
    int nimg;            // distinct images: instance b reads image b % nimg
    float v, lambda;
    int iterations;
    int table;           // 1: cost tables, 0: constant costs (lambda = 0)
    int fast;            // tables with fused multiply-adds and the approximate root
    float tv[3], th[3];  // (1 - lambda) * s2 of the row-edge and column-edge offsets
    float cv[3], chh[3]; // sqrt of the above (constant-cost mode)
    float* Dw;           // [B][H][Wp]
    float* Dt;           // [B][W][Hp]
    float* Ev;           // [B][3][H][Wp]
    float* Eh;           // [B][3][W][Hp]
    unsigned long long* xbuf;  // [B][max_tiles][2 parity][2 side][kMaxRing]
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
    int K, T;            // ring and owned widths of multi-tile passes
    int tiles_v, tiles_h;
    int max_tiles;
    // speculative line segments (1: a pass runs as one chain)
    int nseg_v, nseg_h;      // segments of a vertical / horizontal pass
    int seglen_v, seglen_h;  // lines per segment (whole chunks)
    int max_seg;             // exchange areas per image (kMaxSeg, or 1)
    int bnd_ld;              // floats per boundary line (max(H, W) rounded up)
    float* bnd;              // [B][kMaxSeg - 1][bnd_ld] boundary lines the segments started from
    unsigned int* segflag;   // [B][kMaxSeg][2]: boundary changed (phase A, re-run), tag t_app + 1;
                             // then [4]: 1 + the last application of each pass with re-runs
    unsigned int* ckpt;      // [B][kMaxSeg][kMaxCk]: re-run checkpoints (arrivals | changed << 16)
    // tensor maps of the single-call launch (box: the 128 region columns of a
    // chunk of kCh lines): Dw, Dt, Ev, Eh; tma = 0: per-lane copies instead
    CUtensorMap tmap[4];
    int tma;
};

using namespace dev;
using namespace chain;
// Cost of the undirected edge between a and b (same channel stride n), in the
// fixed arithmetic order: di2 = sum_ch (I(a)-I(b))^2, c = sqrt(t + lambda*di2).
__device__ __forceinline__ float edge_cost(const float* ia, const float* ib, int C, int64_t n,
                                           float t, float lam, bool fast) {
    float di2 = 0.0f;
    for (int ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(__ldg(ia + ch * n), __ldg(ib + ch * n));
        di2 = fast ? __fmaf_rn(d, d, di2) : __fadd_rn(di2, __fmul_rn(d, d));
    }
    return fast ? fast_sqrt(__fmaf_rn(lam, di2, t)) : __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

// Producer/consumer organisation of one tile, three warps.  The chain warp
// holds four columns per lane in registers and applies the min-plus update
// in fully unrolled chunks of kCh lines; the producer warp copies the rows of
// old distances and edge costs into a ring of chunks ahead of it (cp.async,
// completion tracked by one mbarrier per chunk); the flusher warp writes the
// finished chunks to global memory, transposed where the pass requires.
// Waits, ring exchanges and hand-overs happen only between chunks, so the
// per-line code has no branches.
constexpr int kCh = 16;             // lines per chunk (staging and hand-over unit)
constexpr int kSub = 8;             // ring refreshes fall on multiples of kSub lines
constexpr int kNci = 4;             // chunks in the input ring
constexpr int kNo = 3;              // chunks in the output ring
constexpr int kRow = kRegion + 8;   // floats per input row: 4 pad | 128 | 4 pad
constexpr int kOutLd = kRegion + 4; // floats per output row (conflict-free transposes)
// The flusher waits for chunks on the input ring's barriers by phase parity:
// the chain, at most kNo chunks ahead of it, must not complete two phases of
// one input slot in between.
static_assert(kNo <= kNci, "output ring deeper than the input ring");

struct TileSmem {
    // in_full: the producer's copies of a chunk have landed; done: the chain
    // has finished a chunk (its input slot is free, its output is ready);
    // out_empty: the flusher has written an output slot out
    unsigned long long in_full[kNci], done[kNci], out_empty[kNo];
    unsigned long long pad_[2 - (2 * kNci + kNo) % 2];  // keeps the rings 16-byte aligned
    int stop_chunk;                 // a re-run stopped early: chunks from here are skipped
    int pad2_[3];
    float in[kNci][kCh][4][kRow];   // per line: old values, edge rows E0, E1, E2
    float out[kNo][kCh][kOutLd];    // chain results per line
    uint8_t outc[kNo][kCh][kRegion];  // parent codes per line (when recorded)
};

// Source of the +inf rows copied into the ring for lanes outside the array.
__device__ __align__(16) unsigned int g_inf_row[4] = {0x7f800000u, 0x7f800000u, 0x7f800000u,
                                                      0x7f800000u};

__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned int parity,
                                          const Chain2DArgs& a) {
    return chain::mbar_wait(b, parity, a.status, a.timeout_ns);
}

// Geometry of one tile of one pass (or of one line segment of it), identical
// in the three warps.
struct TileGeo {
    int L, Q, ld, ntiles, K, T, q0, q1, r0, nch;
    int s0, ns;      // first step and number of steps of the segment
    bool multi;
    const float* src;
    const float* E;
    int64_t eplane;
    float* out;
    int out_ld;
    uint8_t* codes;  // codes of this pass application and image (image order), or null
    bool codes_rows; // the pass's lines are rows of the image (vertical pass)
    unsigned long long* xb;  // exchange area of this image and segment
    unsigned int tag_base;
    const float* bline;      // values of the line before step s0 (element q at q * bstride), or null
    int bstride;
    const float* cmp;        // line the next segment started from (element q at q), or null
    unsigned int* flag;      // set to flag_tag when the last line differs from it
    const unsigned int* flag_first;  // the flag the first run set (a re-run that stops early
                                     // keeps the first run's last line)
    unsigned int flag_tag;
    unsigned int* ck;        // re-run checkpoints of this image and segment, or null
    int ck_every;            // chunks between checkpoints
};

// Line of step s of a pass in sweep order.
__device__ __forceinline__ int line_of(bool fwd, int L, int s) { return fwd ? s : L - 1 - s; }

// Segment `seg` of the pass (seg = 0 with one segment: the whole pass);
// rerun: the segment runs again from the exact line before it.
__device__ __forceinline__ TileGeo tile_geo(const Chain2DArgs& a, int t_app, int pass, int b,
                                            int tile, int seg = 0, bool rerun = false,
                                            int nseg = 1) {
    TileGeo g;
    const bool vert = pass < 2;  // rows of Dw (TB/BT) or rows of Dt (LR/RL)
    g.L = vert ? a.H : a.W;
    g.Q = vert ? a.W : a.H;
    g.ld = vert ? a.Wp : a.Hp;
    g.ntiles = vert ? a.tiles_v : a.tiles_h;
    g.multi = g.ntiles > 1;
    g.K = g.multi ? a.K : 0;
    g.T = g.multi ? a.T : g.Q;
    g.q0 = g.multi ? tile * g.T : 0;
    g.q1 = min(g.Q, g.q0 + g.T);
    g.r0 = g.q0 - g.K;
    g.src = vert ? a.Dw + (int64_t)b * a.H * a.Wp : a.Dt + (int64_t)b * a.W * a.Hp;
    g.E = vert ? a.Ev + (int64_t)b * 3 * a.H * a.Wp : a.Eh + (int64_t)b * 3 * a.W * a.Hp;
    g.eplane = (int64_t)g.L * g.ld;
    const bool last_rl = (pass == 3) && (t_app == a.iterations * 4 - 1);
    if (pass == 0) { g.out = a.Dw + (int64_t)b * a.H * a.Wp; g.out_ld = a.Wp; }
    else if (pass == 1) { g.out = a.Dt + (int64_t)b * a.W * a.Hp; g.out_ld = a.Hp; }
    else if (pass == 2) { g.out = a.Dt + (int64_t)b * a.W * a.Hp; g.out_ld = a.Hp; }
    else if (last_rl) { g.out = a.dist + (int64_t)b * a.H * a.W; g.out_ld = a.W; }
    else { g.out = a.Dw + (int64_t)b * a.H * a.Wp; g.out_ld = a.Wp; }
    g.codes = a.codes ? a.codes + ((int64_t)t_app * a.B + b) * a.H * a.W : nullptr;
    g.codes_rows = vert;
    const int seglen = nseg > 1 ? (vert ? a.seglen_v : a.seglen_h) : g.L;
    g.s0 = seg * seglen;
    g.ns = min(seglen, g.L - g.s0);
    g.nch = (g.ns + kCh - 1) / kCh;
    g.xb = a.xbuf + ((size_t)b * a.max_seg + seg) * a.max_tiles * (4 * kMaxRing);
    // tags differ between pass applications and between a segment's first
    // run and its re-run (both use the same exchange area)
    g.tag_base = ((unsigned int)(2 * t_app + (rerun ? 2 : 1))) << 16;
    g.bline = nullptr;
    g.bstride = 1;
    g.cmp = nullptr;
    g.flag = nullptr;
    g.flag_first = nullptr;
    g.flag_tag = (unsigned int)(t_app + 1);
    g.ck = nullptr;
    g.ck_every = 1;
    if (seg > 0) {
        if (rerun) {
            // the exact line before the segment, as the pass wrote it
            const int line = line_of(pass == 0 || pass == 2, g.L, g.s0 - 1);
            const bool fwd = pass == 0 || pass == 2;
            g.bline = fwd ? g.out + (int64_t)line * g.out_ld : g.out + line;
            g.bstride = fwd ? 1 : g.out_ld;
        } else {
            g.bline = a.bnd + ((int64_t)b * (kMaxSeg - 1) + seg - 1) * a.bnd_ld;
        }
    }
    if (seg + 1 < nseg) {
        g.cmp = a.bnd + ((int64_t)b * (kMaxSeg - 1) + seg) * a.bnd_ld;
        unsigned int* f = a.segflag + ((int64_t)b * kMaxSeg + seg + 1) * 2;
        g.flag = f + (rerun ? 1 : 0);
        g.flag_first = f;
    }
    // a re-run can stop early where the first run's values are its old
    // values: in the passes that update their lines in place
    const bool fwd = pass == 0 || pass == 2;
    if (seg > 0 && rerun && fwd) {
        g.ck = a.ckpt + ((int64_t)b * kMaxSeg + seg) * kMaxCk;
        const int base = g.multi ? max(1, g.K / kCh) : 3;
        const int npts = (g.nch + base - 1) / base;
        g.ck_every = base * ((npts + kMaxCk - 2) / (kMaxCk - 1));
    }
    return g;
}

// Input ring layouts.  Per-lane copies fill in[slot][line][array][4 + column]
// (padded rows, +inf padding); tensor copies fill dense boxes of the region
// columns of a chunk, [slot][array][row][column], starting at the first
// 128-byte boundary of the ring, rows in increasing line order (row
// kCh-1-j holds step j of a backward pass).  A row pointer points at region
// column 0; the chain also reads one element before it and one after the
// 128 columns (the edge lanes' neighbouring costs, whose parents are +inf).
__device__ __forceinline__ const float* tma_ring(const TileSmem& sm) {
    const unsigned int a0 = saddr(&sm.in[0][0][0][0]);
    return &sm.in[0][0][0][0] + (((128u - (a0 & 127u)) & 127u) >> 2);
}
template <bool TMA, bool fwd>
__device__ __forceinline__ const float* ring_row(const TileSmem& sm, const float* tbase, int slot,
                                                 int j, int arr) {
    if (!TMA) return &sm.in[slot][j][arr][4];
    return tbase + ((slot * 4 + arr) * kCh + (fwd ? j : kCh - 1 - j)) * kRegion;
}

// Producer with tensor copies (one elected thread): chunk c of the tile is
// one box of kCh lines x 128 region columns per array (distances, then the
// three edge-cost rows), issued once the chain has released the slot and
// completed on the slot's mbarrier by transaction count.  Outside the array
// the copies fill NaN, which never wins a min (like the +inf of the padding).
// The edge rows of a forward step s are rows s-1 of the table, of a backward
// step its own line; the first line of a sweep has no parents and reads the
// fill.  After a failed wait the copies in flight are waited for (bounded)
// before returning.
template <bool fwd, bool table>
__device__ bool producer_tma(const Chain2DArgs& a, const TileGeo& g, TileSmem& sm,
                             unsigned int cb, int b, bool vert) {
    if ((threadIdx.x & 31) != 0) return true;
    const float* tbase = tma_ring(sm);
    const CUtensorMap* md = &a.tmap[vert ? 0 : 1];
    const CUtensorMap* me = &a.tmap[vert ? 2 : 3];
    const unsigned int bytes = (unsigned int)((table ? 4 : 1) * kCh * kRegion * 4);
    bool ok = true;
    int issued = 0;
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = slot_of(gc, kNci);
        if (gc >= (unsigned)kNci && !mbar_wait(&sm.done[slot], empty_parity(gc, kNci), a)) {
            ok = false;
            break;
        }
        if (c >= *(volatile int*)&sm.stop_chunk) {
            // a re-run that stopped early: the chunk is only handed over
            mbar_arrive(&sm.in_full[slot]);
            continue;
        }
        const int s = g.s0 + c * kCh;
        const int y = fwd ? s : g.L - kCh - s;  // first line of the box
        mbar_expect_tx(&sm.in_full[slot], bytes);
        tma_load3(ring_row<true, true>(sm, tbase, slot, 0, 0), md, g.r0, y, b, &sm.in_full[slot]);
        if (table) {
            const int ye = fwd ? s - 1 : y;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                tma_load3(ring_row<true, true>(sm, tbase, slot, 0, 1 + k), me, g.r0, ye, 3 * b + k,
                          &sm.in_full[slot]);
        }
        issued = c + 1;
    }
    if (!ok) {
        // let this block's copies land before the shared memory is reused
        for (int c = max(0, issued - kNci); c < issued; ++c) {
            const unsigned int gc = cb + c;
            const long long t0 = gtimer();
            while (!mbar_test(&sm.in_full[slot_of(gc, kNci)], full_parity(gc, kNci)) &&
                   gtimer() - t0 <= a.timeout_ns) {
            }
        }
    }
    return ok;
}

// Producer warp: chunk c of the tile goes to ring slot (cb + c) % kNci once
// the chain has released that slot.  The edge row between steps s-1 and s is
// row s-1 of the table in a forward pass and row L-1-s in a backward one;
// the first line of a sweep has no parents and gets no edge row.
template <bool fwd, bool table>
__device__ bool producer_tile(const Chain2DArgs& a, const TileGeo& g, TileSmem& sm,
                              unsigned int cb) {
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    const bool lane_loads = (c0 >= 0) && (c0 < g.Q);
    const int L = g.L;
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = slot_of(gc, kNci);
        if (gc >= (unsigned)kNci &&
            !__all_sync(0xffffffffu, mbar_wait(&sm.done[slot], empty_parity(gc, kNci), a))) {
            cp_async_wait_all();
            return false;
        }
        if (c >= *(volatile int*)&sm.stop_chunk) {
            // a re-run that stopped early: the chunk is only handed over
            mbar_arrive(&sm.in_full[slot]);
            continue;
        }
        const int jn = min(kCh, g.ns - c * kCh);
        for (int j = 0; j < jn; ++j) {
            const int s = g.s0 + c * kCh + j;
            const int line = fwd ? s : (L - 1 - s);
            float(*row)[kRow] = sm.in[slot][j];
            // lanes outside the array get +inf rows: their columns stay at
            // +inf and cost nothing to the columns next to them
            cp_async16(&row[0][4 + 4 * lane],
                       lane_loads ? (const void*)(g.src + (int64_t)line * g.ld + c0) : g_inf_row);
            if (table && s >= 1) {
                const float* ep = g.E + (int64_t)(fwd ? s - 1 : line) * g.ld + c0;
                cp_async16(&row[1][4 + 4 * lane], lane_loads ? (const void*)ep : g_inf_row);
                cp_async16(&row[2][4 + 4 * lane], lane_loads ? (const void*)(ep + g.eplane) : g_inf_row);
                cp_async16(&row[3][4 + 4 * lane],
                           lane_loads ? (const void*)(ep + 2 * g.eplane) : g_inf_row);
            }
        }
        cp_async_arrive_noinc(&sm.in_full[slot]);
    }
    return true;
}

// Flusher warp: writes the owned columns of each finished chunk.
template <bool fwd, bool codes>
__device__ bool flusher_tile(const Chain2DArgs& a, const TileGeo& g, TileSmem& sm,
                             unsigned int cb) {
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    const int L = g.L;
    bool owned[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) owned[i] = (c0 + i >= g.q0) && (c0 + i < g.q1);
    const bool all_owned = owned[0] && owned[3];
    const int ncol = g.q1 - g.q0;
    const int off = g.q0 - g.r0;
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = slot_of(gc, kNo);
        if (!__all_sync(0xffffffffu,
                        mbar_wait(&sm.done[slot_of(gc, kNci)], full_parity(gc, kNci), a)))
            return false;
        const int s0 = g.s0 + c * kCh;
        const int nl = min(kCh, g.ns - c * kCh);
        if (c >= *(volatile int*)&sm.stop_chunk) {
            // a re-run that stopped early: these lines already hold their values
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.out_empty[slot]);
            continue;
        }
        if (fwd) {
            // rows of the output array: each lane writes its own four
            // columns; the values go to registers first and the output slot
            // is handed back before the global stores (without codes)
            float4 v[kCh];
#pragma unroll
            for (int j = 0; j < kCh; ++j)
                v[j] = *reinterpret_cast<const float4*>(&sm.out[slot][j][4 * lane]);
            if (!codes) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.out_empty[slot]);
            }
#pragma unroll
            for (int j = 0; j < kCh; ++j) {
                if (j >= nl) break;
                float* row = g.out + (int64_t)(s0 + j) * g.out_ld + c0;
                if (all_owned) {
                    *reinterpret_cast<float4*>(row) = v[j];
                } else {
                    if (owned[0]) row[0] = v[j].x;
                    if (owned[1]) row[1] = v[j].y;
                    if (owned[2]) row[2] = v[j].z;
                    if (owned[3]) row[3] = v[j].w;
                }
            }
        } else {
            // transposed: consecutive lanes write consecutive lines of a
            // column (32 / kCh columns per warp-wide store)
            const int jj = lane & (kCh - 1);
            const int line = L - 1 - (s0 + jj);
            for (int col = lane / kCh; col < ncol; col += 32 / kCh)
                if (jj < nl) g.out[(int64_t)(g.q0 + col) * g.out_ld + line] = sm.out[slot][jj][off + col];
            if (!codes) {
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.out_empty[slot]);
            }
        }
        if (codes) {
            if (g.codes_rows) {
                // vertical pass: the lines are rows of the image
#pragma unroll
                for (int j = 0; j < kCh; ++j) {
                    if (j >= nl) break;
                    const int line = fwd ? s0 + j : L - 1 - (s0 + j);
                    const uint8_t* cj = &sm.outc[slot][j][4 * lane];
                    uint8_t* row = g.codes + (int64_t)line * g.Q + c0;
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (owned[i]) row[i] = cj[i];
                }
            } else {
                // horizontal pass: the lines are columns of the image
                const int jj = lane & (kCh - 1);
                const int line = fwd ? s0 + jj : L - 1 - (s0 + jj);
                for (int col = lane / kCh; col < ncol; col += 32 / kCh)
                    if (jj < nl) g.codes[(int64_t)(g.q0 + col) * L + line] = sm.outc[slot][jj][off + col];
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.out_empty[slot]);
        }
    }
    return true;
}

// One line of chain input in registers: old values and the costs of the
// three parents (column offsets -1, 0, +1) of each of the lane's columns.
struct LineIn {
    float dold[4];
    float c0[4], c1[4], c2[4];
};

// Reads line j of a ring chunk.  Ring row k+1 holds E_k[e][x], the cost of
// the edge from column x of one line to column x+k-1 of the next.  In a
// forward step the parent of x at offset k-1 sits on the previous line, so
// its cost is E_{2-k}[x+k-1] (the two shifted rows need one extra element
// from the padding or the neighbouring lane's range); in a backward step the
// parent sits on the next line and the cost is E_k[x].
template <bool fwd, bool table>
__device__ __forceinline__ void load_line(const float* r0, const float* r1, const float* r2,
                                          const float* r3, int lane, LineIn& r, float k0,
                                          float k1, float k2) {
    const float4 o = *reinterpret_cast<const float4*>(r0 + 4 * lane);
    r.dold[0] = o.x; r.dold[1] = o.y; r.dold[2] = o.z; r.dold[3] = o.w;
    if (!table) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            r.c0[i] = k0;
            r.c1[i] = k1;
            r.c2[i] = k2;
        }
        return;
    }
    const float4 e0 = *reinterpret_cast<const float4*>(r1 + 4 * lane);
    const float4 e1 = *reinterpret_cast<const float4*>(r2 + 4 * lane);
    const float4 e2 = *reinterpret_cast<const float4*>(r3 + 4 * lane);
    if (fwd) {
        const float e2m = r3[4 * lane - 1];
        const float e0p = r1[4 * lane + 4];
        r.c0[0] = e2m;  r.c0[1] = e2.x; r.c0[2] = e2.y; r.c0[3] = e2.z;
        r.c2[0] = e0.y; r.c2[1] = e0.z; r.c2[2] = e0.w; r.c2[3] = e0p;
    } else {
        r.c0[0] = e0.x; r.c0[1] = e0.y; r.c0[2] = e0.z; r.c0[3] = e0.w;
        r.c2[0] = e2.x; r.c2[1] = e2.y; r.c2[2] = e2.z; r.c2[3] = e2.w;
    }
    r.c1[0] = e1.x; r.c1[1] = e1.y; r.c1[2] = e1.z; r.c1[3] = e1.w;
}

// One min-plus line update (Jacobi within the line): candidates in the fixed
// order old value, own parents, then the parents held by the neighbouring
// lanes.  Columns outside the array stay at +inf: with cost tables their old
// values and the costs of every edge into them are +inf already (table and
// array padding, +inf ring rows), with constant costs they are masked.
// The neighbouring lanes' edge columns of the previous line; issued before
// the next line's shared-memory loads so that the shuffles, which sit on the
// line-to-line chain, do not queue behind them.
__device__ __forceinline__ void chain_shuffle(const float (&dp)[4], int lane, float& left,
                                              float& right) {
    left = __shfl_up_sync(0xffffffffu, dp[3], 1);
    right = __shfl_down_sync(0xffffffffu, dp[0], 1);
    if (lane == 0) left = kInf;
    if (lane == 31) right = kInf;
}

template <bool masked, bool codes>
__device__ __forceinline__ void chain_step(float (&dp)[4], float left, float right,
                                           const LineIn& c, const bool (&valid)[4], float* out,
                                           uint8_t* outc) {
    float nd[4];
    unsigned int packed = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float x0 = (i > 0) ? __fadd_rn(dp[i - 1], c.c0[i]) : 0.0f;
        const float x1 = __fadd_rn(dp[i], c.c1[i]);
        const float x2 = (i < 3) ? __fadd_rn(dp[i + 1], c.c2[i]) : 0.0f;
        float best = c.dold[i];
        if (i > 0) best = fminf(best, x0);
        best = fminf(best, x1);
        if (i < 3) best = fminf(best, x2);
        const float y0 = (i == 0) ? __fadd_rn(left, c.c0[0]) : x0;
        const float y2 = (i == 3) ? __fadd_rn(right, c.c2[3]) : x2;
        if (i == 0) best = fminf(best, y0);
        if (i == 3) best = fminf(best, y2);
        nd[i] = (!masked || valid[i]) ? best : kInf;
        if (codes) {
            // 0: kept its value; else 1 + the lowest parent index reaching the
            // (strictly smaller) minimum, in integer arithmetic (no branch on
            // the data in the chain step)
            const unsigned int lt = nd[i] < c.dold[i] ? 1u : 0u;
            const unsigned int ne0 = y0 != nd[i] ? 1u : 0u;
            const unsigned int ne1 = x1 != nd[i] ? 1u : 0u;
            packed |= (lt * (1u + ne0 + (ne0 & ne1))) << (8 * i);
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dp[i] = nd[i];
    *reinterpret_cast<float4*>(out) = make_float4(nd[0], nd[1], nd[2], nd[3]);
    if (codes) *reinterpret_cast<unsigned int*>(outc) = packed;
}

// Ring refresh of a multi-tile pass before step s (dp holds line s-1).
__device__ __forceinline__ bool exchange(const Chain2DArgs& a, const TileGeo& g, int b, int tile,
                                         unsigned int tg, int par, float (&dp)[4],
                                         const bool (&valid)[4]) {
    (void)b;
    const RingLink x{g.xb, a.status, a.timeout_ns};
    return ring_exchange(x, tile, g.ntiles, g.q0, g.K, g.T, g.r0 + 4 * (int)(threadIdx.x & 31),
                         tg, par, dp, valid, kInf);
}

// Checkpoint k >= 1 of a re-run (at a chunk boundary; dp holds the last
// line of the previous chunk, dl that line's old values, i.e. the first
// run's).  Each tile adds one arrival to the checkpoint's word, plus 1 << 16
// if its owned columns of that line changed (a single reduction: no fence).
// The decision at checkpoint k concerns checkpoint k - kCkLag, whose word
// was read one checkpoint earlier (pv) and is complete by then unless a tile
// lags that far behind (then it is read again until complete): a line in
// which no column changed means every later line equals the first run's (the
// same line step from the same line), so all tiles stop at this chunk.
// Returns false on a failed wait.
constexpr int kCkLag = 2;
__device__ __forceinline__ bool checkpoint(const Chain2DArgs& a, const TileGeo& g, int k,
                                           const float (&dp)[4], const float (&dl)[4], int c0,
                                           unsigned int& pv, bool& stop) {
    const int lane = threadIdx.x & 31;
    bool ch = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = c0 + i;
        if (c >= g.q0 && c < g.q1 && __float_as_uint(dp[i]) != __float_as_uint(dl[i])) ch = true;
    }
    ch = __any_sync(0xffffffffu, ch);
    int verdict = 0;  // 0: go on, 1: stop, -1: failed
    if (lane == 0) {
        atomicAdd(g.ck + k, ch ? 0x10001u : 1u);
        if (k > kCkLag) {
            const unsigned int want = (unsigned int)g.ntiles;
            long long t0 = 0;
            for (unsigned int it = 0; (pv & 0xffffu) < want; ++it) {
                pv = ld_relaxed_u32(g.ck + k - kCkLag);
                if ((it & 15u) == 15u) {
                    const long long now = gtimer();
                    if (t0 == 0) t0 = now;
                    if (status_of(a.status) != 0) { verdict = -1; break; }
                    if (now - t0 > a.timeout_ns) {
                        record_timeout(a.status);
                        verdict = -1;
                        break;
                    }
                }
            }
            if (verdict == 0 && (pv >> 16) == 0u) verdict = 1;
        }
        if (k + 1 > kCkLag) pv = ld_relaxed_u32(g.ck + k + 1 - kCkLag);  // for the next checkpoint
    }
    verdict = __shfl_sync(0xffffffffu, verdict, 0);
    stop = verdict == 1;
    return verdict >= 0;
}

// Chain warp.  Line j of chunk c is step s = kCh*c + j; the first step (the
// first line of the sweep, which has no parents) runs with +inf parents and
// so keeps the old values.  AHEAD lines of input are held in registers ahead
// of the step that uses them.
template <bool fwd, bool table, bool codes, int AHEAD, bool CK, bool TMA>
__device__ bool chain_tile(const Chain2DArgs& a, const TileGeo& g, int t_app, int b, int tile,
                           TileSmem& sm, unsigned int cb, float k0, float k1, float k2) {
    constexpr int NB = AHEAD == 1 ? 2 : 4;  // register buffers (divides kCh)
    const float* tbase = TMA ? tma_ring(sm) : nullptr;
    auto load = [&](int slot, int j, LineIn& r) {
        load_line<fwd, table>(ring_row<TMA, fwd>(sm, tbase, slot, j, 0),
                              ring_row<TMA, fwd>(sm, tbase, slot, j, 1),
                              ring_row<TMA, fwd>(sm, tbase, slot, j, 2),
                              ring_row<TMA, fwd>(sm, tbase, slot, j, 3), threadIdx.x & 31, r, k0,
                              k1, k2);
    };
    const int lane = threadIdx.x & 31;
    const int c0 = g.r0 + 4 * lane;
    bool valid[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) valid[i] = (c0 + i >= 0) && (c0 + i < g.Q);
    (void)t_app;
    const unsigned int tag_base = g.tag_base;
    // the line before the first step: none at the start of a pass (+inf
    // parents), else the line the segment starts from
    float dp[4] = {kInf, kInf, kInf, kInf};
    if (g.bline) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (valid[i]) dp[i] = __ldcg(g.bline + (int64_t)(c0 + i) * g.bstride);
    }
    LineIn buf[NB];
    // ring positions (slot, phase parity) of chunks gc, gc+1, gc+2 of the
    // input ring and gc, gc+1 of the output ring, advanced without divisions
    RingPos i0(cb, kNci), i1 = i0.next(kNci), i2 = i1.next(kNci);
    RingPos o0(cb, kNo), o1 = o0.next(kNo);
    if (!__all_sync(0xffffffffu, mbar_wait(&sm.in_full[i0.slot], i0.par, a))) return false;
#pragma unroll
    for (int j = 0; j < AHEAD; ++j) load(i0.slot, j, buf[j]);
    int next_refresh = g.multi ? g.K : 0x7fffffff;
    int blk = 0;
    // Hand-overs are tested one chunk in advance (non-blocking) so the test's
    // latency overlaps a chunk of work; a blocking wait follows only when the
    // test found the chunk not ready yet.
    bool in_ready = g.nch < 2 || mbar_peek(&sm.in_full[i1.slot], i1.par);
    bool out_ready = cb < (unsigned)kNo || mbar_peek(&sm.out_empty[o0.slot], o0.par ^ 1u);
    bool skip = false;  // a re-run found its values equal to the first run's
    unsigned int ck_prev = 0;  // checkpoint word read one checkpoint earlier
    for (int c = 0; c < g.nch; ++c) {
        const unsigned int gc = cb + c;
        const int slot = i0.slot, nslot = i1.slot, oslot = o0.slot;
        if (!__all_sync(0xffffffffu, in_ready) &&
            !__all_sync(0xffffffffu, mbar_wait(&sm.in_full[nslot], i1.par, a)))
            return false;
        if (!__all_sync(0xffffffffu, out_ready) &&
            !__all_sync(0xffffffffu, mbar_wait(&sm.out_empty[oslot], o0.par ^ 1u, a)))
            return false;
        in_ready = c + 2 >= g.nch || mbar_peek(&sm.in_full[i2.slot], i2.par);
        out_ready = gc + 1 < (unsigned)kNo || mbar_peek(&sm.out_empty[o1.slot], o1.par ^ 1u);
        i0 = i1;
        i1 = i2;
        i2 = i2.next(kNci);
        o0 = o1;
        o1 = o1.next(kNo);
        if (CK && !skip && c > 0 && c % g.ck_every == 0) {
            if (!checkpoint(a, g, c / g.ck_every, dp, buf[(kCh - 1) % NB].dold, c0, ck_prev,
                            skip))
                return false;
            if (skip && lane == 0) *(volatile int*)&sm.stop_chunk = c;
        }
        if (CK && skip) {
            // the rest of the segment keeps the first run's values: chunks
            // are only handed over
            __syncwarp();
            if (lane == 0) mbar_arrive(&sm.done[slot]);
            continue;
        }
#pragma unroll
        for (int j = 0; j < kCh; ++j) {
            if (j % kSub == 0 && !skip && c * kCh + j == next_refresh) {
                if (!exchange(a, g, b, tile, tag_base | (unsigned int)(blk + 1), blk & 1, dp,
                              valid))
                    return false;
                next_refresh += g.K;
                ++blk;
            }
            const int nj = j + AHEAD;
            float left, right;
            chain_shuffle(dp, lane, left, right);
            load(nj < kCh ? slot : nslot, nj < kCh ? nj : nj - kCh, buf[nj % NB]);
            chain_step<!table, codes>(dp, left, right, buf[j % NB], valid,
                                      &sm.out[oslot][j][4 * lane], &sm.outc[oslot][j][4 * lane]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.done[slot]);
    }
    if (CK && skip) {
        // the last line is the first run's: so is its comparison
        if (g.flag && lane == 0 && ld_relaxed_u32(g.flag_first) == g.flag_tag)
            atomicMax(g.flag, g.flag_tag);
    } else if (g.cmp) {
        // the segment's last line against the line the next segment started from
        bool diff = false;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = c0 + i;
            if (c >= g.q0 && c < g.q1 &&
                __float_as_uint(dp[i]) != __float_as_uint(__ldcg(g.cmp + c)))
                diff = true;
        }
        if (__any_sync(0xffffffffu, diff) && lane == 0) atomicMax(g.flag, g.flag_tag);
    }
    return true;
}

// Initial distances and cost tables, one 32 x 32 pixel tile per block
// (32 x 8 threads, four rows each): Dw = v * M, Ev[k][h][w] = cost of the edge
// (h, w) - (h+1, w+k-1), Eh[k][w][h] = cost of the edge (h, w) - (h+k-1, w+1)
// (written through a shared-memory transpose so both tables are stored along
// their contiguous dimension); padding columns and missing edges are +inf.
// CC > 0: the CC channels of the tile and a one-pixel halo are staged in
// shared memory once; CC == 0: any channel count, read from global memory.
constexpr int kInitTile = 32;
constexpr int kHalo = kInitTile + 2;
template <int CC>
__device__ __forceinline__ void init_tile(const Chain2DArgs& a, int b) {
    __shared__ float eh[3][kInitTile][kInitTile + 1];
    __shared__ float tile[CC > 0 ? CC : 1][kHalo][kHalo + 1];
    const int64_t N = (int64_t)a.H * a.W;
    const int w0 = blockIdx.x * kInitTile, h0 = blockIdx.y * kInitTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const float* img = a.image + (int64_t)(b % a.nimg) * a.C * N;
    if (CC > 0 && a.table) {
        // rows h0-1 .. h0+32, columns w0-1 .. w0+32 (0 outside the image)
        for (int idx = ty * 32 + tx; idx < kHalo * kHalo; idx += 256) {
            const int r = idx / kHalo, c = idx - r * kHalo;
            const int h = h0 - 1 + r, w = w0 - 1 + c;
            const bool in = h >= 0 && h < a.H && w >= 0 && w < a.W;
#pragma unroll
            for (int ch = 0; ch < (CC > 0 ? CC : 1); ++ch)
                tile[ch][r][c] = in ? img[ch * N + (int64_t)h * a.W + w] : 0.0f;
        }
        __syncthreads();
    }
    const int w = w0 + tx;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int hl = ty + 8 * i, h = h0 + hl;
        if (h < a.H && w < a.Wp) {
            const int64_t row = (int64_t)b * a.H + h;
            a.Dw[row * a.Wp + w] = w < a.W ? __fmul_rn(a.v, a.mask[row * a.W + w]) : kInf;
        }
        if (!a.table) continue;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float cv = kInf, ch = kInf;
            const int wn = w + k - 1, hn = h + k - 1;
            const bool has_v = h < a.H && w < a.W && h + 1 < a.H && wn >= 0 && wn < a.W;
            const bool has_h = h < a.H && w < a.W && w + 1 < a.W && hn >= 0 && hn < a.H;
            if (CC > 0) {
                // fixed arithmetic order: di2 = sum_ch (I(a)-I(b))^2, c = sqrt(t + lambda*di2)
                float dv = 0.0f, dh = 0.0f;
#pragma unroll
                for (int c = 0; c < (CC > 0 ? CC : 1); ++c) {
                    const float self = tile[c][hl + 1][tx + 1];
                    const float x = __fsub_rn(tile[c][hl + 2][tx + k], self);
                    const float y = __fsub_rn(tile[c][hl + k][tx + 2], self);
                    dv = a.fast ? __fmaf_rn(x, x, dv) : __fadd_rn(dv, __fmul_rn(x, x));
                    dh = a.fast ? __fmaf_rn(y, y, dh) : __fadd_rn(dh, __fmul_rn(y, y));
                }
                if (a.fast) {
                    if (has_v) cv = fast_sqrt(__fmaf_rn(a.lambda, dv, a.tv[k]));
                    if (has_h) ch = fast_sqrt(__fmaf_rn(a.lambda, dh, a.th[k]));
                } else {
                    if (has_v) cv = __fsqrt_rn(__fadd_rn(a.tv[k], __fmul_rn(a.lambda, dv)));
                    if (has_h) ch = __fsqrt_rn(__fadd_rn(a.th[k], __fmul_rn(a.lambda, dh)));
                }
            } else {
                const float* self = img + (int64_t)h * a.W + w;
                if (has_v)
                    cv = edge_cost(img + (int64_t)(h + 1) * a.W + wn, self, a.C, N, a.tv[k],
                                   a.lambda, a.fast);
                if (has_h)
                    ch = edge_cost(img + (int64_t)hn * a.W + w + 1, self, a.C, N, a.th[k],
                                   a.lambda, a.fast);
            }
            if (h < a.H && w < a.Wp) a.Ev[(((int64_t)b * 3 + k) * a.H + h) * a.Wp + w] = cv;
            eh[k][tx][hl] = ch;  // [w local][h local]
        }
    }
    __syncthreads();
    // transposed write-out: rows w of Eh (and the +inf padding rows of Dt)
    const int h = h0 + tx;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int wl = ty + 8 * i, ww = w0 + wl;
        if (ww >= a.W || h >= a.Hp) continue;
        const int64_t row = (int64_t)b * a.W + ww;
        if (h >= a.H) a.Dt[row * a.Hp + h] = kInf;
        if (a.table) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
                a.Eh[(((int64_t)b * 3 + k) * a.W + ww) * a.Hp + h] = h < a.H ? eh[k][wl][tx] : kInf;
        }
    }
}

template <int CC>
__global__ void __launch_bounds__(256) chain2d_init_kernel(const Chain2DArgs a) {
    init_tile<CC>(a, blockIdx.z);
}

// Batched launch: instance blockIdx.z of an array of single-image arguments.
template <int CC>
__global__ void __launch_bounds__(256) chain2d_init_batched_kernel(const Chain2DArgs* desc) {
    const Chain2DArgs& a = desc[blockIdx.z];
    if ((int)blockIdx.x * kInitTile >= a.Wp || (int)blockIdx.y * kInitTile >= a.Hp) return;
    init_tile<CC>(a, 0);
}

// Not inlined: the pass driver calls it from two places, and each variant's
// chain loop keeps its own register allocation.
template <bool fwd, bool table, bool codes, bool CK, bool TMA>
__device__ __noinline__ bool run_tile(const Chain2DArgs& a, int t_app, int pass, int b, int tile,
                         TileSmem& sm, unsigned int cb, int seg, bool rerun, int nseg) {
    const TileGeo g = tile_geo(a, t_app, pass, b, tile, seg, rerun, nseg);
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        const bool vert = pass < 2;
        const float k0 = vert ? a.cv[0] : a.chh[0];
        const float k1 = vert ? a.cv[1] : a.chh[1];
        const float k2 = vert ? a.cv[2] : a.chh[2];
        return chain_tile<fwd, table, codes, table ? 2 : 1, CK, TMA>(a, g, t_app, b, tile, sm, cb,
                                                                 k0, k1, k2);
    }
    if (warp == 1)
        return TMA ? producer_tma<fwd, table>(a, g, sm, cb, b, pass < 2)
                   : producer_tile<fwd, table>(a, g, sm, cb);
    return flusher_tile<fwd, codes>(a, g, sm, cb);
}

template <bool codes, bool TMA>
__device__ __forceinline__ bool run_pass_tile(const Chain2DArgs& a, bool fwd, int t_app, int pass,
                                              int b, int tile, TileSmem& sm, unsigned int cb,
                                              int seg = 0, bool rerun = false, int nseg = 1) {
    // re-runs of in-place passes carry the early-stop checkpoints
    const bool ck = rerun && seg > 0 && !codes;
    if (fwd && a.table && ck)
        return run_tile<true, true, false, true, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
    if (fwd && ck)
        return run_tile<true, false, false, true, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
    if (fwd && a.table)
        return run_tile<true, true, codes, false, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
    if (fwd)
        return run_tile<true, false, codes, false, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
    if (a.table)
        return run_tile<false, true, codes, false, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
    return run_tile<false, false, codes, false, TMA>(a, t_app, pass, b, tile, sm, cb, seg, rerun, nseg);
}

// Speculative segments of one pass application (all images in one wave: the
// host sizes the grid for B * S * ntiles blocks).  Phase A: the tiles of
// segments 1 .. S-1 save the line before their segment (the values the pass
// starts from), then every segment runs at once from its saved line.  A pass
// only lowers values, so a segment that started from a line whose exact value
// differs from the saved one holds values >= the exact ones; running it again
// from the exact line over those values gives the exact result (a min-plus
// line step is monotone and min(old, spec, exact chain) = min(old, exact
// chain)).  Phase B visits the segments in order: segment j runs again when
// the exact last line of segment j-1 differs from the line j started from
// (each segment's chain compares its last line and sets the boundary's
// flag).  In the passes that update their lines in place a re-run reads the
// first run's values as old values and stops as soon as a whole line equals
// them (checkpoints every ring refresh).  Every block takes the same decisions
// from the same flags, so all blocks meet the same grid barriers.
template <bool codes, bool TMA>
__device__ bool run_pass_segments(const Chain2DArgs& a, int t_app, int pass, int S, int ntiles,
                                  TileSmem& sm, unsigned int& cb, unsigned int& epoch,
                                  uint8_t* rr) {
    const bool fwd = (pass == 0 || pass == 2);
    const bool vert = pass < 2;
    const int L = vert ? a.H : a.W;
    const int u = blockIdx.x;
    const bool active = u < a.B * S * ntiles;
    const int b = active ? u / (S * ntiles) : 0;
    const int seg = active ? (u / ntiles) % S : 0;
    const int tile = u % ntiles;
    // phase A.1: save the owned columns of the line before each segment
    if (active && seg > 0 && tile == 0) {
        unsigned int* ck = a.ckpt + ((int64_t)b * kMaxSeg + seg) * kMaxCk;
        for (int i = threadIdx.x; i < kMaxCk; i += blockDim.x) ck[i] = 0u;
    }
    if (active && seg > 0) {
        const TileGeo g = tile_geo(a, t_app, pass, b, tile, seg, false, S);
        const int line = line_of(fwd, L, g.s0 - 1);
        const float* srow = g.src + (int64_t)line * g.ld;
        float* dst = a.bnd + ((int64_t)b * (kMaxSeg - 1) + seg - 1) * a.bnd_ld;
        for (int q = g.q0 + (int)threadIdx.x; q < g.q1; q += blockDim.x) dst[q] = __ldcg(srow + q);
    }
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns)) return false;
    // phase A.2: all segments at once
    bool ok = true;
    if (active) {
        ok = run_pass_tile<codes, TMA>(a, fwd, t_app, pass, b, tile, sm, cb, seg, false, S);
        const TileGeo g = tile_geo(a, t_app, pass, b, tile, seg, false, S);
        cb += (unsigned int)g.nch;
    }
    if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns) || !ok) return false;
    // phase B: segments in order, again where their start line changed
    __shared__ int any;
    if (threadIdx.x == 0)
        for (int i = 0; i < a.B; ++i) rr[i] = 0;
    const unsigned int tag = (unsigned int)(t_app + 1);
    for (int j = 1; j < S; ++j) {
        if (threadIdx.x == 0) sm.stop_chunk = 0x7fffffff;
        __syncthreads();
        if (threadIdx.x == 0) {
            any = 0;
            for (int i = 0; i < a.B; ++i) {
                const unsigned int* f = a.segflag + ((int64_t)i * kMaxSeg + j) * 2;
                const unsigned int fv = ld_relaxed_u32(f + (rr[i] ? 1 : 0));
                rr[i] = fv == tag;
                any |= rr[i];
            }
        }
        __syncthreads();
        if (!any) continue;
        if (blockIdx.x == 0 && threadIdx.x == 0)  // remembered for this pass's next application
            *(a.segflag + (int64_t)a.B * kMaxSeg * 2 + pass) = (unsigned int)(t_app + 1);
        const int bb = u / ntiles;
        if (u < a.B * ntiles && rr[bb]) {
            ok = run_pass_tile<codes, TMA>(a, fwd, t_app, pass, bb, tile, sm, cb, j, true, S);
            const TileGeo g = tile_geo(a, t_app, pass, bb, tile, j, true, S);
            cb += (unsigned int)g.nch;
        }
        if (!grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns) || !ok) return false;
    }
    if (threadIdx.x == 0) sm.stop_chunk = 0x7fffffff;
    __syncthreads();
    return true;
}

// One persistent launch for all passes; `codes` selects the variant that also
// records the parent codes.
template <bool codes, bool TMA>
__global__ void __launch_bounds__(kBlockThreads, 1)
    chain2d_kernel(const __grid_constant__ Chain2DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem& sm = *reinterpret_cast<TileSmem*>(smem_raw);
    const int64_t N = (int64_t)a.H * a.W;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int epoch = 1;
    if (a.iterations == 0) {
        for (int64_t i = tid; i < a.B * N; i += nthreads) a.dist[i] = __fmul_rn(a.v, a.mask[i]);
        return;
    }
    // ring rows start at +inf (the padding columns are never written again)
    for (int i = threadIdx.x; i < kNci * kCh * 4 * kRow; i += blockDim.x)
        (&sm.in[0][0][0][0])[i] = kInf;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNci; ++i) {
            // one transaction-counted arrival (tensor copies) or one
            // asynchronous arrival per producer lane
            mbar_init(&sm.in_full[i], TMA ? 1 : 32);
            mbar_init(&sm.done[i], 1);
        }
        for (int i = 0; i < kNo; ++i) mbar_init(&sm.out_empty[i], 1);
        sm.stop_chunk = 0x7fffffff;
        if (TMA) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the ring's initial +inf (ordinary stores) before tensor copies write it
    if (TMA) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        timeline[0] = timeline[1] = (unsigned long long)gtimer();
    bool alive = true;
    unsigned int cb = 0;  // chunks handed over so far in this block
    const int napps = a.iterations * 4;
    __shared__ uint8_t rerun[kMaxSegImages];
    for (int t_app = 0; t_app < napps && alive; ++t_app) {
        const int pass = t_app % 4;
        const int ntiles = pass < 2 ? a.tiles_v : a.tiles_h;
        const int L = pass < 2 ? a.H : a.W;
        const int S = pass < 2 ? a.nseg_v : a.nseg_h;
        // Segments from the second iteration on (the first one changes nearly
        // every line: its start lines always move), and not in a pass whose
        // segments ran again in the previous iteration.
        const bool speculate = S > 1 && t_app >= 4 &&
                               ld_relaxed_u32(a.segflag + (int64_t)a.B * kMaxSeg * 2 + pass) !=
                                   (unsigned int)(t_app - 4 + 1);
        if (speculate && a.B <= kMaxSegImages && a.B * S * ntiles <= (int)gridDim.x) {
            alive = run_pass_segments<codes, TMA>(a, t_app, pass, S, ntiles, sm, cb, epoch, rerun);
            if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 2 < 16)
                timeline[t_app + 2] = (unsigned long long)gtimer();
            continue;
        }
        const int per_wave = gridDim.x / ntiles;
        const int nwaves = (a.B + per_wave - 1) / per_wave;
        bool ok = true;
        for (int wv = 0; wv < nwaves && ok; ++wv) {
            if ((int)blockIdx.x < per_wave * ntiles) {
                const int b = wv * per_wave + blockIdx.x / ntiles;
                if (b < a.B) {
                    const int tile = blockIdx.x % ntiles;
                    const bool fwd = (pass == 0 || pass == 2);
                    ok = run_pass_tile<codes, TMA>(a, fwd, t_app, pass, b, tile, sm, cb);
                    cb += (unsigned int)((L + kCh - 1) / kCh);
                }
            }
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 2 < 16)
            timeline[t_app + 2] = (unsigned long long)gtimer();
    }
}

// Work list of a batched launch of single images of uneven shapes: round r
// applies pass r % 4 of every instance that has r < 4 * iterations; the
// round's (instance, tile) items are packed into waves of at most one item
// per block, so that all tiles of an instance's pass run together.
struct Chain2DBatch {
    const Chain2DArgs* desc;   // [n] single-image arguments
    int rounds;
    const int* round_waves;    // [rounds + 1] first wave of each round
    const int* wave_items;     // [waves][gridDim.x]: (instance << 16) | tile, or -1
    unsigned int* barrier;
    int* status;
    long long timeout_ns;
};

__global__ void __launch_bounds__(kBlockThreads, 1) chain2d_batched_kernel(const Chain2DBatch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem& sm = *reinterpret_cast<TileSmem*>(smem_raw);
    for (int i = threadIdx.x; i < kNci * kCh * 4 * kRow; i += blockDim.x)
        (&sm.in[0][0][0][0])[i] = kInf;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kNci; ++i) {
            mbar_init(&sm.in_full[i], 32);
            mbar_init(&sm.done[i], 1);
        }
        for (int i = 0; i < kNo; ++i) mbar_init(&sm.out_empty[i], 1);
        sm.stop_chunk = 0x7fffffff;  // no early stops in batched runs
    }
    __syncthreads();
    unsigned int epoch = 1;
    unsigned int cb = 0;
    bool alive = true;
    for (int r = 0; r < bt.rounds && alive; ++r) {
        const int pass = r & 3;
        const bool fwd = pass == 0 || pass == 2;
        bool ok = true;
        for (int wv = bt.round_waves[r]; wv < bt.round_waves[r + 1] && ok; ++wv) {
            const int item = bt.wave_items[(int64_t)wv * gridDim.x + blockIdx.x];
            if (item < 0) continue;
            const Chain2DArgs& a = bt.desc[item >> 16];
            ok = run_pass_tile<false, false>(a, fwd, r, pass, 0, item & 0xffff, sm, cb);
            const int L = pass < 2 ? a.H : a.W;
            cb += (unsigned int)((L + kCh - 1) / kCh);
        }
        alive = grid_barrier(bt.barrier, epoch++, bt.status, bt.timeout_ns);
    }
}

}  // namespace

// ---------------------------------------------------------------- host ----


int chain2d_geometry(int64_t H, int64_t W, const fgx_options* opt, int* K, int* T, int* tv,
                     int* th) {
    // K: lines between ring refreshes, a multiple of kSub lines; T >= K so
    // a ring never reaches past the neighbouring tile
    int k = (opt && opt->tile_lines) ? opt->tile_lines : 40;
    k = std::max(kSub, std::min(40, (k + kSub - 1) / kSub * kSub));
    int t = kRegion - 2 * k;
    if (opt && opt->tile_width) t = std::min(t, std::max(kSub, opt->tile_width & ~3));
    if (t < k) k = t / kSub * kSub;
    *K = k;
    *T = t;
    // a line that fits one region is one tile, unless a tile width is forced
    const int64_t single = (opt && opt->tile_width) ? t : kRegion;
    *tv = W <= single ? 1 : (int)((W + t - 1) / t);
    *th = H <= single ? 1 : (int)((H + t - 1) / t);
    return FGX_OK;
}

namespace {

// Fills the arguments of B images of one shape: the status word and barrier
// counter are `hdr`'s, the exchange words start at `xb`, the other buffers
// (Dw, Dt, Ev, Eh) are laid out from `sec` (any of them null for a size
// query).  Returns the bytes from `sec`; *xbytes receives the exchange bytes.
// max_seg: exchange areas per image (kMaxSeg for speculative segments, 1
// without); the segment counts themselves are set by the caller (1 here).
size_t fill_chain_args(Chain2DArgs* a, const float* image, const float* mask, float* dist,
                       uint8_t* codes, int64_t B, int64_t C, int64_t H, int64_t W, float v,
                       float lambda, int iterations, const fgx_options* opt, char* hdr, char* xb,
                       char* sec, size_t* xbytes, int max_seg) {
    std::memset(a, 0, sizeof(*a));
    int K, T, tv, th;
    chain2d_geometry(H, W, opt, &K, &T, &tv, &th);
    const int max_tiles = std::max(tv, th);
    a->image = image;
    a->mask = mask;
    a->dist = dist;
    a->codes = codes;
    a->B = (int)B;
    a->nimg = (int)std::max<int64_t>(B, 1);
    a->C = (int)C;
    a->H = (int)H;
    a->W = (int)W;
    a->Wp = (int)((W + 3) & ~int64_t(3));
    a->Hp = (int)((H + 3) & ~int64_t(3));
    a->v = v;
    a->lambda = lambda;
    a->iterations = iterations;
    a->table = lambda != 0.0f;
    // fast math where the general formula applies (the lambda = 1 single
    // channel cost sqrt(d*d) stays exact), never for recorded codes
    a->fast = opt && opt->fast_math && lambda != 0.0f && !(lambda == 1.0f && C == 1) && !codes;
    const float unit[3] = {1.f, 1.f, 1.f};
    float t9[9];
    pass_offsets_t(2, 1, unit, lambda, t9);  // pass along H: offsets along W
    for (int k = 0; k < 3; ++k) { a->tv[k] = t9[k]; a->cv[k] = std::sqrt(t9[k]); }
    pass_offsets_t(2, 2, unit, lambda, t9);  // pass along W: offsets along H
    for (int k = 0; k < 3; ++k) { a->th[k] = t9[k]; a->chh[k] = std::sqrt(t9[k]); }
    a->K = K;
    a->T = T;
    a->tiles_v = tv;
    a->tiles_h = th;
    a->max_tiles = max_tiles;
    a->timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) * 1000000LL;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    a->status = (int*)hdr;
    a->barrier = (unsigned int*)(hdr ? hdr + 64 : nullptr);
    // no segment areas where no pass can be split
    if (std::max(H, W) < 2 * kMinSegLines || B > kMaxSegImages || (opt && opt->segments == 1))
        max_seg = 1;
    a->nseg_v = a->nseg_h = 1;
    a->seglen_v = (int)H;
    a->seglen_h = (int)W;
    a->max_seg = max_seg;
    a->bnd_ld = (int)((std::max(H, W) + 3) & ~int64_t(3));
    a->xbuf = (unsigned long long*)xb;
    *xbytes = al((size_t)B * max_seg * max_tiles * 4 * kMaxRing * 8);
    // segment flags live in the zeroed exchange area
    a->segflag = (unsigned int*)(xb && max_seg > 1 ? xb + *xbytes : nullptr);
    // (then one word per pass: 1 + the last application whose segments ran again)
    if (max_seg > 1) *xbytes += al((size_t)B * kMaxSeg * 2 * 4 + 4 * 4);
    size_t off = 0;
    a->Dw = (float*)(sec ? sec + off : nullptr);
    off += al((size_t)B * H * a->Wp * 4);
    a->Dt = (float*)(sec ? sec + off : nullptr);
    off += al((size_t)B * W * a->Hp * 4);
    a->Ev = (float*)(sec ? sec + off : nullptr);
    off += al((size_t)B * 3 * H * a->Wp * 4);
    a->Eh = (float*)(sec ? sec + off : nullptr);
    off += al((size_t)B * 3 * W * a->Hp * 4);
    a->bnd = (float*)(sec && max_seg > 1 ? sec + off : nullptr);
    if (max_seg > 1) off += al((size_t)B * (kMaxSeg - 1) * a->bnd_ld * 4);
    a->ckpt = (unsigned int*)(sec && max_seg > 1 ? sec + off : nullptr);
    if (max_seg > 1) off += al((size_t)B * kMaxSeg * kMaxCk * 4);
    return off;
}

// Segments per pass for a grid of `blocks` resident blocks: as many as fit
// (all images' tiles of every segment at once), at least kMinSegLines lines
// each, at most `want` (0: kMaxSeg).
void choose_segments(Chain2DArgs* a, int64_t blocks, int want) {
    const int cap = want > 0 ? std::min(want, kMaxSeg) : kMaxSeg;
    auto pick = [&](int L, int tiles, int* nseg, int* seglen) {
        *nseg = 1;
        *seglen = L;
        if (a->max_seg <= 1 || a->B > kMaxSegImages) return;
        int S = (int)std::min<int64_t>(cap, blocks / ((int64_t)a->B * tiles));
        S = std::min(S, L / kMinSegLines);
        if (S < 2) return;
        const int len = ((L + S - 1) / S + kCh - 1) / kCh * kCh;
        *seglen = len;
        *nseg = (L + len - 1) / len;
        if (*nseg < 2) { *nseg = 1; *seglen = L; }
    };
    pick(a->H, a->tiles_v, &a->nseg_v, &a->seglen_v);
    pick(a->W, a->tiles_h, &a->nseg_h, &a->seglen_h);
}

}  // namespace

size_t chain2d_workspace_bytes(int64_t B, int64_t C, int64_t H, int64_t W,
                               const fgx_options* opt) {
    Chain2DArgs a;
    size_t xbytes = 0;
    const size_t sec = fill_chain_args(&a, nullptr, nullptr, nullptr, nullptr, B, C, H, W, 1.0f,
                                       0.5f, 1, opt, nullptr, nullptr, nullptr, &xbytes, kMaxSeg);
    return kHeaderBytes + xbytes + sec;
}

int run_chain2d(const float* image, const float* mask, float* dist, uint8_t* codes, int64_t B,
                int64_t C, int64_t H, int64_t W, float v, float lambda, int iterations,
                void* workspace, size_t ws_bytes, const fgx_options* opt, int sms, void* stream,
                int64_t nimg) {
    Chain2DArgs a;
    char* p = (char*)workspace;
    size_t xbytes = 0;
    fill_chain_args(&a, image, mask, dist, codes, B, C, H, W, v, lambda, iterations, opt, nullptr,
                    nullptr, nullptr, &xbytes, kMaxSeg);
    const size_t need = kHeaderBytes + xbytes +
                        fill_chain_args(&a, image, mask, dist, codes, B, C, H, W, v, lambda,
                                        iterations, opt, p, p + kHeaderBytes,
                                        p + kHeaderBytes + xbytes, &xbytes, kMaxSeg);
    if (ws_bytes < need) return FGX_ERR_WORKSPACE;
    if (nimg > 0) a.nimg = (int)nimg;
    const int max_tiles = a.max_tiles;

    // tensor copies of the producer: boxes of 128 region columns x kCh lines
    // of the distance rows (Dw, Dt) and the cost tables (Ev, Eh: 3 rows per
    // image); region starts are multiples of 4 columns (K and T are)
    {
        const uint32_t box[3] = {(uint32_t)kRegion, (uint32_t)kCh, 1};
        const uint64_t Bn = (uint64_t)B, Wp = (uint64_t)a.Wp, Hp = (uint64_t)a.Hp;
        const uint64_t dw[3] = {Wp, (uint64_t)H, Bn}, dt[3] = {Hp, (uint64_t)W, Bn};
        const uint64_t ev[3] = {Wp, (uint64_t)H, 3 * Bn}, eh[3] = {Hp, (uint64_t)W, 3 * Bn};
        a.tma = encode_map_f32(&a.tmap[0], a.Dw, 3, dw, box, true) &&
                encode_map_f32(&a.tmap[1], a.Dt, 3, dt, box, true) &&
                (!a.table || (encode_map_f32(&a.tmap[2], a.Ev, 3, ev, box, true) &&
                              encode_map_f32(&a.tmap[3], a.Eh, 3, eh, box, true)));
    }
    const size_t smem = sizeof(TileSmem);
    auto kernel = codes ? (a.tma ? chain2d_kernel<true, true> : chain2d_kernel<true, false>)
                        : (a.tma ? chain2d_kernel<false, true> : chain2d_kernel<false, false>);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlockThreads,
                                                      smem) != cudaSuccess || per_sm < 1)
        return FGX_ERR_CUDA;
    // one tile per block: as many blocks as the tiles of all images, or as
    // many as fit (images then run in waves)
    int64_t grid = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    // speculative segments: by default one block per SM; a forced count may
    // use every resident block.  Not with codes: a re-run over speculative
    // values would take a value already reached for one kept, so the codes
    // variant runs each pass as one chain.
    const int want = opt ? opt->segments : 0;
    if (!codes) choose_segments(&a, want > 0 ? grid : std::min<int64_t>(grid, sms), want);
    const int64_t seg_blocks = std::max<int64_t>((int64_t)a.nseg_v * a.tiles_v,
                                                 (int64_t)a.nseg_h * a.tiles_h);
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, B * std::max<int64_t>(max_tiles,
                                                                               seg_blocks)));
    if (grid < max_tiles) return FGX_ERR_UNSUPPORTED;
    if (B > 65535 || (a.Hp + kInitTile - 1) / kInitTile > 65535) return FGX_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, kHeaderBytes + xbytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    if (iterations > 0) {
        const dim3 ig((unsigned)((a.Wp + kInitTile - 1) / kInitTile),
                      (unsigned)((a.Hp + kInitTile - 1) / kInitTile), (unsigned)B);
        if (C == 1) chain2d_init_kernel<1><<<ig, dim3(32, 8), 0, s>>>(a);
        else if (C == 2) chain2d_init_kernel<2><<<ig, dim3(32, 8), 0, s>>>(a);
        else if (C == 3) chain2d_init_kernel<3><<<ig, dim3(32, 8), 0, s>>>(a);
        else if (C == 4) chain2d_init_kernel<4><<<ig, dim3(32, 8), 0, s>>>(a);
        else chain2d_init_kernel<0><<<ig, dim3(32, 8), 0, s>>>(a);
        if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlockThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

// ---------------------------------------------------- batched 2D instances ----

size_t chain2d_desc_size() { return sizeof(Chain2DArgs); }

size_t chain2d_instance_desc(void* desc, const fgx_instance& it, const fgx_options* opt,
                             char* hdr, char* xb, char* sec, size_t* xbytes, int* tiles_v,
                             int* tiles_h) {
    Chain2DArgs a;
    const size_t n = fill_chain_args(&a, it.image, it.mask, it.dist, nullptr, 1, it.channels,
                                     it.H, it.W, it.v, it.lambda, it.iterations, opt, hdr, xb,
                                     sec, xbytes, 1);
    if (desc) std::memcpy(desc, &a, sizeof(a));
    *tiles_v = a.tiles_v;
    *tiles_h = a.tiles_h;
    return n;
}

int chain2d_batched_geometry(int sms, const fgx_options* opt, int* grid, size_t* smem) {
    *smem = sizeof(TileSmem);
    if (cudaFuncSetAttribute(chain2d_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)*smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain2d_batched_kernel,
                                                      kBlockThreads, *smem) != cudaSuccess ||
        per_sm < 1)
        return FGX_ERR_CUDA;
    int64_t g = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) g = std::min<int64_t>(g, opt->max_blocks);
    *grid = (int)std::max<int64_t>(1, g);
    return FGX_OK;
}

int launch_chain2d_batched(const void* desc, int n, int init_channels, int max_wp, int max_hp,
                           int rounds, const int* round_waves, const int* wave_items, int grid,
                           char* hdr, long long timeout_ns, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    const Chain2DArgs* d = (const Chain2DArgs*)desc;
    const dim3 ig((unsigned)((max_wp + kInitTile - 1) / kInitTile),
                  (unsigned)((max_hp + kInitTile - 1) / kInitTile), (unsigned)n);
    switch (init_channels) {
        case 1: chain2d_init_batched_kernel<1><<<ig, dim3(32, 8), 0, s>>>(d); break;
        case 2: chain2d_init_batched_kernel<2><<<ig, dim3(32, 8), 0, s>>>(d); break;
        case 3: chain2d_init_batched_kernel<3><<<ig, dim3(32, 8), 0, s>>>(d); break;
        case 4: chain2d_init_batched_kernel<4><<<ig, dim3(32, 8), 0, s>>>(d); break;
        default: chain2d_init_batched_kernel<0><<<ig, dim3(32, 8), 0, s>>>(d); break;
    }
    if (cudaGetLastError() != cudaSuccess) return FGX_ERR_CUDA;
    Chain2DBatch bt;
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
    cfg.blockDim = dim3(kBlockThreads);
    cfg.dynamicSmemBytes = sizeof(TileSmem);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, chain2d_batched_kernel, bt) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
