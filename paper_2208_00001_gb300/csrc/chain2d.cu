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
// Work decomposition.  One cooperative persistent launch.  Each warp owns a
// tile of T columns of one line plus a ring of K columns on each side
// (T + 2K = 128, four columns per lane).  Per line a lane reads its prefetched
// slice of the previous-line distances, costs and old values, gets the two
// neighbouring columns across lanes by shuffle and applies the min-plus
// update; the dependency cone shrinks the valid part of the ring by one column
// per line, so after K lines the owned columns are exact.  Every K lines a
// warp publishes the 2K owned columns its neighbours need as 64-bit words
// (value, tag) and polls the neighbours' words until the tags match (bounded
// wait); the ring is then refreshed.  Rows are prefetched kStages lines ahead
// with cp.async.  Passes are separated by a grid barrier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {

namespace {

constexpr int kWarps = 2;              // warps per thread block
constexpr int kStages = 16;            // prefetch depth in lines
constexpr int kRegion = 128;           // columns per warp (4 per lane)
constexpr int kMaxRing = 48;           // words per exchanged strip
constexpr int kStageDepth = 32;        // lines per transposed-output flush
#define kInf __int_as_float(0x7f800000)

struct Chain2DArgs {
    const float* image;  // [B][C][H][W]
    const float* mask;   // [B][H][W]
    float* dist;         // [B][H][W]
    int B, C, H, W, Wp, Hp;
    float v, lambda;
    int iterations;
    int table;           // 1: cost tables, 0: constant costs (lambda = 0)
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
};

using namespace dev;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned int sa = (unsigned int)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Cost of the undirected edge between a and b (same channel stride n), in the
// fixed arithmetic order: di2 = sum_ch (I(a)-I(b))^2, c = sqrt(t + lambda*di2).
__device__ __forceinline__ float edge_cost(const float* ia, const float* ib, int C, int64_t n,
                                           float t, float lam) {
    float di2 = 0.0f;
    for (int ch = 0; ch < C; ++ch) {
        const float d = __fsub_rn(__ldg(ia + ch * n), __ldg(ib + ch * n));
        di2 = __fadd_rn(di2, __fmul_rn(d, d));
    }
    return __fsqrt_rn(__fadd_rn(t, __fmul_rn(lam, di2)));
}

struct WarpSmem {
    float D[kStages][kRegion];
    float E[kStages][3][kRegion];
    float stage[kRegion][kStageDepth + 1];  // transposed-output staging [owned col][line]
};

// One warp sweeps one tile of one pass.  Returns false once the device status
// records a failure (the warp then skips the rest of its work).
template <bool fwd, bool table>
__device__ bool chain_tile(const Chain2DArgs& a, int t_app, int pass, int b, int tile,
                           WarpSmem& sm) {
    const int lane = threadIdx.x & 31;
    const bool vert = pass < 2;          // rows of Dw (TB/BT) or rows of Dt (LR/RL)
    const int L = vert ? a.H : a.W;       // number of lines
    const int Q = vert ? a.W : a.H;       // line length
    const int ld = vert ? a.Wp : a.Hp;    // row stride of the source array
    const int ntiles = vert ? a.tiles_v : a.tiles_h;
    const bool multi = ntiles > 1;
    const int K = multi ? a.K : 0;
    const int T = multi ? a.T : Q;
    const int q0 = multi ? tile * T : 0;
    const int q1 = min(Q, q0 + T);
    const int r0 = q0 - K;
    const int c0 = r0 + 4 * lane;
    const float* src = vert ? a.Dw + (int64_t)b * a.H * a.Wp : a.Dt + (int64_t)b * a.W * a.Hp;
    const float* E = vert ? a.Ev + (int64_t)b * 3 * a.H * a.Wp : a.Eh + (int64_t)b * 3 * a.W * a.Hp;
    const int64_t eplane = (int64_t)L * ld;
    const float tc0 = vert ? a.cv[0] : a.chh[0];
    const float tc1 = vert ? a.cv[1] : a.chh[1];
    const float tc2 = vert ? a.cv[2] : a.chh[2];
    // output
    const bool transposed_out = !fwd;  // BT -> Dt, RL -> Dw or dist
    const bool last_rl = (pass == 3) && (t_app == a.iterations * 4 - 1);
    float* out;
    int out_ld;
    if (pass == 0) { out = a.Dw + (int64_t)b * a.H * a.Wp; out_ld = a.Wp; }
    else if (pass == 1) { out = a.Dt + (int64_t)b * a.W * a.Hp; out_ld = a.Hp; }
    else if (pass == 2) { out = a.Dt + (int64_t)b * a.W * a.Hp; out_ld = a.Hp; }
    else if (last_rl) { out = a.dist + (int64_t)b * a.H * a.W; out_ld = a.W; }
    else { out = a.Dw + (int64_t)b * a.H * a.Wp; out_ld = a.Wp; }

    bool valid[4], owned[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = c0 + i;
        valid[i] = c >= 0 && c < Q;
        owned[i] = c >= q0 && c < q1;
    }
    // each lane prefetches (and later reads) only its own 16-byte slice of
    // every row, so no cross-lane synchronisation is needed for the ring
    const bool lane_loads = (c0 >= 0) && (c0 < Q);

    auto line_of = [&](int s) { return fwd ? s : (L - 1 - s); };

    // prefetch cursors: the next item to fetch, its source rows and stage
    const int64_t step = fwd ? (int64_t)ld : -(int64_t)ld;
    const float* pf_d = src + (int64_t)line_of(0) * ld + c0;
    const float* pf_e = E + (int64_t)(fwd ? 0 : (L - 2)) * ld + c0 - step;  // edge row of item 0 (unused)
    int pf_next = 0;
    auto prefetch = [&]() {
        const int s = pf_next++;
        if (s < L && lane_loads) {
            const int slot = s & (kStages - 1);
            cp_async16(&sm.D[slot][4 * lane], pf_d);
            if (table && s >= 1) {
                cp_async16(&sm.E[slot][0][4 * lane], pf_e);
                cp_async16(&sm.E[slot][1][4 * lane], pf_e + eplane);
                cp_async16(&sm.E[slot][2][4 * lane], pf_e + 2 * eplane);
            }
        }
        pf_d += step;
        pf_e += step;
        cp_async_commit();  // one group per item, possibly empty
    };

    // Registers of one line: old values and the parent costs of the lane's
    // four columns (cost shifts across lanes done at load time, off the chain).
    struct LineRegs {
        float dold[4];
        float cst[3][4];
    };
    auto load_line = [&](int s, LineRegs& r) {
        const int slot = s & (kStages - 1);
        const float4 o4 = *reinterpret_cast<const float4*>(&sm.D[slot][4 * lane]);
        r.dold[0] = o4.x; r.dold[1] = o4.y; r.dold[2] = o4.z; r.dold[3] = o4.w;
        if (s == 0) return;
        if constexpr (table) {
            float e[3][4];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 v4 = *reinterpret_cast<const float4*>(&sm.E[slot][k][4 * lane]);
                e[k][0] = v4.x; e[k][1] = v4.y; e[k][2] = v4.z; e[k][3] = v4.w;
            }
            if constexpr (fwd) {
                // parent at column c+k-1 of the previous line: edge E_{2-k}[line-1][c+k-1]
                const float e2l = __shfl_up_sync(0xffffffffu, e[2][3], 1);
                const float e0r = __shfl_down_sync(0xffffffffu, e[0][0], 1);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    r.cst[0][i] = (i == 0) ? e2l : e[2][i - 1];
                    r.cst[1][i] = e[1][i];
                    r.cst[2][i] = (i == 3) ? e0r : e[0][i + 1];
                }
            } else {
                // parent at column c+k-1 of line+1: edge E_k[line][c]
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int i = 0; i < 4; ++i) r.cst[k][i] = e[k][i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                r.cst[0][i] = tc0;
                r.cst[1][i] = tc1;
                r.cst[2][i] = tc2;
            }
        }
    };

    // items 0 .. kStages-2 in flight; item s is complete once at most
    // kStages-2 younger groups are pending
    for (int s = 0; s < kStages - 1; ++s) prefetch();

    unsigned long long* xb = a.xbuf + ((int64_t)b * a.max_tiles + tile) * (4 * kMaxRing);
    const unsigned int tag_base = ((unsigned int)(t_app + 1)) << 16;

    float dp[4];
    bool alive = true;
    int stage_start = 1;  // first step whose output sits in the staging buffer
    LineRegs cur, nxt;

    // line 0 of the sweep: not updated; it seeds the chain
    cp_async_wait<kStages - 2>();
    load_line(0, cur);
#pragma unroll
    for (int i = 0; i < 4; ++i) dp[i] = valid[i] ? cur.dold[i] : kInf;
    if (transposed_out) {
        const int x0 = line_of(0);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (owned[i]) out[(int64_t)(c0 + i) * out_ld + x0] = dp[i];
    }
    prefetch();
    if (L > 1) {
        cp_async_wait<kStages - 2>();
        load_line(1, cur);
    }
    int s = 1;
    int next_refresh = multi ? 1 + K : L;  // first step of the next exchange block
    int blk = 0;                           // exchange blocks finished so far
    int x = line_of(1);
    float* out_row = out + (int64_t)x * out_ld + c0;  // normal output cursor
    const int64_t out_step = fwd ? (int64_t)out_ld : -(int64_t)out_ld;
#pragma unroll 2
    for (; s < L; ++s, x += fwd ? 1 : -1, out_row += out_step) {
        // keep the pipeline full, then fetch the next line's registers so that
        // their shared-memory latency overlaps this line's chain
        prefetch();
        if (s + 1 < L) {
            cp_async_wait<kStages - 2>();
            load_line(s + 1, nxt);
        }
        // ring refresh every K lines (multi-tile passes)
        if (s == next_refresh) {
            next_refresh += K;
            const unsigned int tg = tag_base | (unsigned int)(blk + 1);
            const int par = blk & 1;
            unsigned long long* mine = xb + par * (2 * kMaxRing);
            // publish: left-facing strip = owned columns [q0, q0+K), right-facing
            // strip = owned columns [q0+T-K, q0+T)
            const int rq = q0 + T - K;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int c = c0 + i;
                const unsigned long long w =
                    ((unsigned long long)tg << 32) | (unsigned int)__float_as_uint(dp[i]);
                if (c >= q0 && c < q0 + K) st_relaxed_u64(mine + (c - q0), w);
                if (c >= rq && c < q0 + T) st_relaxed_u64(mine + kMaxRing + (c - rq), w);
            }
            // ring lanes: [q0-K, q0) and [q0+T, q0+T+K); lanes beyond the right
            // ring (when T + 2K < 128) hold columns outside the cone and are
            // never refreshed
            const bool left_ring = c0 < q0 && tile > 0;
            const bool right_ring = c0 >= q0 + T && c0 < q0 + T + K && tile + 1 < ntiles;
            const unsigned long long* nb = nullptr;
            int base = 0;
            if (left_ring) {
                nb = a.xbuf + ((int64_t)b * a.max_tiles + tile - 1) * (4 * kMaxRing) +
                     par * (2 * kMaxRing) + kMaxRing;  // left neighbour's right-facing strip
                base = c0 - (q0 - K);
            } else if (right_ring) {
                nb = a.xbuf + ((int64_t)b * a.max_tiles + tile + 1) * (4 * kMaxRing) +
                     par * (2 * kMaxRing);             // right neighbour's left-facing strip
                base = c0 - (q0 + T);
            }
            float got[4] = {dp[0], dp[1], dp[2], dp[3]};
            bool ok = (nb == nullptr);
            const long long t0 = gtimer();
            for (;;) {
                if (!ok) {
                    bool all = true;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const unsigned long long w = ld_relaxed_u64(nb + base + i);
                        if ((unsigned int)(w >> 32) != tg) all = false;
                        got[i] = __uint_as_float((unsigned int)w);
                    }
                    ok = all;
                }
                if (__all_sync(0xffffffffu, ok)) break;
                int fail = 0;
                if (lane == 0) {
                    if (status_of(a.status) != 0) fail = 1;
                    else if (gtimer() - t0 > a.timeout_ns) {
                        record_timeout(a.status);
                        fail = 1;
                    }
                }
                if (__shfl_sync(0xffffffffu, fail, 0)) { alive = false; break; }
                __nanosleep(20);
            }
            if (!alive) break;
            if (nb) {
#pragma unroll
                for (int i = 0; i < 4; ++i) dp[i] = valid[i] ? got[i] : kInf;
            }
            ++blk;
        }
        // min-plus update; the shuffled neighbours enter last so the chain
        // through the lanes is shuffle -> add -> min
        float left = __shfl_up_sync(0xffffffffu, dp[3], 1);
        float right = __shfl_down_sync(0xffffffffu, dp[0], 1);
        if (lane == 0) left = kInf;
        if (lane == 31) right = kInf;
        float nd[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float best = cur.dold[i];
            // parents in the lane's own registers first
            if (i > 0) best = fminf(best, __fadd_rn(dp[i - 1], cur.cst[0][i]));
            best = fminf(best, __fadd_rn(dp[i], cur.cst[1][i]));
            if (i < 3) best = fminf(best, __fadd_rn(dp[i + 1], cur.cst[2][i]));
            if (i == 0) best = fminf(best, __fadd_rn(left, cur.cst[0][0]));
            if (i == 3) best = fminf(best, __fadd_rn(right, cur.cst[2][3]));
            nd[i] = valid[i] ? best : kInf;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) dp[i] = nd[i];
        // owned outputs
        if (!transposed_out) {
            if (owned[0] && owned[3]) {
                *reinterpret_cast<float4*>(out_row) = make_float4(nd[0], nd[1], nd[2], nd[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (owned[i]) out_row[i] = nd[i];
            }
        } else {
            const int j = s - stage_start;  // line slot in the staging buffer
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (owned[i]) sm.stage[c0 + i - q0][j] = nd[i];
            if (j + 1 == kStageDepth || s == L - 1) {
                __syncwarp();
                const int nl = j + 1;
                const int ncol = q1 - q0;
                // slot jj holds step stage_start + jj; consecutive lanes write
                // consecutive lines of one owned column (one output row)
                if (nl == 32) {
                    const int xx = line_of(stage_start + lane);
                    for (int col = 0; col < ncol; ++col)
                        out[(int64_t)(q0 + col) * out_ld + xx] = sm.stage[col][lane];
                } else {
                    for (int e = lane; e < ncol * nl; e += 32) {
                        const int col = e / nl, jj = e % nl;
                        const int xx = line_of(stage_start + jj);
                        out[(int64_t)(q0 + col) * out_ld + xx] = sm.stage[col][jj];
                    }
                }
                __syncwarp();
                stage_start = s + 1;
            }
        }
        cur = nxt;
    }
    // no copy may still target the staging ring when the next tile starts
    cp_async_wait<0>();
    __syncwarp();
    return alive;
}

__global__ void __launch_bounds__(kWarps * 32, 1) chain2d_kernel(const Chain2DArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem& sm = reinterpret_cast<WarpSmem*>(smem_raw)[threadIdx.x >> 5];
    const int64_t N = (int64_t)a.H * a.W;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int epoch = 1;
    // D0 = v * M (and the cost tables)
    if (a.iterations == 0) {
        for (int64_t i = tid; i < a.B * N; i += nthreads) a.dist[i] = __fmul_rn(a.v, a.mask[i]);
        return;
    }
    for (int64_t i = tid; i < a.B * N; i += nthreads) {
        const int64_t b = i / N, r = i % N;
        const int h = (int)(r / a.W), w = (int)(r % a.W);
        a.Dw[(b * a.H + h) * a.Wp + w] = __fmul_rn(a.v, a.mask[i]);
    }
    if (a.table) {
        // Ev[k][h][w]: edge (h, w) - (h+1, w+k-1);  Eh[k][w][h]: edge (h, w) - (h+k-1, w+1)
        for (int64_t i = tid; i < a.B * N; i += nthreads) {
            const int64_t b = i / N, r = i % N;
            const int h = (int)(r / a.W), w = (int)(r % a.W);
            const float* img = a.image + b * a.C * N;
            const float* self = img + (int64_t)h * a.W + w;
            for (int k = 0; k < 3; ++k) {
                float cv = kInf, ch = kInf;
                const int wn = w + k - 1, hn = h + k - 1;
                if (h + 1 < a.H && wn >= 0 && wn < a.W)
                    cv = edge_cost(img + (int64_t)(h + 1) * a.W + wn, self, a.C, N, a.tv[k], a.lambda);
                if (w + 1 < a.W && hn >= 0 && hn < a.H)
                    ch = edge_cost(img + (int64_t)hn * a.W + w + 1, self, a.C, N, a.th[k], a.lambda);
                a.Ev[((b * 3 + k) * a.H + h) * a.Wp + w] = cv;
                a.Eh[((b * 3 + k) * a.W + w) * a.Hp + h] = ch;
            }
        }
    }
    unsigned long long* timeline = (unsigned long long*)((char*)a.status + 128);
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[0] = (unsigned long long)gtimer();
    bool alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
    if (blockIdx.x == 0 && threadIdx.x == 0) timeline[1] = (unsigned long long)gtimer();
    const int gwarp = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * kWarps;
    const int napps = a.iterations * 4;
    for (int t_app = 0; t_app < napps && alive; ++t_app) {
        const int pass = t_app % 4;
        const int ntiles = pass < 2 ? a.tiles_v : a.tiles_h;
        const int per_wave = nwarps / ntiles;
        const int nwaves = (a.B + per_wave - 1) / per_wave;
        bool ok = true;
        for (int wv = 0; wv < nwaves && ok; ++wv) {
            if (gwarp < per_wave * ntiles) {
                const int b = wv * per_wave + gwarp / ntiles;
                if (b < a.B) {
                    const int tile = gwarp % ntiles;
                    const bool fwd = (pass == 0 || pass == 2);
                    if (fwd && a.table) ok = chain_tile<true, true>(a, t_app, pass, b, tile, sm);
                    else if (fwd) ok = chain_tile<true, false>(a, t_app, pass, b, tile, sm);
                    else if (a.table) ok = chain_tile<false, true>(a, t_app, pass, b, tile, sm);
                    else ok = chain_tile<false, false>(a, t_app, pass, b, tile, sm);
                }
            }
        }
        alive = grid_barrier(a.barrier, epoch++, a.status, a.timeout_ns);
        if (blockIdx.x == 0 && threadIdx.x == 0 && t_app + 2 < 16)
            timeline[t_app + 2] = (unsigned long long)gtimer();
    }
}

}  // namespace

// ---------------------------------------------------------------- host ----

size_t chain2d_workspace_bytes(int64_t B, int64_t C, int64_t H, int64_t W, int tiles) {
    (void)C;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const int64_t Wp = (W + 3) & ~int64_t(3), Hp = (H + 3) & ~int64_t(3);
    size_t n = kHeaderBytes;
    n += al((size_t)B * tiles * 4 * kMaxRing * 8);
    n += al((size_t)B * H * Wp * 4);
    n += al((size_t)B * W * Hp * 4);
    n += al((size_t)B * 3 * H * Wp * 4);
    n += al((size_t)B * 3 * W * Hp * 4);
    return n;
}

int chain2d_geometry(int64_t H, int64_t W, const fgx_options* opt, int* K, int* T, int* tv,
                     int* th) {
    int k = (opt && opt->tile_lines) ? opt->tile_lines : 40;
    k = std::max(4, std::min(kMaxRing, (k + 3) & ~3));
    int t = kRegion - 2 * k;
    if (opt && opt->tile_width) t = std::min(t, std::max(4, opt->tile_width & ~3));
    if (t < k) { k = std::max(4, (kRegion / 3) & ~3); t = kRegion - 2 * k; }
    *K = k;
    *T = t;
    // a line that fits one warp region is one tile, unless a tile width is forced
    const int64_t single = (opt && opt->tile_width) ? t : kRegion;
    *tv = W <= single ? 1 : (int)((W + t - 1) / t);
    *th = H <= single ? 1 : (int)((H + t - 1) / t);
    return FGX_OK;
}

int run_chain2d(const float* image, const float* mask, float* dist, int64_t B, int64_t C,
                int64_t H, int64_t W, float v, float lambda, int iterations, void* workspace,
                size_t ws_bytes, const fgx_options* opt, int sms, void* stream) {
    Chain2DArgs a;
    std::memset(&a, 0, sizeof(a));
    int K, T, tv, th;
    chain2d_geometry(H, W, opt, &K, &T, &tv, &th);
    const int max_tiles = std::max(tv, th);
    const size_t need = chain2d_workspace_bytes(B, C, H, W, max_tiles);
    if (ws_bytes < need) return FGX_ERR_WORKSPACE;
    a.image = image;
    a.mask = mask;
    a.dist = dist;
    a.B = (int)B;
    a.C = (int)C;
    a.H = (int)H;
    a.W = (int)W;
    a.Wp = (int)((W + 3) & ~int64_t(3));
    a.Hp = (int)((H + 3) & ~int64_t(3));
    a.v = v;
    a.lambda = lambda;
    a.iterations = iterations;
    a.table = lambda != 0.0f;
    const float unit[3] = {1.f, 1.f, 1.f};
    float t9[9];
    pass_offsets_t(2, 1, unit, lambda, t9);  // pass along H: offsets along W
    for (int k = 0; k < 3; ++k) { a.tv[k] = t9[k]; a.cv[k] = std::sqrt(t9[k]); }
    pass_offsets_t(2, 2, unit, lambda, t9);  // pass along W: offsets along H
    for (int k = 0; k < 3; ++k) { a.th[k] = t9[k]; a.chh[k] = std::sqrt(t9[k]); }
    a.K = K;
    a.T = T;
    a.tiles_v = tv;
    a.tiles_h = th;
    a.max_tiles = max_tiles;
    a.timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) * 1000000LL;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    char* p = (char*)workspace;
    a.status = (int*)p;
    a.barrier = (unsigned int*)(p + 64);
    size_t off = kHeaderBytes;
    a.xbuf = (unsigned long long*)(p + off);
    const size_t xbytes = al((size_t)B * max_tiles * 4 * kMaxRing * 8);
    off += xbytes;
    a.Dw = (float*)(p + off);
    off += al((size_t)B * H * a.Wp * 4);
    a.Dt = (float*)(p + off);
    off += al((size_t)B * W * a.Hp * 4);
    a.Ev = (float*)(p + off);
    off += al((size_t)B * 3 * H * a.Wp * 4);
    a.Eh = (float*)(p + off);

    const size_t smem = sizeof(WarpSmem) * kWarps;
    if (cudaFuncSetAttribute(chain2d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return FGX_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain2d_kernel, kWarps * 32,
                                                      smem) != cudaSuccess || per_sm < 1)
        return FGX_ERR_CUDA;
    int64_t grid = (int64_t)per_sm * sms;
    if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
    const int64_t want = (B * max_tiles + kWarps - 1) / kWarps;
    grid = std::max<int64_t>(1, std::min<int64_t>(grid, std::max<int64_t>(want, sms)));
    if (grid * kWarps < max_tiles) return FGX_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(workspace, 0, kHeaderBytes + xbytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kWarps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, chain2d_kernel, a) != cudaSuccess) return FGX_ERR_CUDA;
    return FGX_OK;
}

}  // namespace fgx
