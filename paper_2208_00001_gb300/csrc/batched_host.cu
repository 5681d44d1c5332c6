// Batched launch of instances of uneven shapes (2D and 3D mixed): host-side
// planning of the work lists and the C ABI entry points.
//
// Every instance runs the same raster-scan schedule as a single call (4 or 6
// passes per iteration, FastGeodis Implementation section).  2D instances
// run on the line-chain kernel, 3D instances on the plane-tile kernel, the
// rest (tile options, more channels than it stages) on the tiled engine: up
// to three persistent launches.  In each, instances advance one pass
// application per round; a round packs whole instances into waves of
// co-resident thread blocks (first fit), so the tiles of an instance that
// wait on one another always run together; rounds are separated by a grid
// barrier inside the launch.
//
// The line-chain and plane-tile launches of a batch holding both run at the
// same time: the 2D one on a side stream forked from the caller's stream,
// each with one block per SM of a disjoint share.  Their blocks never share
// an SM (neither kernel leaves room for a block of the other) and together
// they number at most the SM count, so every block of both launches is
// resident at once and neither launch waits for SMs the other holds; each
// waits only on its own blocks, with its own grid-barrier counter.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fgx_internal.h"

namespace fgx {
namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct Schedule {
    // tiled engine (3D instances, and 2D instances with no iteration)
    std::vector<InstDesc> desc;
    std::vector<int> round_waves;
    std::vector<int> wave_items;
    int grid = 0, rounds = 0, region = 1, kmax = 1;
    size_t smem = 0, flags_bytes = 0;
    size_t desc_off = 0, waves_off = 0, items_off = 0, total = 0;
    long long timeout_ns = 0;
    // line-chain kernel (2D instances)
    std::vector<int> c_index;                 // instance index of each chain instance
    std::vector<int> c_tiles_v, c_tiles_h;
    std::vector<size_t> c_xoff, c_soff;       // exchange words / buffers, relative
    std::vector<int> c_round_waves, c_wave_items;
    int c_grid = 0, c_rounds = 0, c_channels = 0, c_max_wp = 0, c_max_hp = 0;
    size_t c_smem = 0, c_xbuf_bytes = 0, c_sec_bytes = 0;
    size_t c_xbuf_off = 0, c_desc_off = 0, c_waves_off = 0, c_items_off = 0, c_sec_off = 0;
    // plane-tile kernel (3D instances)
    std::vector<int> v_index;
    std::vector<std::vector<int>> v_tiles;
    std::vector<SweepArgs> v_args;
    std::vector<size_t> v_xoff, v_woff;
    std::vector<int> v_round_waves, v_wave_items;
    int v_grid = 0, v_rounds = 0, v_ci = 0, v_max_tiles = 0;
    int sms = 0;
    // line-chain and plane-tile launches at the same time: SM shares
    bool concurrent = false;
    int c_sms = 0, v_sms = 0;
    size_t v_smem = 0, v_xbuf_bytes = 0, v_work_bytes = 0, v_work_off = 0;
    size_t v_flag_off = 0, v_xbuf_off = 0, v_desc_off = 0, v_waves_off = 0, v_items_off = 0;
};

// Packing of whole instances into waves of `grid` blocks, one round per pass
// application; tiles(i, r) is instance i's tile count in round r (0 once the
// instance is done) and lines(i, r) its number of line steps.  A wave lasts
// about as long as its longest instance, so the instances go in order of
// decreasing line count (then tile count) into the first wave with room:
// long instances share waves and short ones fill the gaps.
template <class Tiles, class Lines>
void pack_rounds(int n, int rounds, int grid, Tiles tiles, Lines lines,
                 std::vector<int>* round_waves, std::vector<int>* wave_items) {
    round_waves->assign(1, 0);
    wave_items->clear();
    std::vector<int> order;
    for (int r = 0; r < rounds; ++r) {
        order.clear();
        for (int i = 0; i < n; ++i)
            if (tiles(i, r) > 0) order.push_back(i);
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            const int64_t lx = lines(x, r), ly = lines(y, r);
            if (lx != ly) return lx > ly;
            return tiles(x, r) > tiles(y, r);
        });
        std::vector<int> used;                                   // blocks used per wave
        std::vector<std::vector<std::pair<int, int>>> members;  // (instance, first block)
        for (int i : order) {
            const int nt = tiles(i, r);
            size_t w = 0;
            while (w < used.size() && used[w] + nt > grid) ++w;
            if (w == used.size()) {
                used.push_back(0);
                members.emplace_back();
            }
            members[w].push_back({i, used[w]});
            used[w] += nt;
        }
        for (size_t w = 0; w < used.size(); ++w) {
            const size_t base = wave_items->size();
            wave_items->resize(base + grid, -1);
            for (auto& m : members[w])
                for (int t = 0; t < tiles(m.first, r); ++t)
                    (*wave_items)[base + m.second + t] = (m.first << 16) | t;
        }
        round_waves->push_back(round_waves->back() + (int)used.size());
    }
}

int check_instance(const fgx_instance& it) {
    if (it.ndim != 2 && it.ndim != 3) return FGX_ERR_ARG;
    if (it.channels < 1 || it.channels > 64) return it.channels < 1 ? FGX_ERR_SHAPE
                                                                    : FGX_ERR_UNSUPPORTED;
    if (it.D < 0 || it.H < 0 || it.W < 0) return FGX_ERR_SHAPE;
    if (it.ndim == 2 && it.D != 1) return FGX_ERR_SHAPE;
    if (!(std::isfinite(it.v) && it.v > 0.f)) return FGX_ERR_ARG;
    if (!(it.lambda >= 0.f && it.lambda <= 1.f)) return FGX_ERR_ARG;
    if (it.iterations < 0) return FGX_ERR_ARG;
    if (it.ndim == 3)
        for (int k = 0; k < 3; ++k)
            if (!(std::isfinite(it.spacing[k]) && it.spacing[k] > 0.f)) return FGX_ERR_ARG;
    return FGX_OK;
}

// Options of the 3D instances of a batch: tile_lines and tile_width shape the
// 2D line tiles (an autotuned batch carries them), so the 3D instances keep
// the plane-tile kernel's own geometry; tile_height, a 3D tile extent, sends
// them to the tiled engine with all three.
const fgx_options* options_3d(const fgx_options* opt, fgx_options* buf) {
    if (!opt || opt->tile_height) return opt;
    *buf = *opt;
    buf->tile_lines = 0;
    buf->tile_width = 0;
    return buf;
}

// SMs for the line-chain launch when it runs beside the plane-tile launch:
// the share of the estimated work of the 2D part, counted in tile steps (one
// line of a 2D tile, one plane of a 3D tile) weighted 0.3 : 1.7, the ratio
// that put the split of the 64 + 16 instance batch (2D sides 128..1024, 3D
// 64..192) near its measured best on GB300.  An estimate: the batch
// autotuner times shares around it.
int split_estimate(const Schedule& S, const fgx_instance* items, int sms) {
    double w2 = 0.0, w3 = 0.0;
    for (size_t k = 0; k < S.c_index.size(); ++k) {
        const fgx_instance& it = items[S.c_index[k]];
        w2 += 2.0 * it.iterations * ((double)S.c_tiles_v[k] * it.H + (double)S.c_tiles_h[k] * it.W);
    }
    for (size_t k = 0; k < S.v_index.size(); ++k)
        for (int r = 0; r < kMaxPasses; ++r)
            w3 += (double)items[S.v_index[k]].iterations * S.v_tiles[k][r] *
                  (double)S.v_args[k].pass[r].L;
    w2 *= 0.3;
    w3 *= 1.7;
    if (!(w2 + w3 > 0.0)) return sms / 2;
    return (int)std::lround(sms * w2 / (w2 + w3));
}

// Plans the plane tiles of the 3D instances again for `share` SMs (ring
// widths and tile counts); false, with the schedule unchanged, when an
// instance needs more tiles than that.
bool replan_vol3d(const fgx_instance* items, const fgx_options* opt3, int share, Schedule* S) {
    const size_t n = S->v_index.size();
    std::vector<std::vector<int>> tiles(n);
    std::vector<size_t> xoff(n);
    size_t xbytes = 0;
    int max_tiles = 0;
    for (size_t k = 0; k < n; ++k) {
        size_t xb = 0, wb = 0;
        int ci = 0, mt = 0, t[kMaxPasses];
        if (!vol3d_instance_desc(nullptr, items[S->v_index[k]], S->v_args[k], opt3, share, nullptr,
                                 nullptr, nullptr, nullptr, &xb, &wb, &ci, &mt, t))
            return false;
        tiles[k].assign(t, t + kMaxPasses);
        xoff[k] = xbytes;
        xbytes += al256(xb);
        max_tiles = std::max(max_tiles, mt);
    }
    if (max_tiles > share) return false;
    S->v_tiles = tiles;
    S->v_xoff = xoff;
    S->v_xbuf_bytes = xbytes;
    S->v_max_tiles = max_tiles;
    return true;
}

// Builds descriptors and the round/wave work list; pointers are checked only
// when `check_ptrs`.
int build_schedule(const fgx_instance* items, int n, const fgx_options* opt, bool check_ptrs,
                   Schedule* S) {
    if (n < 0 || (n > 0 && !items)) return FGX_ERR_ARG;
    if (n > 32767) return FGX_ERR_UNSUPPORTED;
    fgx_options o3;
    const fgx_options* opt3 = options_3d(opt, &o3);
    int sms = 0;
    int max_tiles_any = 1, flags_total = 0;
    S->desc.clear();
    for (int i = 0; i < n; ++i) {
        const fgx_instance& it = items[i];
        int st = check_instance(it);
        if (st != FGX_OK) return st;
        const int64_t N = it.D * it.H * it.W;
        if (N == 0) continue;
        if (it.ndim == 2 && it.iterations > 0) {
            // line-chain kernel; pointers are checked below
            if (check_ptrs) {
                if (!it.image || !it.mask || !it.dist) return FGX_ERR_ARG;
                if (!device_pointer(it.image) || !device_pointer(it.mask) ||
                    !device_pointer(it.dist))
                    return FGX_ERR_NOT_DEVICE_PTR;
                const char* d = (const char*)it.dist;
                const char* im = (const char*)it.image;
                if (d < im + N * it.channels * 4 && im < d + N * 4) return FGX_ERR_ARG;
            }
            int tv = 0, th = 0;
            size_t xb = 0;
            const size_t sb = chain2d_instance_desc(nullptr, it, opt, nullptr, nullptr, nullptr,
                                                    &xb, &tv, &th);
            if (std::max(tv, th) > 65535) return FGX_ERR_UNSUPPORTED;
            S->c_index.push_back(i);
            S->c_tiles_v.push_back(tv);
            S->c_tiles_h.push_back(th);
            S->c_xoff.push_back(S->c_xbuf_bytes);
            S->c_soff.push_back(S->c_sec_bytes);
            S->c_xbuf_bytes += xb;
            S->c_sec_bytes += sb;
            S->c_rounds = std::max(S->c_rounds, it.iterations * 4);
            S->c_max_wp = std::max<int>(S->c_max_wp, (int)((it.W + 3) & ~int64_t(3)));
            S->c_max_hp = std::max<int>(S->c_max_hp, (int)((it.H + 3) & ~int64_t(3)));
            S->c_channels = S->c_index.size() == 1 ? (int)it.channels
                            : (S->c_channels == it.channels ? S->c_channels : 0);
            continue;
        }
        if (check_ptrs) {
            if (!it.image || !it.mask || !it.dist) return FGX_ERR_ARG;
            if (!device_pointer(it.image) || !device_pointer(it.mask) ||
                !device_pointer(it.dist))
                return FGX_ERR_NOT_DEVICE_PTR;
            const char* d = (const char*)it.dist;
            const char* im = (const char*)it.image;
            if (d < im + N * it.channels * 4 && im < d + N * 4) return FGX_ERR_ARG;
        }
        SweepArgs a;
        st = plan_instance(it.ndim, it.channels, it.D, it.H, it.W, it.spacing, it.lambda,
                           it.ndim == 3 ? opt3 : opt, &a, &sms);
        if (st != FGX_OK) return st;
        if (it.ndim == 3) {
            size_t xb = 0, wb = 0;
            int ci = 0, mt = 0, tiles[kMaxPasses];
            if (vol3d_instance_desc(nullptr, it, a, opt3, sms, nullptr, nullptr, nullptr, nullptr,
                                    &xb, &wb, &ci, &mt, tiles)) {
                if (check_ptrs) {
                    if (!it.image || !it.mask || !it.dist) return FGX_ERR_ARG;
                    if (!device_pointer(it.image) || !device_pointer(it.mask) ||
                        !device_pointer(it.dist))
                        return FGX_ERR_NOT_DEVICE_PTR;
                    const char* d = (const char*)it.dist;
                    const char* im = (const char*)it.image;
                    if (d < im + N * it.channels * 4 && im < d + N * 4) return FGX_ERR_ARG;
                }
                a.timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) *
                               1000000LL;
                S->v_index.push_back(i);
                S->v_tiles.emplace_back(tiles, tiles + kMaxPasses);
                S->v_args.push_back(a);
                S->v_xoff.push_back(S->v_xbuf_bytes);
                S->v_xbuf_bytes += al256(xb);
                S->v_woff.push_back(S->v_work_bytes);
                S->v_work_bytes += al256(wb);
                S->v_ci = std::max(S->v_ci, ci);
                S->v_max_tiles = std::max(S->v_max_tiles, mt);
                S->v_rounds = std::max(S->v_rounds, it.iterations * kMaxPasses);
                continue;
            }
        }
        InstDesc d;
        std::memset(&d, 0, sizeof(d));
        d.image = it.image;
        d.mask = it.mask;
        d.dist = it.dist;
        d.N = N;
        d.C = it.channels;
        d.ndim = it.ndim;
        d.v = it.v;
        d.lambda = it.lambda;
        d.npass = a.npass;
        d.napps = it.iterations * a.npass;
        d.cost_mode = a.cost_mode;
        d.flags_off = flags_total;
        d.region = a.smem_region;
        d.kmax = a.kmax;
        for (int k = 0; k < kMaxPasses; ++k) d.pass[k] = a.pass[k];
        flags_total += a.max_tiles;
        max_tiles_any = std::max(max_tiles_any, a.max_tiles);
        if (a.max_tiles > 65535) return FGX_ERR_UNSUPPORTED;
        S->region = std::max(S->region, a.smem_region);
        S->kmax = std::max(S->kmax, a.kmax);
        S->smem = std::max(S->smem, sweep_smem_bytes(a.cost_mode == kCostConst ? 0 : it.channels,
                                                     a.smem_region, a.kmax));
        S->desc.push_back(d);
        S->timeout_ns = a.timeout_ns;
    }
    if (S->smem > 200 * 1024) return FGX_ERR_UNSUPPORTED;
    if (S->desc.empty()) {
        S->grid = 0;
        S->rounds = 0;
    } else {
        int per_sm = 0;
        int st = batched_max_blocks_per_sm(S->smem, &per_sm);
        if (st != FGX_OK) return st;
        if (per_sm < 1) return FGX_ERR_UNSUPPORTED;
        int64_t grid = (int64_t)per_sm * sms;
        if (opt && opt->max_blocks) grid = std::min<int64_t>(grid, opt->max_blocks);
        if (grid < max_tiles_any) return FGX_ERR_UNSUPPORTED;
        S->grid = (int)grid;
    }
    if (S->timeout_ns == 0)
        S->timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) * 1000000LL;
    // rounds and waves of the engine
    int rounds = 0;
    for (const InstDesc& d : S->desc) rounds = std::max(rounds, d.napps);
    S->rounds = rounds;
    pack_rounds((int)S->desc.size(), rounds, std::max(S->grid, 1),
                [&](int i, int r) {
                    const InstDesc& d = S->desc[i];
                    if (r >= d.napps) return 0;
                    const PassGeom& g = d.pass[r % d.npass];
                    return g.ntp * g.ntq;
                },
                [&](int i, int r) -> int64_t {
                    const InstDesc& d = S->desc[i];
                    return d.pass[r % d.npass].L;
                },
                &S->round_waves, &S->wave_items);
    // line-chain and plane-tile instances together: both launches run at
    // once, each on its own share of the SMs with one block per SM
    S->c_sms = S->v_sms = sms;
    if (!S->c_index.empty() && !S->v_index.empty() && sms > 1 &&
        !(opt && opt->split_sms < 0)) {
        // the largest instance of each launch needs all its tiles resident
        int need2 = 1, need3 = 1;
        for (size_t k = 0; k < S->c_index.size(); ++k)
            need2 = std::max({need2, S->c_tiles_v[k], S->c_tiles_h[k]});
        for (const std::vector<int>& t : S->v_tiles)
            for (int x : t) need3 = std::max(need3, x);
        int s2 = (opt && opt->split_sms > 0) ? opt->split_sms
                                             : split_estimate(*S, items, sms);
        s2 = std::max(need2, std::min(s2, sms - need3));
        if (s2 < sms && replan_vol3d(items, opt3, sms - s2, S)) {
            S->concurrent = true;
            S->c_sms = s2;
            S->v_sms = sms - s2;
        }
    }
    // the plane-tile launch for the 3D instances
    if (!S->v_index.empty()) {
        const int st = vol3d_batched_geometry(S->v_sms, S->v_ci, S->v_ci > kMaxChannels3 ? 1 : 0,
                                              opt, &S->v_grid, &S->v_smem);
        if (st != FGX_OK) return st;
        if (S->concurrent) S->v_grid = std::min(S->v_grid, S->v_sms);
        if (S->v_max_tiles > S->v_grid) return FGX_ERR_UNSUPPORTED;
        pack_rounds((int)S->v_index.size(), S->v_rounds, S->v_grid,
                    [&](int k, int r) {
                        if (r >= items[S->v_index[k]].iterations * kMaxPasses) return 0;
                        return S->v_tiles[k][r % kMaxPasses];
                    },
                    [&](int k, int r) -> int64_t {
                        return S->v_args[k].pass[r % kMaxPasses].L;
                    },
                    &S->v_round_waves, &S->v_wave_items);
        if (S->timeout_ns == 0)
            S->timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) *
                            1000000LL;
    }
    // the line-chain launch for the 2D instances
    if (S->c_channels > 4) S->c_channels = 0;
    if (!S->c_index.empty()) {
        if (sms == 0) {
            const float unit[3] = {1.f, 1.f, 1.f};
            SweepArgs tmp;
            const int st = plan_instance(2, 1, 1, 8, 8, unit, 0.5f, opt, &tmp, &sms);
            if (st != FGX_OK) return st;
        }
        const int st = chain2d_batched_geometry(S->concurrent ? S->c_sms : sms, opt, &S->c_grid,
                                                &S->c_smem);
        if (st != FGX_OK) return st;
        if (S->concurrent) S->c_grid = std::min(S->c_grid, S->c_sms);
        for (size_t k = 0; k < S->c_index.size(); ++k)
            if (std::max(S->c_tiles_v[k], S->c_tiles_h[k]) > S->c_grid) return FGX_ERR_UNSUPPORTED;
        const int nc = (int)S->c_index.size();
        pack_rounds(nc, S->c_rounds, S->c_grid,
                    [&](int k, int r) {
                        if (r >= items[S->c_index[k]].iterations * 4) return 0;
                        return (r & 3) < 2 ? S->c_tiles_v[k] : S->c_tiles_h[k];
                    },
                    [&](int k, int r) -> int64_t {
                        const fgx_instance& it = items[S->c_index[k]];
                        return (r & 3) < 2 ? it.H : it.W;
                    },
                    &S->c_round_waves, &S->c_wave_items);
        if (S->timeout_ns == 0)
            S->timeout_ns = (long long)((opt && opt->timeout_ms) ? opt->timeout_ms : 2000) *
                            1000000LL;
    }
    S->sms = sms;
    S->flags_bytes = al256((size_t)std::max(flags_total, 1) * 8);
    // layout: header | engine tags | chain exchange words | plane-tile range
    // flags and exchange words (the cleared prefix) | engine tables | chain
    // tables | plane-tile tables | chain buffers | plane-tile working copies
    S->c_xbuf_off = kHeaderBytes + S->flags_bytes;
    S->v_flag_off = S->c_xbuf_off + al256(S->c_xbuf_bytes);
    S->v_xbuf_off = S->v_flag_off + al256(S->v_index.size() * sizeof(int));
    S->desc_off = S->v_xbuf_off + al256(S->v_xbuf_bytes);
    S->waves_off = S->desc_off + al256(S->desc.size() * sizeof(InstDesc) + 1);
    S->items_off = S->waves_off + al256(S->round_waves.size() * sizeof(int));
    S->c_desc_off = S->items_off + al256(S->wave_items.size() * sizeof(int) + 1);
    S->c_waves_off = S->c_desc_off + al256(S->c_index.size() * chain2d_desc_size() + 1);
    S->c_items_off = S->c_waves_off + al256(S->c_round_waves.size() * sizeof(int) + 1);
    S->v_desc_off = S->c_items_off + al256(S->c_wave_items.size() * sizeof(int) + 1);
    S->v_waves_off = S->v_desc_off + al256(S->v_index.size() * vol3d_desc_size() + 1);
    S->v_items_off = S->v_waves_off + al256(S->v_round_waves.size() * sizeof(int) + 1);
    S->c_sec_off = S->v_items_off + al256(S->v_wave_items.size() * sizeof(int) + 1);
    S->v_work_off = S->c_sec_off + al256(S->c_sec_bytes);
    S->total = S->v_work_off + al256(S->v_work_bytes);
    return FGX_OK;
}

// The side stream of the concurrent batched launches, with its fork and join
// events: one set per host thread and device, so that calls from different
// threads never share an event (an event wait refers to the last record);
// released when the thread exits.
struct SideStreams {
    static constexpr int kDevices = 64;
    cudaStream_t stream[kDevices] = {};
    cudaEvent_t fork[kDevices] = {}, join[kDevices] = {};
    ~SideStreams() {
        for (int i = 0; i < kDevices; ++i) {
            if (fork[i]) cudaEventDestroy(fork[i]);
            if (join[i]) cudaEventDestroy(join[i]);
            if (stream[i]) cudaStreamDestroy(stream[i]);
        }
    }
};
thread_local SideStreams tl_side;

bool side_stream(cudaStream_t* s, cudaEvent_t* fork, cudaEvent_t* join) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SideStreams::kDevices)
        return false;
    SideStreams& t = tl_side;
    if (!t.stream[dev]) {
        cudaStream_t st = nullptr;
        cudaEvent_t f = nullptr, j = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return false;
        if (cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&j, cudaEventDisableTiming) != cudaSuccess) {
            if (f) cudaEventDestroy(f);
            cudaStreamDestroy(st);
            return false;
        }
        t.stream[dev] = st;
        t.fork[dev] = f;
        t.join[dev] = j;
    }
    *s = t.stream[dev];
    *fork = t.fork[dev];
    *join = t.join[dev];
    return true;
}

}  // namespace
}  // namespace fgx

using namespace fgx;

extern "C" {

int fgx_batched_workspace_size(const fgx_instance* items, int n, const fgx_options* opt,
                               size_t* bytes) {
    if (!bytes) return FGX_ERR_ARG;
    if (opt && opt->size != sizeof(fgx_options)) return FGX_ERR_ARG;
    Schedule S;
    const int st = build_schedule(items, n, opt, false, &S);
    if (st != FGX_OK) return st;
    *bytes = S.total;
    return FGX_OK;
}

int fgx_batched_prepare(const fgx_instance* items, int n, void* workspace,
                        size_t workspace_bytes, const fgx_options* opt,
                        fgx_batched_plan* plan, void* stream) {
    if (!plan) return FGX_ERR_ARG;
    if (opt && opt->size != sizeof(fgx_options)) return FGX_ERR_ARG;
    Schedule S;
    int st = build_schedule(items, n, opt, true, &S);
    if (st != FGX_OK) return st;
    if (!workspace || workspace_bytes < S.total) return FGX_ERR_WORKSPACE;
    if (!device_pointer(workspace)) return FGX_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)workspace;
    auto put = [&](size_t off, const void* src, size_t bytes) {
        return bytes == 0 ||
               cudaMemcpyAsync(w + off, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess;
    };
    // chain arguments carry device pointers into this workspace
    std::vector<unsigned char> cdesc(S.c_index.size() * chain2d_desc_size());
    for (size_t k = 0; k < S.c_index.size(); ++k) {
        size_t xb = 0;
        int tv = 0, th = 0;
        chain2d_instance_desc(cdesc.data() + k * chain2d_desc_size(), items[S.c_index[k]], opt, w,
                              w + S.c_xbuf_off + S.c_xoff[k], w + S.c_sec_off + S.c_soff[k], &xb,
                              &tv, &th);
    }
    std::vector<unsigned char> vdesc(S.v_index.size() * vol3d_desc_size());
    for (size_t k = 0; k < S.v_index.size(); ++k) {
        size_t xb = 0, wb = 0;
        int ci = 0, mt = 0, tiles[kMaxPasses];
        fgx_options o3;
        if (!vol3d_instance_desc(vdesc.data() + k * vol3d_desc_size(), items[S.v_index[k]],
                                 S.v_args[k], options_3d(opt, &o3), S.v_sms, w,
                                 (int*)(w + S.v_flag_off) + k,
                                 w + S.v_xbuf_off + S.v_xoff[k], w + S.v_work_off + S.v_woff[k],
                                 &xb, &wb, &ci, &mt, tiles))
            return FGX_ERR_UNSUPPORTED;
    }
    if (!put(S.desc_off, S.desc.data(), S.desc.size() * sizeof(InstDesc)) ||
        !put(S.v_desc_off, vdesc.data(), vdesc.size()) ||
        !put(S.v_waves_off, S.v_round_waves.data(), S.v_round_waves.size() * sizeof(int)) ||
        !put(S.v_items_off, S.v_wave_items.data(), S.v_wave_items.size() * sizeof(int)) ||
        !put(S.waves_off, S.round_waves.data(), S.round_waves.size() * sizeof(int)) ||
        !put(S.items_off, S.wave_items.data(), S.wave_items.size() * sizeof(int)) ||
        !put(S.c_desc_off, cdesc.data(), cdesc.size()) ||
        !put(S.c_waves_off, S.c_round_waves.data(), S.c_round_waves.size() * sizeof(int)) ||
        !put(S.c_items_off, S.c_wave_items.data(), S.c_wave_items.size() * sizeof(int)))
        return FGX_ERR_CUDA;
    // the host vectors are freed on return: finish the copies first
    if (cudaStreamSynchronize(s) != cudaSuccess) return FGX_ERR_CUDA;
    std::memset(plan, 0, sizeof(*plan));
    plan->size = sizeof(fgx_batched_plan);
    plan->n = (int)S.desc.size();
    plan->grid = S.grid;
    plan->smem_bytes = (int)S.smem;
    plan->rounds = S.rounds;
    plan->region = S.region;
    plan->kmax = S.kmax;
    plan->timeout_ms = (int)(S.timeout_ns / 1000000LL);
    plan->clear_bytes = S.desc_off;  // header, engine tags and chain exchange words
    plan->desc_off = S.desc_off;
    plan->waves_off = S.waves_off;
    plan->items_off = S.items_off;
    plan->workspace = workspace;
    plan->workspace_bytes = S.total;
    plan->n2d = (int)S.c_index.size();
    plan->grid2d = S.c_grid;
    plan->rounds2d = S.c_rounds;
    plan->channels2d = S.c_channels;
    plan->max_wp2d = S.c_max_wp;
    plan->max_hp2d = S.c_max_hp;
    plan->desc2d_off = S.c_desc_off;
    plan->waves2d_off = S.c_waves_off;
    plan->items2d_off = S.c_items_off;
    plan->n3d = (int)S.v_index.size();
    plan->grid3d = S.v_grid;
    plan->rounds3d = S.v_rounds;
    plan->smem3d = (int)S.v_smem;
    plan->desc3d_off = S.v_desc_off;
    plan->waves3d_off = S.v_waves_off;
    plan->items3d_off = S.v_items_off;
    plan->tables3d = S.v_ci > kMaxChannels3 ? 1 : 0;
    plan->concurrent = S.concurrent ? 1 : 0;
    if (S.concurrent) {
        cudaStream_t s2;
        cudaEvent_t f, j;
        if (!side_stream(&s2, &f, &j)) return FGX_ERR_CUDA;
    }
    return FGX_OK;
}

int fgx_batched_run(const fgx_batched_plan* plan, void* stream) {
    if (!plan || plan->size != sizeof(fgx_batched_plan) || !plan->workspace) return FGX_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)plan->workspace;
    if (cudaMemsetAsync(w, 0, plan->clear_bytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    const long long timeout_ns = (long long)plan->timeout_ms * 1000000LL;
    const bool both = plan->concurrent && plan->n2d > 0 && plan->n3d > 0;
    cudaStream_t s2 = s;
    cudaEvent_t join = nullptr;
    if (both) {
        // fork: the line-chain launch runs on the side stream after
        // everything before it on the caller's stream (the clear above)
        cudaEvent_t fork = nullptr;
        if (!side_stream(&s2, &fork, &join) || cudaEventRecord(fork, s) != cudaSuccess ||
            cudaStreamWaitEvent(s2, fork, 0) != cudaSuccess)
            return FGX_ERR_CUDA;
    }
    int st = FGX_OK;
    if (plan->n2d > 0)
        st = launch_chain2d_batched(
            w + plan->desc2d_off, plan->n2d, plan->channels2d, plan->max_wp2d, plan->max_hp2d,
            plan->rounds2d, (const int*)(w + plan->waves2d_off),
            (const int*)(w + plan->items2d_off), plan->grid2d, w, timeout_ns, s2);
    if (st == FGX_OK && plan->n3d > 0) {
        // one after the other the launches reuse one grid-barrier counter; at
        // the same time the plane-tile launch counts in the next word
        int dev = 0, sms = 0;
        if ((plan->n2d > 0 && !both && cudaMemsetAsync(w + 64, 0, 4, s) != cudaSuccess) ||
            cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            st = FGX_ERR_CUDA;
        else
            st = launch_vol3d_batched(
                w + plan->desc3d_off, plan->n3d, plan->rounds3d,
                (const int*)(w + plan->waves3d_off), (const int*)(w + plan->items3d_off),
                plan->grid3d, (size_t)plan->smem3d, plan->tables3d, w,
                (unsigned int*)(w + (both ? 128 : 64)), timeout_ns, sms, stream);
    }
    // join (also after a failed launch): the caller's stream waits for the
    // line-chain launch
    if (both && (cudaEventRecord(join, s2) != cudaSuccess ||
                 cudaStreamWaitEvent(s, join, 0) != cudaSuccess))
        return FGX_ERR_CUDA;
    if (st != FGX_OK) return st;
    if (plan->n == 0) return FGX_OK;
    if ((plan->n2d > 0 || plan->n3d > 0) && cudaMemsetAsync(w + 64, 0, 4, s) != cudaSuccess)
        return FGX_ERR_CUDA;  // fresh grid-barrier counter for this launch
    BatchedArgs a;
    std::memset(&a, 0, sizeof(a));
    a.desc = (const InstDesc*)(w + plan->desc_off);
    a.n = plan->n;
    a.rounds = plan->rounds;
    a.round_waves = (const int*)(w + plan->waves_off);
    a.wave_items = (const int*)(w + plan->items_off);
    a.flags = (unsigned long long*)(w + kHeaderBytes);
    a.barrier = (unsigned int*)(w + 64);
    a.status = (int*)w;
    a.timeout_ns = timeout_ns;
    int per_sm = 0;
    st = batched_max_blocks_per_sm((size_t)plan->smem_bytes, &per_sm);
    if (st != FGX_OK) return st;
    return launch_batched(a, plan->grid, (size_t)plan->smem_bytes, stream);
}

int fgx_batched_autotune(const fgx_instance* items, int n, void* workspace,
                         size_t workspace_bytes, const fgx_options* candidates, int ncand,
                         int reps, int* best_index, float* best_ms, void* stream) {
    if (!candidates || ncand < 1 || reps < 1 || !best_index || !best_ms) return FGX_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FGX_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FGX_ERR_CUDA;
    }
    int st = FGX_OK, best = -1;
    float best_t = 0.f;
    for (int i = 0; i < ncand && st == FGX_OK; ++i) {
        size_t need = 0;
        int r = fgx_batched_workspace_size(items, n, candidates + i, &need);
        if (r == FGX_ERR_UNSUPPORTED || (r == FGX_OK && need > workspace_bytes)) continue;
        if (r != FGX_OK) { st = r; break; }
        fgx_batched_plan plan;
        r = fgx_batched_prepare(items, n, workspace, workspace_bytes, candidates + i, &plan,
                                stream);
        if (r == FGX_ERR_UNSUPPORTED) continue;
        if (r == FGX_OK) r = fgx_batched_run(&plan, stream);  // warm-up
        if (r != FGX_OK) { st = r; break; }
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = FGX_ERR_CUDA; break; }
        for (int k = 0; k < reps && r == FGX_OK; ++k) r = fgx_batched_run(&plan, stream);
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

int fgx_geodesic_batched(const fgx_instance* items, int n, void* workspace,
                         size_t workspace_bytes, const fgx_options* opt, void* stream) {
    fgx_batched_plan plan;
    const int st = fgx_batched_prepare(items, n, workspace, workspace_bytes, opt, &plan, stream);
    if (st != FGX_OK) return st;
    return fgx_batched_run(&plan, stream);
}

}  // extern "C"
