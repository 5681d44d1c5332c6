// Batched launch of instances of uneven shapes (2D and 3D mixed): host-side
// planning of the work list and the C ABI entry points.
//
// Every instance runs the same raster-scan schedule as a single call (4 or 6
// passes per iteration, FastGeodis Implementation section) on the tiled
// engine.  Instances advance one pass application per round; a round packs
// whole instances into waves of co-resident thread blocks (first fit), so
// the tiles of an instance that wait on one another always run together; the
// rounds are separated by a grid barrier inside the one persistent launch.
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
    std::vector<InstDesc> desc;
    std::vector<int> round_waves;
    std::vector<int> wave_items;
    int grid = 0, rounds = 0, region = 1, kmax = 1;
    size_t smem = 0, flags_bytes = 0;
    size_t desc_off = 0, waves_off = 0, items_off = 0, total = 0;
    long long timeout_ns = 0;
};

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

// Builds descriptors and the round/wave work list; pointers are checked only
// when `check_ptrs`.
int build_schedule(const fgx_instance* items, int n, const fgx_options* opt, bool check_ptrs,
                   Schedule* S) {
    if (n < 0 || (n > 0 && !items)) return FGX_ERR_ARG;
    if (n > 32767) return FGX_ERR_UNSUPPORTED;
    int sms = 0;
    int max_tiles_any = 1, flags_total = 0;
    S->desc.clear();
    for (int i = 0; i < n; ++i) {
        const fgx_instance& it = items[i];
        int st = check_instance(it);
        if (st != FGX_OK) return st;
        const int64_t N = it.D * it.H * it.W;
        if (N == 0) continue;
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
        st = plan_instance(it.ndim, it.channels, it.D, it.H, it.W, it.spacing, it.lambda, opt, &a,
                           &sms);
        if (st != FGX_OK) return st;
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
    // rounds and waves
    int rounds = 0;
    for (const InstDesc& d : S->desc) rounds = std::max(rounds, d.napps);
    S->rounds = rounds;
    S->round_waves.assign(1, 0);
    S->wave_items.clear();
    for (int r = 0; r < rounds; ++r) {
        std::vector<int> used;  // blocks used per wave of this round
        std::vector<std::vector<std::pair<int, int>>> members;  // (instance, first block)
        for (int i = 0; i < (int)S->desc.size(); ++i) {
            const InstDesc& d = S->desc[i];
            if (r >= d.napps) continue;
            const PassGeom& g = d.pass[r % d.npass];
            const int tiles = g.ntp * g.ntq;
            size_t w = 0;
            while (w < used.size() && used[w] + tiles > S->grid) ++w;
            if (w == used.size()) {
                used.push_back(0);
                members.emplace_back();
            }
            members[w].push_back({i, used[w]});
            used[w] += tiles;
        }
        for (size_t w = 0; w < used.size(); ++w) {
            const size_t base = S->wave_items.size();
            S->wave_items.resize(base + S->grid, -1);
            for (auto& m : members[w]) {
                const InstDesc& d = S->desc[m.first];
                const PassGeom& g = d.pass[r % d.npass];
                for (int t = 0; t < g.ntp * g.ntq; ++t)
                    S->wave_items[base + m.second + t] = (m.first << 16) | t;
            }
        }
        S->round_waves.push_back(S->round_waves.back() + (int)used.size());
    }
    S->flags_bytes = al256((size_t)std::max(flags_total, 1) * 8);
    S->desc_off = kHeaderBytes + S->flags_bytes;
    S->waves_off = S->desc_off + al256(S->desc.size() * sizeof(InstDesc) + 1);
    S->items_off = S->waves_off + al256(S->round_waves.size() * sizeof(int));
    S->total = S->items_off + al256(S->wave_items.size() * sizeof(int) + 1);
    return FGX_OK;
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
    if (!S.desc.empty()) {
        if (cudaMemcpyAsync(w + S.desc_off, S.desc.data(), S.desc.size() * sizeof(InstDesc),
                            cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(w + S.waves_off, S.round_waves.data(),
                            S.round_waves.size() * sizeof(int), cudaMemcpyHostToDevice,
                            s) != cudaSuccess ||
            (!S.wave_items.empty() &&
             cudaMemcpyAsync(w + S.items_off, S.wave_items.data(),
                             S.wave_items.size() * sizeof(int), cudaMemcpyHostToDevice,
                             s) != cudaSuccess))
            return FGX_ERR_CUDA;
        // the host vectors are freed on return: finish the copies first
        if (cudaStreamSynchronize(s) != cudaSuccess) return FGX_ERR_CUDA;
    }
    std::memset(plan, 0, sizeof(*plan));
    plan->size = sizeof(fgx_batched_plan);
    plan->n = (int)S.desc.size();
    plan->grid = S.grid;
    plan->smem_bytes = (int)S.smem;
    plan->rounds = S.rounds;
    plan->region = S.region;
    plan->kmax = S.kmax;
    plan->timeout_ms = (int)(S.timeout_ns / 1000000LL);
    plan->clear_bytes = kHeaderBytes + S.flags_bytes;
    plan->desc_off = S.desc_off;
    plan->waves_off = S.waves_off;
    plan->items_off = S.items_off;
    plan->workspace = workspace;
    plan->workspace_bytes = S.total;
    return FGX_OK;
}

int fgx_batched_run(const fgx_batched_plan* plan, void* stream) {
    if (!plan || plan->size != sizeof(fgx_batched_plan) || !plan->workspace) return FGX_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    char* w = (char*)plan->workspace;
    if (cudaMemsetAsync(w, 0, plan->clear_bytes, s) != cudaSuccess) return FGX_ERR_CUDA;
    if (plan->n == 0) return FGX_OK;
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
    a.timeout_ns = (long long)plan->timeout_ms * 1000000LL;
    int per_sm = 0;
    int st = batched_max_blocks_per_sm((size_t)plan->smem_bytes, &per_sm);
    if (st != FGX_OK) return st;
    return launch_batched(a, plan->grid, (size_t)plan->smem_bytes, stream);
}

int fgx_geodesic_batched(const fgx_instance* items, int n, void* workspace,
                         size_t workspace_bytes, const fgx_options* opt, void* stream) {
    fgx_batched_plan plan;
    const int st = fgx_batched_prepare(items, n, workspace, workspace_bytes, opt, &plan, stream);
    if (st != FGX_OK) return st;
    return fgx_batched_run(&plan, stream);
}

}  // extern "C"
