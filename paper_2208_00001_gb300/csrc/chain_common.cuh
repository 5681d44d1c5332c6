// Building blocks shared by the warp-chain kernels (2D forward and 2D
// reverse sweep): shared-memory hand-over rings guarded by mbarriers, per-lane
// cp.async, and the ring refresh between neighbouring line tiles.
//
// Line tiles.  A tile owns T columns of a line plus a ring of K columns on
// each side (T + 2K = 128: four columns per lane of one warp).  A one-line
// step reads only the three neighbouring columns of the previous line, so
// the exact part of the region shrinks by one column per line; after K lines
// the owned columns are still exact and the ring is refreshed from the
// neighbours, which publish their owned edge strips as 64-bit words
// (value, tag).  A word is valid once its tag matches: no fence or flag
// precedes the read.
#pragma once

#include <cuda_runtime.h>

#include "device_sync.cuh"

namespace fgx {
namespace chain {
namespace {

using namespace dev;

constexpr int kMaxRing = 48;  // words per exchanged strip (K <= kMaxRing)

__device__ __forceinline__ unsigned int saddr(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr(smem)), "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(saddr(b))
                 : "memory");
}
// One arrival on *b that also expects `bytes` of tensor copies to complete
// the phase.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     saddr(b)),
                 "r"(bytes)
                 : "memory");
}
// One box of a 3D tensor map (x innermost) into shared memory at `dst`,
// completed on *mbar by transaction count.
__device__ __forceinline__ void tma_load3(const void* dst, const void* map, int x, int y, int z,
                                          unsigned long long* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(saddr(mbar))
        : "memory");
}
// One arrival on *b once every cp.async this thread issued so far has landed.
__device__ __forceinline__ void cp_async_arrive_noinc(unsigned long long* b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(b))
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}
// Tests (and, if incomplete, waits a little for) the phase of parity
// `parity` of *b.
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned int parity) {
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Non-blocking test of the same phase.
__device__ __forceinline__ bool mbar_peek(unsigned long long* b, unsigned int parity) {
    unsigned int ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits (bounded) for the completion of the phase of parity `parity` of *b;
// false on timeout or an earlier failure recorded in the status word.
__device__ __noinline__ bool mbar_wait_slow(unsigned long long* b, unsigned int parity,
                                            int* status, long long timeout_ns) {
    const long long t0 = gtimer();
    for (;;) {
        if (mbar_test(b, parity)) return true;
        if (status_of(status) != 0) return false;
        if (gtimer() - t0 > timeout_ns) {
            record_timeout(status);
            return false;
        }
    }
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned int parity,
                                          int* status, long long timeout_ns) {
    if (mbar_test(b, parity)) return true;
    return mbar_wait_slow(b, parity, status, timeout_ns);
}
// Position of chunk gc in a ring of n slots: the slot and the parity of the
// slot's phase that the chunk fills.
struct RingPos {
    int slot;
    unsigned int par;
    __device__ RingPos(unsigned int gc, int n)
        : slot((int)(gc % (unsigned)n)), par((gc / (unsigned)n) & 1u) {}
    __device__ RingPos(int s, unsigned int p) : slot(s), par(p) {}
    __device__ __forceinline__ RingPos next(int n) const {
        return slot + 1 == n ? RingPos(0, par ^ 1u) : RingPos(slot + 1, par);
    }
};
// Chunk gc of a ring of n slots: slot, parity of its "full" phase, and parity
// of the "empty" phase that frees the slot (the release of chunk gc - n).
__device__ __forceinline__ int slot_of(unsigned int gc, int n) { return (int)(gc % (unsigned)n); }
__device__ __forceinline__ unsigned int full_parity(unsigned int gc, int n) {
    return (gc / (unsigned)n) & 1u;
}
__device__ __forceinline__ unsigned int empty_parity(unsigned int gc, int n) {
    return ((gc / (unsigned)n) & 1u) ^ 1u;
}

// Exchange area of one image: [tiles][2 parities][2 sides][kMaxRing] words.
struct RingLink {
    unsigned long long* xbuf;  // this image's area
    int* status;
    long long timeout_ns;
};

// Ring refresh of a multi-tile pass before step s (v holds line s-1 of the
// lane's four columns c0 .. c0+3): publish the owned columns the neighbours'
// rings cover, then take the ring columns from the neighbours (two staggered
// polls in flight, bounded wait).  Columns outside the line get `fill`.
__device__ __forceinline__ bool ring_exchange(const RingLink& x, int tile, int ntiles, int q0,
                                              int K, int T, int c0, unsigned int tg, int par,
                                              float (&v)[4], const bool (&valid)[4], float fill) {
    const int lane = threadIdx.x & 31;
    unsigned long long* mine = x.xbuf + (size_t)tile * (4 * kMaxRing) + par * (2 * kMaxRing);
    const int rq = q0 + T - K;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int c = c0 + i;
        const unsigned long long w =
            ((unsigned long long)tg << 32) | (unsigned int)__float_as_uint(v[i]);
        if (c >= q0 && c < q0 + K) st_relaxed_u64(mine + (c - q0), w);
        if (c >= rq && c < q0 + T) st_relaxed_u64(mine + kMaxRing + (c - rq), w);
    }
    // ring lanes [q0-K, q0) and [q0+T, q0+T+K); lanes beyond the right ring
    // hold columns outside the cone and are never refreshed
    const bool left_ring = c0 < q0 && tile > 0;
    const bool right_ring = c0 >= q0 + T && c0 < q0 + T + K && tile + 1 < ntiles;
    const unsigned long long* nb = nullptr;
    int base = 0;
    if (left_ring) {
        nb = x.xbuf + (size_t)(tile - 1) * (4 * kMaxRing) + par * (2 * kMaxRing) + kMaxRing;
        base = c0 - (q0 - K);
    } else if (right_ring) {
        nb = x.xbuf + (size_t)(tile + 1) * (4 * kMaxRing) + par * (2 * kMaxRing);
        base = c0 - (q0 + T);
    }
    // Two polls stay in flight, the second issued ~100 ns after the first,
    // so one of them tends to reach the cache just after the neighbour's
    // store instead of a full round trip later.
    float got[4] = {v[0], v[1], v[2], v[3]};
    bool done = (nb == nullptr);
    unsigned long long wa[4], wb[4];
    auto issue = [&](unsigned long long (&w)[4]) {
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = ld_relaxed_u64(nb + base + i);
    };
    auto take = [&](const unsigned long long (&w)[4]) {
        bool all = true;
#pragma unroll
        for (int i = 0; i < 4; ++i) all = all && (unsigned int)(w[i] >> 32) == tg;
        if (all) {
#pragma unroll
            for (int i = 0; i < 4; ++i) got[i] = __uint_as_float((unsigned int)w[i]);
        }
        return all;
    };
    if (!done) issue(wa);
    __nanosleep(50);
    if (!done) issue(wb);
    long long t0 = 0;
    for (unsigned int it = 0;; ++it) {
        if (!done) {
            done = take(wa);
            if (!done) issue(wa);
        }
        if (__all_sync(0xffffffffu, done)) break;
        if (!done) {
            done = take(wb);
            if (!done) issue(wb);
        }
        if (__all_sync(0xffffffffu, done)) break;
        // the status word and the clock are read every 8th round only
        if ((it & 7u) == 7u) {
            int fail = 0;
            if (lane == 0) {
                const long long now = gtimer();
                if (t0 == 0) t0 = now;
                if (status_of(x.status) != 0) fail = 1;
                else if (now - t0 > x.timeout_ns) {
                    record_timeout(x.status);
                    fail = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, fail, 0)) return false;
        }
    }
    if (nb) {
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = valid[i] ? got[i] : fill;
    }
    return true;
}

}  // namespace
}  // namespace chain
}  // namespace fgx
