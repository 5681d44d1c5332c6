// Device-side synchronisation helpers shared by the library's persistent
// kernels: memory accesses with explicit scope and ordering, bounded waits on
// progress tags, and a grid barrier.  Every wait gives up after a time limit,
// records FGX_ERR_TIMEOUT in the device status word and returns false, so a
// missing peer never hangs the GPU.
#pragma once

#include <cuda_runtime.h>

#include "fgx_internal.h"

namespace fgx {
namespace dev {

__device__ __forceinline__ long long gtimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int status_of(const int* s) { return *(volatile const int*)s; }

__device__ __forceinline__ void record_timeout(int* status) {
    atomicCAS(status, 0, (int)FGX_ERR_TIMEOUT);
}

// Thread-level wait until *f >= target (release/acquire pairing with
// st_release_u64 by the producer).  False on timeout or an earlier failure.
__device__ inline bool wait_tag(const unsigned long long* f, unsigned long long target,
                                int* status, long long timeout_ns) {
    if (ld_acquire_u64(f) >= target) return true;
    const long long t0 = gtimer();
    for (;;) {
        __nanosleep(64);
        if (ld_acquire_u64(f) >= target) return true;
        if (status_of(status) != 0) return false;
        if (gtimer() - t0 > timeout_ns) {
            record_timeout(status);
            return false;
        }
    }
}

// Grid barrier for a cooperative launch; `epoch` is the 1-based count of
// barriers passed.  Thread 0 polls with relaxed loads and back-off (an
// acquiring load in a tight loop disturbs warps sharing the SM), then fences.
// Returns false (for every thread of the block) once the status word records
// a failure.
__device__ inline bool grid_barrier(unsigned int* ctr, unsigned int epoch, int* status,
                                    long long timeout_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        const unsigned int target = epoch * gridDim.x;
        ok = status_of(status) == 0;
        const long long t0 = gtimer();
        while (ok && ld_relaxed_u32(ctr) < target) {
            if (status_of(status) != 0) { ok = 0; break; }
            if (gtimer() - t0 > timeout_ns) {
                record_timeout(status);
                ok = 0;
                break;
            }
            __nanosleep(256);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int64_t mn64(int64_t x, int64_t y) { return x < y ? x : y; }
__device__ __forceinline__ int64_t mx64(int64_t x, int64_t y) { return x > y ? x : y; }

}  // namespace dev
}  // namespace fgx
