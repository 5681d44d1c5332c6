// Failure-detection check: one thread waits, with the bounded wait that every
// inter-block hand-over of the library uses, for a tag that nothing writes.
// The wait gives up after its limit and records FGX_ERR_TIMEOUT in the status
// word; nothing faults and the context stays usable.
#include <cuda_runtime.h>

#include "device_sync.cuh"
#include "fgx_internal.h"

namespace fgx {
namespace {

__global__ void wait_probe_kernel(const unsigned long long* tag, int* status,
                                  long long timeout_ns) {
    if (threadIdx.x == 0 && blockIdx.x == 0) dev::wait_tag(tag, 1ull, status, timeout_ns);
}

}  // namespace

void launch_wait_probe(const unsigned long long* tag, int* status, long long timeout_ns,
                       void* stream) {
    wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(tag, status, timeout_ns);
}

}  // namespace fgx
