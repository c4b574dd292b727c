// Failure-detection self test of the kernels' bounded waits (the paper has no
// counterpart).  One thread arms a shared-memory barrier for a transfer that
// is never issued and waits on it with the particle kernel's bounded wait,
// under a short time limit; the wait gives up and sets the sticky timeout
// flag that the host reads.  Nothing spins without a bound and no fault is
// raised.
#include "pic_internal.cuh"

namespace picgb {

__global__ void k_wait_probe(int* __restrict__ err, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    mbar_expect_tx(&bar, 64u);  // the one arrival, expecting 64 bytes that never come
    if (!mbar_wait_bounded(&bar, 0u, WAIT_LIMIT, limit_ns)) atomicOr(err, ERRBIT_TIMEOUT);
}

cudaError_t wait_probe_launch(cudaStream_t st, int* err, uint64_t limit_ns) {
    k_wait_probe<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace picgb
