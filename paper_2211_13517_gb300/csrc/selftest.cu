// Failure-path check of the bounded mbarrier waits: a barrier armed for bytes
// that never arrive, waited on with a short limit.  No copy is issued, so
// nothing is in flight when the CTA exits.
#include "fdas_internal.cuh"
#include "tma.cuh"

namespace fdas {
namespace {

__global__ void stuck_wait_kernel(unsigned int *flags, long long limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);   // 16 bytes nobody sends
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(flags, 2u);
}

}  // namespace

fdas_status launch_stuck_wait(unsigned int *flags, long long limit_cycles, cudaStream_t s) {
    stuck_wait_kernel<<<1, 32, 0, s>>>(flags, limit_cycles);
    FDAS_CUDA_TRY(cudaGetLastError());
    return FDAS_OK;
}

}  // namespace fdas
