// Check of the bounded waits that guard every bulk-copy pipeline of the library.
//
// One thread initialises an mbarrier that expects one arrival and waits on its
// first phase with the same bounded wait the copy pipelines use.  Nothing
// arrives and no copy is issued, so the wait gives up after its time bound; the
// kernel records that in the error word (bit 4, the bit the host turns into
// HERMES_ERR_TIMEOUT) and exits normally, leaving the context usable.
#include "kernels.h"
#include "async_copy.cuh"

namespace hermes {

__global__ void k_wait_unarrived(unsigned* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    ac::mbar_init(&bar, 1);
    ac::mbar_init_fence();
    if (!ac::mbar_wait(&bar, 0)) atomicOr(err, 4u);
    ac::mbar_inval(&bar);
}

cudaError_t launch_wait_unarrived(unsigned* err, cudaStream_t st, const Tracer& tr) {
    tr(K_WAIT_CHECK, 0, st);
    k_wait_unarrived<<<1, 32, 0, st>>>(err);
    tr(K_WAIT_CHECK, 1, st);
    return cudaGetLastError();
}

}  // namespace hermes
