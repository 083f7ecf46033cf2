// TMA-staged step kernels for float population storage.
#include "step_tma.cuh"

namespace lbsc {

template <>
long long tma_step<float>(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map,
                        const StepArgs<float>* args, cudaStream_t stream)
{
    return tma_dispatch<float>(op, tile_y, stages, tau_one, map, args, stream);
}

template <>
long long tma_batch<float>(int op, int tile_y, bool tau_one, const void* maps, const StepArgs<float>* args,
                        const int4* items, int nitems, int parity, int nbox, uint32_t* done, int grid,
                        cudaStream_t stream)
{
    return tma_batch_dispatch<float>(op, tile_y, tau_one, maps, args, items, nitems, parity, nbox, done, grid, stream);
}

}  // namespace lbsc

namespace lbsc {

// Self-test of the bounded wait: the same try_wait loop as the TMA step, on
// an mbarrier that no copy or arrival will ever complete, with a short limit.
// The wait gives up, the kernel writes the status word and returns; nothing is
// in flight, so the CTA exits cleanly.
__global__ void wait_probe_kernel(int* err, uint32_t limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    bool ok = false;
    for (uint32_t i = 0; i < limit && !ok; ++i) ok = mbar_try_wait(&bar, 0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, kErrWait);
}

cudaError_t launch_wait_probe(int* err, unsigned limit, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(err, limit);
    return cudaGetLastError();
}

}  // namespace lbsc
