// TMA-staged step kernels for __nv_bfloat16 population storage.
#include "step_tma.cuh"

namespace lbsc {

template <>
long long tma_step<__nv_bfloat16>(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map,
                        const StepArgs<__nv_bfloat16>* args, cudaStream_t stream)
{
    return tma_dispatch<__nv_bfloat16>(op, tile_y, stages, tau_one, map, args, stream);
}

template <>
long long tma_batch<__nv_bfloat16>(int op, int tile_y, bool tau_one, const void* maps, const StepArgs<__nv_bfloat16>* args,
                        const int4* items, int nitems, int parity, int nbox, uint32_t* done, int grid,
                        cudaStream_t stream)
{
    return tma_batch_dispatch<__nv_bfloat16>(op, tile_y, tau_one, maps, args, items, nitems, parity, nbox, done, grid, stream);
}

}  // namespace lbsc
