// TMA-staged step kernels for __half population storage.
#include "step_tma.cuh"

namespace lbsc {

template <>
long long tma_step<__half>(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map,
                        const StepArgs<__half>* args, cudaStream_t stream)
{
    return tma_dispatch<__half>(op, tile_y, stages, tau_one, map, args, stream);
}

}  // namespace lbsc
