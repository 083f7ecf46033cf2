// TMA-staged step kernels for float population storage.
#include "step_tma.cuh"

namespace lbsc {

template <>
long long tma_step<float>(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map,
                        const StepArgs<float>* args, cudaStream_t stream)
{
    return tma_dispatch<float>(op, tile_y, stages, tau_one, map, args, stream);
}

}  // namespace lbsc
