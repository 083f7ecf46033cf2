// TMA-staged step kernels for __nv_bfloat16 population storage.
#include "step_tma.cuh"

namespace lbsc {

template <>
long long tma_step<__nv_bfloat16>(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map,
                        const StepArgs<__nv_bfloat16>* args, cudaStream_t stream)
{
    return tma_dispatch<__nv_bfloat16>(op, tile_y, stages, tau_one, map, args, stream);
}

}  // namespace lbsc
