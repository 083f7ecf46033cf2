// Internal definitions of the lbsc CUDA library: the D3Q19 lattice, the
// population storage codecs and the argument blocks of the kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace lbsc {

constexpr int Q = 19;

// D3Q19 velocities (Sec. 2): k = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 the
// twelve face diagonals, each followed by its opposite.
__host__ __device__ __forceinline__ constexpr int cx(int k)
{
    constexpr int v[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
    return v[k];
}
__host__ __device__ __forceinline__ constexpr int cy(int k)
{
    constexpr int v[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
    return v[k];
}
__host__ __device__ __forceinline__ constexpr int cz(int k)
{
    constexpr int v[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
    return v[k];
}
// index of -c_k: pairs (1,2), (3,4), ..., (17,18)
__host__ __device__ __forceinline__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }
// lattice weights zeta_k (rest 1/3, axis 1/18, diagonal 1/36), c_s^2 = 1/3
__host__ __device__ __forceinline__ constexpr float zeta(int k)
{
    return k == 0 ? 1.0f / 3.0f : (k <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ __forceinline__ constexpr bool is_axis(int k) { return k >= 1 && k <= 6; }

// Population storage. FP32 holds n_k. The 16-bit formats hold the normalised
// deviation e_k = n_k / zeta_k - rho_ref of the component, so n_k = zeta_k (rho_ref + e_k);
// all arithmetic is FP32.
template <class S>
struct Codec;

template <>
struct Codec<float> {
    static constexpr bool kDeviation = false;
    static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};
template <>
struct Codec<__half> {
    static constexpr bool kDeviation = true;
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
    static constexpr bool kDeviation = true;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Lattice storage: 2*19 population planes of `slot` elements each, slot
// index a*19 + k; inside a slot, node (x, y, z) at z*plane + y*px + x with the
// row pitch px a multiple of 32 elements.
struct Layout {
    int nx, ny, nz, px;
    long long plane, slot;
};

// Parameters as the kernels use them.
struct KParams {
    float gk;            // g_br * force_scale
    float Gax, Gdi;      // neighbour weights on axis and diagonal links
    float tau[2], itau[2];
    float eta[2];        // psi stand-ins on solid nodes: [0] for psi^r, [1] for psi^b
    float ref[2];        // 16-bit deviation references rho_ref
};

template <class S>
struct StepArgs {
    const S* __restrict__ src;
    S* __restrict__ dst;
    const uint32_t* __restrict__ nbmask;  // general geometry: bit k = (x + c_k solid), bit 31 = x solid
    Layout L;
    KParams P;
    int tiles_x, tiles_y;
    int zlo, zhi;  // fluid plane range [zlo, zhi)
    int nseg;      // z segments per tile column
};

constexpr uint32_t kSelfSolid = 1u << 31;

__host__ __device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

}  // namespace lbsc
