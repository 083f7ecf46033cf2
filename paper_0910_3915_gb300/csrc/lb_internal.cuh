// Internal definitions of the lbsc CUDA library: the D3Q19 lattice, the
// population storage codecs, the ghosted storage layout and the argument
// blocks of the kernels.
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
    static __device__ __forceinline__ float val(float v) { return v; }
    static __device__ __forceinline__ float round(float v) { return v; }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
};
// Stochastic rounding to a 16-bit format with `mant` explicit mantissa bits:
// add a uniform dither of one unit in the last place, then round to nearest.
// u01 in [0, 1); the result's expected value is v (no rounding bias).
__device__ __forceinline__ float dither_ulp(float v, float u01, int mant)
{
    const int e = ((__float_as_int(v) >> 23) & 0xff);  // biased FP32 exponent of |v|
    const int eu = e - mant > 1 ? e - mant : 1;        // exponent of one ulp (FP32 normal range)
    return v + (u01 - 0.5f) * __int_as_float(eu << 23);
}

// Uniform in [0, 1) from three 32-bit keys: a multiply-xorshift hash (the
// 32-bit finaliser of MurmurHash3) of a combined key.
__device__ __forceinline__ float hash_u01(uint32_t node, uint32_t comp, uint32_t key)
{
    uint32_t h = node * 0x9E3779B1u ^ (key * 0x85EBCA77u + comp * 0xC2B2AE3Du);
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return (float)(h >> 8) * (1.0f / 16777216.0f);
}

template <>
struct Codec<__half> {
    static constexpr bool kDeviation = true;
    static constexpr int kMant = 10;
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float val(__half v) { return __half2float(v); }
    static __device__ __forceinline__ float round(float v) { return __half2float(__float2half_rn(v)); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
    static constexpr bool kDeviation = true;
    static constexpr int kMant = 7;
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float val(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Lattice storage: 2*19 population planes of `slot` elements each, slot
// index a*19 + k. Inside a slot, node (x, y, z) sits at
//   z*plane + (y + 1)*px + (x + gx),
// with gx = 128 bytes of row padding on the left (so x = 0 starts a 128-byte
// line) and at least one element on the right, and one ghost row above and
// below each plane. Ghost column x = -1 mirrors x = nx-1, x = nx mirrors
// x = 0, and likewise rows y = -1 and y = ny, so a tile plus its one-node
// ring is one box even on the periodic edges. The step kernels write real
// nodes only; the images are refreshed by a separate pass where a reader
// needs them (the TMA-staged step).
struct Layout {
    int nx, ny, nz, px, gx;
    long long plane, slot;
    __host__ __device__ __forceinline__ long long off(int x, int y, int z) const
    {
        return (long long)z * plane + (long long)(y + 1) * px + (x + gx);
    }
};

// Write the ghost images (only) of node (x, y) of the plane at zoff.
template <class S>
__device__ __forceinline__ void put_ghosts(S* __restrict__ p, const Layout& L, int x, int y, long long zoff, float v)
{
    const long long row = zoff + (long long)(y + 1) * L.px + L.gx;
    const bool xl = x == L.nx - 1, xr = x == 0;
    if (xl) Codec<S>::store(p + row - 1, v);
    if (xr) Codec<S>::store(p + row + L.nx, v);
    if (y == L.ny - 1) {
        const long long g = zoff + L.gx;  // row y = -1
        Codec<S>::store(p + g + x, v);
        if (xl) Codec<S>::store(p + g - 1, v);
        if (xr) Codec<S>::store(p + g + L.nx, v);
    }
    if (y == 0) {
        const long long g = zoff + (long long)(L.ny + 1) * L.px + L.gx;  // row y = ny
        Codec<S>::store(p + g + x, v);
        if (xl) Codec<S>::store(p + g - 1, v);
        if (xr) Codec<S>::store(p + g + L.nx, v);
    }
}

// 1 if node (x, y) has a ghost image
__host__ __device__ __forceinline__ bool has_ghost(const Layout& L, int x, int y)
{
    return x == 0 || x == L.nx - 1 || y == 0 || y == L.ny - 1;
}

// Store v for node (x, y) of the plane at zoff into slot base p, with the
// ghost images of edge nodes.
template <class S>
__device__ __forceinline__ void put(S* __restrict__ p, const Layout& L, int x, int y, long long zoff, float v)
{
    Codec<S>::store(p + zoff + (long long)(y + 1) * L.px + L.gx + x, v);
    if (has_ghost(L, x, y)) put_ghosts<S>(p, L, x, y, zoff, v);
}

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
    int* err;                             // device status word (bounded waits that gave up)
    Layout L;
    KParams P;
    int tiles_x, tiles_y;
    int zlo, zhi;  // fluid plane range [zlo, zhi)
    int nseg;      // z segments per tile column
};

constexpr uint32_t kSelfSolid = 1u << 31;

__host__ __device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// elements in 16 bytes: the ring column a TMA box carries on each side of a tile
template <class S>
__host__ __device__ constexpr int ghost_x() { return 16 / (int)sizeof(S); }

}  // namespace lbsc
