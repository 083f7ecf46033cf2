// Internal definitions of the lbsc CUDA library: the D3Q19 lattice, the
// population storage codecs, the padded storage layout and the argument
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
    using Pair = float2;  // the two components' values of one velocity, side by side
    static constexpr bool kDeviation = false;
    static constexpr bool kDitherMoving = false;
    static __device__ __forceinline__ float load(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float2 load2(const float* p) { return __ldg((const float2*)p); }
    static __device__ __forceinline__ float val(float v) { return v; }
    static __device__ __forceinline__ float2 val2(float2 v) { return v; }
    static __device__ __forceinline__ void store(float* p, float v) { *p = v; }
    static __device__ __forceinline__ void store2(float* p, float a, float b) { *(float2*)p = make_float2(a, b); }
};
// Random bits for stochastic rounding. A 32-bit hash per node and step (the
// 32-bit finaliser of MurmurHash3 applied to a combined key); the pair of
// values of velocity j takes the 32-bit word h * M_j with the odd multiplier
// M_j = 0x9E3779B1 (2j + 1). Multiplication by an odd number permutes the
// 32-bit integers, so each word is uniform when h is. The rest value
// balances the node's mass against the rounded moving values, so when those
// are dithered too its bits come from a second mixing round of h: bits
// shared with the moving values would correlate with the fraction being
// rounded and bias the mass.
__device__ __forceinline__ uint32_t node_hash(uint32_t node, uint32_t key)
{
    uint32_t h = node * 0x9E3779B1u ^ key * 0x85EBCA77u;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}
// 32 random bits for the pair of values of velocity j (both components)
__device__ __forceinline__ uint32_t rand32(uint32_t h, int j) { return h * (0x9E3779B1u * (2u * (uint32_t)j + 1u)); }

// Stochastic rounding of a pair of FP32 values into a 16-bit pair, in one
// conversion instruction (cvt.rs, sm_100 and later): each value's magnitude
// gets uniform random bits added below its last kept bit and is then
// truncated, so it rounds up with probability equal to the discarded
// fraction. The first value (stored in the low half) takes the low 16 bits
// of m, the second (high half) the high 16 bits; BF16 uses all 16 of a
// half, FP16 its low 13 (the 13 discarded bits of a normal FP16 value).
// .satfinite clamps an overflow to the largest finite value.
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float2 v, uint32_t m)
{
    uint32_t packed;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(packed) : "f"(v.y), "f"(v.x), "r"(m));
    return packed;
}
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float2 v, uint32_t m)
{
    uint32_t packed;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(packed) : "f"(v.y), "f"(v.x), "r"(m));
    return packed;
}

template <>
struct Codec<__half> {
    using Pair = __half2;
    static constexpr bool kDeviation = true;
    static constexpr bool kDitherMoving = false;  // 11 significant bits: only the rest value is dithered
    static __device__ __forceinline__ float load(const __half* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float2 load2(const __half* p) { return __half22float2(__ldg((const __half2*)p)); }
    static __device__ __forceinline__ float val(__half v) { return __half2float(v); }
    static __device__ __forceinline__ float2 val2(__half2 v) { return __half22float2(v); }
    static __device__ __forceinline__ void put2(__half* p, __half a, __half b) { *(__half2*)p = __halves2half2(a, b); }
    // both values rounded to nearest into one pair (one conversion), and the stored values back in FP32
    static __device__ __forceinline__ __half2 rn2(float2 v, float2& back)
    {
        const __half2 h = __float22half2_rn(v);
        back = __half22float2(h);
        return h;
    }
    // stochastic rounding of both values from one random word m (cvt_rs_f16x2),
    // and the stored values back in FP32
    static __device__ __forceinline__ __half2 sr2(float2 v, uint32_t m, float2& back)
    {
        const uint32_t packed = cvt_rs_f16x2(v, m);
        __half2 h;
        *(uint32_t*)&h = packed;
        back = __half22float2(h);
        return h;
    }
    static __device__ __forceinline__ __half rn(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ void store(__half* p, float v) { *p = __float2half_rn(v); }
};
template <>
struct Codec<__nv_bfloat16> {
    using Pair = __nv_bfloat162;
    static constexpr bool kDeviation = true;
    static constexpr bool kDitherMoving = true;  // 8 significant bits: every value is dithered
    static __device__ __forceinline__ float load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float2 load2(const __nv_bfloat16* p)
    {
        return __bfloat1622float2(__ldg((const __nv_bfloat162*)p));
    }
    static __device__ __forceinline__ float val(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ float2 val2(__nv_bfloat162 v) { return __bfloat1622float2(v); }
    static __device__ __forceinline__ void put2(__nv_bfloat16* p, __nv_bfloat16 a, __nv_bfloat16 b)
    {
        *(__nv_bfloat162*)p = __halves2bfloat162(a, b);
    }
    // stochastic rounding of both values from one random word m (cvt_rs_bf16x2),
    // and the stored values back in FP32 (a BF16 value is the upper half of its
    // FP32 word)
    static __device__ __forceinline__ __nv_bfloat162 sr2(float2 v, uint32_t m, float2& back)
    {
        const uint32_t packed = cvt_rs_bf16x2(v, m);
        back = make_float2(__uint_as_float(packed << 16), __uint_as_float(packed & 0xFFFF0000u));
        __nv_bfloat162 h;
        *(uint32_t*)&h = packed;
        return h;
    }
    static __device__ __forceinline__ __nv_bfloat16 rn(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }
};

// Lattice storage: 19 population planes ("slots") of `slot` nodes each, one
// per velocity k, every node holding the two components' values side by side
// (r then b): value (a, k) of the node at offset o sits at element
// 2 (k slot + o) + a. So one 8-byte (FP32) or 4-byte (16-bit) access moves
// both components of a velocity, and a warp's access to one slot covers 256
// (128) contiguous bytes. Inside a slot, node (x, y, z) sits at
//   o = z*plane + (y + 1)*px + (x + gx),
// with gx = 256 bytes of row padding on the left (so x = 0 starts a 256-byte
// unit) and at least one node on the right, and one spare row above and
// below each plane. Nothing reads the padding or the spare rows: the step
// kernels take the periodic images of edge nodes from the real nodes (the
// TMA-staged step loads small extra boxes of real columns and rows for them).
// px, plane and slot count nodes.
struct Layout {
    int nx, ny, nz, px, gx;
    long long plane, slot;
    __host__ __device__ __forceinline__ long long off(int x, int y, int z) const
    {
        return (long long)z * plane + (long long)(y + 1) * px + (x + gx);
    }
    // element index of value (a, k) of the node at slot offset o
    __host__ __device__ __forceinline__ long long at(int a, int k, long long o) const { return 2 * ((long long)k * slot + o) + a; }
};

// Store v for node (x, y) of the plane at zoff through the accessor of one
// (component, velocity) p = f + L.at(a, k, 0).
template <class S>
__device__ __forceinline__ void put(S* __restrict__ p, const Layout& L, int x, int y, long long zoff, float v)
{
    Codec<S>::store(p + 2 * (zoff + (long long)(y + 1) * L.px + L.gx + x), v);
}

// Store both components' values (v0, v1) of velocity k for node (x, y) of the
// plane at zoff (p = f + L.at(0, k, 0)): one paired store.
template <class S>
__device__ __forceinline__ void put_pair(S* __restrict__ p, const Layout& L, int x, int y, long long zoff, float v0,
                                         float v1)
{
    const long long o = zoff + (long long)(y + 1) * L.px + L.gx + x;
    if constexpr (sizeof(S) == 4) Codec<S>::store2(p + 2 * o, v0, v1);
    else Codec<S>::put2(p + 2 * o, Codec<S>::rn(v0), Codec<S>::rn(v1));
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
    uint32_t* clock;                      // [0] step counter of the lattice, [1] CTAs done this step
    Layout L;
    KParams P;
    int tiles_x, tiles_y;  // tile columns: 32-node rows in x; tiles_y even row splits of ny in y
    int zlo, zhi;  // fluid plane range [zlo, zhi)
    int nseg;      // z segments per tile column
    int halo;      // planar walls: bit 0 = plane 0, bit 1 = plane nz-1 is a halo plane of a z slab, not a wall
    uint32_t hkey; // added to a node's offset in the rounding dither's hash (a slab's offset in its lattice)
};

constexpr uint32_t kSelfSolid = 1u << 31;

// Device status word bits (StepArgs::err): a bounded wait gave up; an index
// fell outside its buffer (only a build with LBSC_DEBUG_BOUNDS checks indices);
// an input density failed the re-initialisation's check.
constexpr int kErrWait = 1;
constexpr int kErrBounds = 2;
constexpr int kErrInput = 4;  // lb_reset: a density was negative or not finite
#ifdef LBSC_DEBUG_BOUNDS
constexpr bool kCheckBounds = true;
#else
constexpr bool kCheckBounds = false;
#endif
// Bounds check of the debug build: true if 0 <= i < n; otherwise records
// kErrBounds in the status word and the caller skips the access.
__device__ __forceinline__ bool in_bounds(long long i, long long n, int* err)
{
    if (i >= 0 && i < n) return true;
    atomicOr(err, kErrBounds);
    return false;
}

// first row of y-tile t when n rows are split into nt tiles as evenly as possible
__host__ __device__ __forceinline__ int tile_row(int t, int n, int nt) { return (int)((long long)t * n / nt); }

__host__ __device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Device-side step counter (16-bit storage: it drives the rounding dither).
// Every CTA reads it on entry; the last CTA to finish the step advances it, so
// the count stays right under CUDA-graph replay without any host update.
__device__ __forceinline__ uint32_t clock_read(const uint32_t* clk) { return *(const volatile uint32_t*)clk; }
__device__ __forceinline__ void clock_tick(uint32_t* clk)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&clk[1], 1u);
        if (t == gridDim.x - 1) {
            atomicExch(&clk[1], 0u);
            atomicAdd(&clk[0], 1u);
        }
    }
}

// nodes in 16 bytes (a node holds two values): the ring columns a TMA box
// carries on each side of a tile
template <class S>
__host__ __device__ constexpr int edge_x() { return 16 / (2 * (int)sizeof(S)); }

}  // namespace lbsc
