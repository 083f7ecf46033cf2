// Non-step kernels: initial equilibrium, FP64 conservation sums, moment
// fields for readback, contact-angle reductions and population copies.
// All reductions are deterministic: the conservation sums are exact integer
// (fixed-point) sums; the others use a fixed grid, fixed per-thread ranges,
// warp shuffles and a final pass over the per-block partials in block order.
#include "lb_fields.cuh"

#include <type_traits>

namespace lbsc {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Reduce NV values per thread into out[blockIdx.x*NV + i]; entries listed in
// `is_max` are max-reduced, all others summed. blockDim.x must be kRedThreads.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&acc)[NV], uint32_t is_max, double* out)
{
    __shared__ double sh[kRedThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        const double v = ((is_max >> i) & 1u) ? warp_max(acc[i]) : warp_sum(acc[i]);
        if (lane == 0) sh[warp][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        const int i = threadIdx.x;
        double v = sh[0][i];
        for (int w = 1; w < kRedThreads / 32; ++w) v = ((is_max >> i) & 1u) ? fmax(v, sh[w][i]) : v + sh[w][i];
        out[(long long)blockIdx.x * NV + i] = v;
    }
}

// Sum (or max) nrows partial rows of NV values: block v reduces value v,
// thread t taking rows t, t + 256, ... in order, then a fixed shuffle tree per
// warp and the warps in order. Launched as NV blocks of 256 threads.
template <int NV>
__global__ void __launch_bounds__(256) finish_rows_kernel(const double* __restrict__ part, int nrows, uint32_t is_max,
                                                          double* __restrict__ out)
{
    const int v = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (v >= NV) return;
    const bool mx = (is_max >> v) & 1u;
    double a = mx ? -1e300 : 0.0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        const double p = part[(long long)r * NV + v];
        a = mx ? fmax(a, p) : a + p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double w = __shfl_down_sync(0xffffffffu, a, o);
        a = mx ? fmax(a, w) : a + w;
    }
    __shared__ double sw[8];
    if (lane == 0) sw[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = sw[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = mx ? fmax(t, sw[w]) : t + sw[w];
        out[v] = t;
    }
}

// blocks for n items at `threads` per block, at most cap (grid-stride loops cover the rest)
static int grid_for(long long n, int threads, int cap)
{
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <class S>
__device__ __forceinline__ float decode(const S* p, int k, float ref)
{
    const float v = Codec<S>::load(p);
    if constexpr (Codec<S>::kDeviation) return zeta(k) * (ref + v);
    else return v;
}

// both components' n_k of one node from their paired storage
template <class S>
__device__ __forceinline__ void decode2(const S* p, int k, const float (&ref)[2], float& n0, float& n1)
{
    const float2 v = Codec<S>::load2(p);
    if constexpr (Codec<S>::kDeviation) {
        // explicitly rounded, so that no kernel fuses the product into a later
        // sum: every readback pass sees the same n_k (and the same rho)
        n0 = __fmul_rn(zeta(k), __fadd_rn(ref[0], v.x));
        n1 = __fmul_rn(zeta(k), __fadd_rn(ref[1], v.y));
    } else {
        n0 = v.x;
        n1 = v.y;
    }
}

__device__ __forceinline__ bool node_solid(const FieldArgs& F, int x, int y, int z, long long off)
{
    if (F.general) return (F.nbmask[off] & kSelfSolid) != 0;
    return z == 0 || z == F.L.nz - 1;
}

// ---------------------------------------------------------------- init
// populations at rest: n_k = zeta_k rho (Eq. Equil at u = 0). err (may be
// NULL): kErrInput is set for a density that is negative or not finite.
template <class S>
__global__ void init_kernel(FieldArgs F, S* __restrict__ f, const double* __restrict__ rr, const double* __restrict__ rb,
                            int* err)
{
    const unsigned nxy = (unsigned)F.L.nx * (unsigned)F.L.ny;
    const unsigned N = nxy * (unsigned)F.L.nz;  // below 2^31 (the layout's limit)
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const unsigned z = i / nxy, rem = i - z * nxy;
        const int y = (int)(rem / (unsigned)F.L.nx), x = (int)(rem - (unsigned)y * F.L.nx);
        const double d0 = rr[i], d1 = rb[i];
        if (err && !(isfinite(d0) && d0 >= 0.0 && isfinite(d1) && d1 >= 0.0)) atomicOr(err, kErrInput);
        const float r0 = (float)d0, r1 = (float)d1;
        const long long zoff = (long long)z * F.L.plane;
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if constexpr (Codec<S>::kDeviation)
                put_pair<S>(f + F.L.at(0, k, 0), F.L, x, y, zoff, r0 - F.P.ref[0], r1 - F.P.ref[1]);
            else
                put_pair<S>(f + F.L.at(0, k, 0), F.L, x, y, zoff, zeta(k) * r0, zeta(k) * r1);
        }
    }
}

// ---------------------------------------------------------------- conservation
// cons = {M_r, M_b, Px, Py, Pz, non-finite count, fluid nodes, -}
// A grid-stride walk over the nodes of the fluid planes, x fastest, so that a
// warp's load of one population slot covers consecutive addresses, with a
// node's 38 loads independent of each other. A node's mass and momentum are
// summed in FP32 over its 19 values per component, and each thread adds its
// nodes in FP32. The threads' sums then go into 64-bit integers in units of
// 2^-28 (kConsFix) and are added as integers: across warps, blocks and the
// whole grid, by shuffles and atomics. Integer addition is exact and
// associative, so the totals do not depend on the grid or on the order the
// blocks finish, and no FP64 arithmetic (slow on this GPU) runs per node. The
// last block to finish converts the totals to FP64 into out[0..7] and clears
// the accumulators (acc[0..7], ticket) for the next call.
__device__ __forceinline__ long long to_fix(float v) { return __float2ll_rn(v * kConsFix); }

// With phi non-NULL the same pass also writes phi = rho_r - rho_b of every
// node (0 on solid nodes), summed as the contact angle's phi pass sums it, so
// a measurement of both needs one read of the populations.
template <class S>
__global__ void __launch_bounds__(kRedThreads) cons_kernel(FieldArgs F, const S* __restrict__ f,
                                                           unsigned long long* __restrict__ acc,
                                                           unsigned int* __restrict__ ticket, double* __restrict__ out,
                                                           float* __restrict__ phi)
{
    float m[2] = {0.f, 0.f}, j[3] = {0.f, 0.f, 0.f};
    int bad = 0, fluid = 0;
    const int nx = F.L.nx, ny = F.L.ny;
    const unsigned nxy = (unsigned)nx * (unsigned)ny;
    const unsigned n = nxy * (unsigned)F.L.nz;  // below 2^31 (the layout's limit)
    const unsigned T = gridDim.x * blockDim.x;
    const float ref[2] = {F.P.ref[0], F.P.ref[1]};
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += T) {
        const unsigned zr = i / nxy, rem = i - zr * nxy;
        const int y = (int)(rem / (unsigned)nx), x = (int)(rem - (unsigned)y * nx), z = (int)zr;
        const long long off = F.L.off(x, y, z);
        if (node_solid(F, x, y, z, off)) {
            if (phi) phi[i] = 0.f;
            continue;
        }
        ++fluid;
        float v[2][Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) decode2<S>(f + F.L.at(0, k, off), k, ref, v[0][k], v[1][k]);
        float rho[2], jn[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float nk = v[a][k];
                bad += isfinite(nk) ? 0 : 1;
                s = __fadd_rn(s, nk);  // as the phi pass
                if (cx(k)) jn[0] += cx(k) * nk;
                if (cy(k)) jn[1] += cy(k) * nk;
                if (cz(k)) jn[2] += cz(k) * nk;
            }
            rho[a] = s;
        }
        if (phi) phi[i] = rho[0] - rho[1];
        m[0] += rho[0];
        m[1] += rho[1];
#pragma unroll
        for (int d = 0; d < 3; ++d) j[d] += jn[d];
    }
    // a non-finite value would make the fixed-point conversion meaningless: it is counted instead
    const bool fin = bad == 0 && isfinite(m[0]) && isfinite(m[1]) && isfinite(j[0]) && isfinite(j[1]) && isfinite(j[2]);
    long long q[7] = {fin ? to_fix(m[0]) : 0, fin ? to_fix(m[1]) : 0, fin ? to_fix(j[0]) : 0, fin ? to_fix(j[1]) : 0,
                      fin ? to_fix(j[2]) : 0, (long long)bad + (fin ? 0 : 1) * (bad == 0), (long long)fluid};
#pragma unroll
    for (int v = 0; v < 7; ++v)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) q[v] += __shfl_down_sync(0xffffffffu, q[v], o);
    __shared__ long long sh[kRedThreads / 32][7];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int v = 0; v < 7; ++v) sh[warp][v] = q[v];
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x < 7) {
        long long t = 0;
        for (int w = 0; w < kRedThreads / 32; ++w) t += sh[w][threadIdx.x];
        atomicAdd(&acc[threadIdx.x], (unsigned long long)t);  // two's complement: signed sums wrap correctly
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x < 8) {
        __threadfence();
        const int v = threadIdx.x;
        const long long t = v < 7 ? (long long)atomicExch(&acc[v], 0ull) : 0;
        out[v] = v < 5 ? (double)t / kConsFix : (double)t;
        if (v == 0) *ticket = 0u;
    }
}

// ---------------------------------------------------------------- moment fields
// rho^r, rho^b, total j and psi of every node (psi = wall pseudo-density on solid)
template <class S>
__global__ void fields_kernel(FieldArgs F, const S* __restrict__ f, Scratch W)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % F.L.nx), y = (int)((i / F.L.nx) % F.L.ny), z = (int)(i / ((long long)F.L.nx * F.L.ny));
        const long long off = F.L.off(x, y, z);
        float rho[2] = {0.f, 0.f}, j[3] = {0.f, 0.f, 0.f};
        const bool solid = node_solid(F, x, y, z, off);
        if (!solid) {
            for (int a = 0; a < 2; ++a)
                for (int k = 0; k < Q; ++k) {
                    const float n = decode<S>(f + F.L.at(a, k, off), k, F.P.ref[a]);
                    rho[a] += n;
                    j[0] += cx(k) * n;
                    j[1] += cy(k) * n;
                    j[2] += cz(k) * n;
                }
        }
        W.rho[0][i] = rho[0];
        W.rho[1][i] = rho[1];
        for (int d = 0; d < 3; ++d) W.j[d][i] = j[d];
        for (int a = 0; a < 2; ++a) W.psi[a][i] = solid ? F.P.eta[a] : -expm1f(-rho[a]);
    }
}

// u = (j + F/2) / (rho_r + rho_b), F the total Shan-Chen force (Eq. SCforce)
__global__ void velocity_kernel(FieldArgs F, Scratch W)
{
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        const long long off = F.L.off(x, y, z);
        const float tot = W.rho[0][i] + W.rho[1][i];
        float u[3] = {0.f, 0.f, 0.f};
        if (!node_solid(F, x, y, z, off) && tot > 0.f) {
            float Ft[3] = {0.f, 0.f, 0.f};
            for (int a = 0; a < 2; ++a) {
                float s[3] = {0.f, 0.f, 0.f};
                for (int k = 1; k < Q; ++k) {
                    const long long ip = (long long)wrapi(x + cx(k), nx) +
                                         (long long)nx * (wrapi(y + cy(k), ny) + (long long)ny * wrapi(z + cz(k), nz));
                    const float G = is_axis(k) ? F.P.Gax : F.P.Gdi;
                    const float ps = W.psi[1 - a][ip];
                    s[0] += G * ps * cx(k);
                    s[1] += G * ps * cy(k);
                    s[2] += G * ps * cz(k);
                }
                const float pre = -F.P.gk * W.psi[a][i];
                for (int d = 0; d < 3; ++d) Ft[d] += pre * s[d];
            }
            for (int d = 0; d < 3; ++d) u[d] = (W.j[d][i] + 0.5f * Ft[d]) / tot;
        }
        for (int d = 0; d < 3; ++d) W.u[d][i] = u[d];
    }
}

// phi = rho_r - rho_b of every node into W.rho[0] (0 on solid nodes), the
// contact angle's only input: FP32 sums of each component's 19 values, then
// their difference
template <class S>
__global__ void phi_kernel(FieldArgs F, const S* __restrict__ f, Scratch W)
{
    const int nx = F.L.nx, ny = F.L.ny;
    const unsigned nxy = (unsigned)nx * (unsigned)ny;
    const unsigned N = nxy * (unsigned)F.L.nz;
    const unsigned T = gridDim.x * blockDim.x;
    const float ref[2] = {F.P.ref[0], F.P.ref[1]};
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += T) {
        const unsigned z = i / nxy, rem = i - z * nxy;
        const int y = (int)(rem / (unsigned)nx), x = (int)(rem - (unsigned)y * nx);
        const long long off = F.L.off(x, y, (int)z);
        float rho[2] = {0.f, 0.f};
        if (!node_solid(F, x, y, (int)z, off)) {
            float v[2][Q];
#pragma unroll
            for (int k = 0; k < Q; ++k) decode2<S>(f + F.L.at(0, k, off), k, ref, v[0][k], v[1][k]);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int k = 0; k < Q; ++k) rho[a] = __fadd_rn(rho[a], v[a][k]);  // as the conservation pass
        }
        W.rho[0][i] = rho[0] - rho[1];
    }
}

// ---------------------------------------------------------------- contact angle
// phi - level in FP64 at a node whose phi is the FP32 value p
__device__ __forceinline__ double phi_at(float p, double level) { return (double)p - level; }

// p > level in FP64, out of line: the rare case the FP32 test below cannot decide
__device__ __noinline__ bool above_fp64(float p, double level) { return (double)p > level; }

// p > level, i.e. phi_at(p, level) > 0, taken in FP32 where that is exact: when
// level is an FP32 number, or when p is far from it (the margin exceeds the
// rounding of level to FP32 many times over); else in FP64.
__device__ __forceinline__ bool above(float p, float lf, bool lexact, double level)
{
    if (lexact || fabsf(p - lf) > 1e-6f * (fabsf(p) + fabsf(lf)) + 1e-30f) return p > lf;
    return above_fp64(p, level);
}

// Positive length along x, from a node to its +x neighbour, of the linear
// interpolant of phi - level on the reference plane z0 + fz (p: phi at the
// node, above it, at the +x neighbour and above that). Out of line, so that
// its FP64 work runs only on that plane's rows.
__device__ __noinline__ double plane_length(float p0, float p0up, float p1, float p1up, double fz, double level)
{
    const double a0 = (1 - fz) * phi_at(p0, level) + fz * phi_at(p0up, level);
    const double a1 = (1 - fz) * phi_at(p1, level) + fz * phi_at(p1up, level);
    if (a0 > 0 && a1 > 0) return 1.0;
    if (a0 <= 0 && a1 <= 0) return 0.0;
    return a0 > 0 ? a0 / (a0 - a1) : a1 / (a1 - a0);
}

// An interface crossing between node (x, y, z) (phi = p0) and its neighbour
// along axis d (phi = p1): the top crossing (along z, from phi > level
// below to phi <= level above) and the sphere-fit sums of the crossing point at
// or above the reference plane, into the thread's accumulators acc[i * stride].
// Kept out of line so that the FP64 work runs only in the warps that meet a
// crossing instead of being predicated into every node's path.
__device__ __noinline__ void add_crossing(double* acc, int stride, int x, int y, int z, int d, float p0, float p1,
                                         double level, bool s0, double zref)
{
    const double q0 = phi_at(p0, level), q1 = phi_at(p1, level);
    const double t = q0 / (q0 - q1);
    if (d == 2 && s0) acc[0] = fmax(acc[0], z + t);  // phi > level below, <= level above
    const double pxv = x + t * (d == 0), pyv = y + t * (d == 1), pzv = z + t * (d == 2);
    if (pzv < zref) return;
    const double row[4] = {2 * pxv, 2 * pyv, 2 * pzv, 1.0};
    const double rhs = pxv * pxv + pyv * pyv + pzv * pzv;
    acc[2 * stride] += 1.0;
    int m = 3;
    for (int r = 0; r < 4; ++r)
        for (int q = r; q < 4; ++q) acc[(m++) * stride] += row[r] * row[q];
    for (int r = 0; r < 4; ++r) acc[(13 + r) * stride] += row[r] * rhs;
}

// One warp per lattice row, a lane per node, reading phi at the node and at
// its +x, +y, +z neighbours (the latter from L1/L2):
//  [0]  (max) top phi = level crossing: z + p0/(p0 - p1) where phi > level
//       below and <= level above (both nodes fluid);
//  [1]  positive length along x of the reference-plane interpolant of phi
//       (the node at z0 adds its segment to x + 1, periodic);
//  [2..16] sphere-fit sums over crossings along +x, +y, +z at or above the
//       reference plane: count, the 10 upper entries of M = sum row row^T and
//       the 4 of v = sum row |p|^2, row = (2p, 1);
//  [17] (max) max of phi over fluid nodes, [18] (max) of -phi (the contrast).
// FP64 arithmetic (slow on this GPU) runs only at crossings and on the
// reference plane; a thread's FP64 sums wait in shared memory, and a warp
// reduces a value only if one of its lanes holds a contribution to it.
__global__ void __launch_bounds__(kRedThreads) angle_kernel(FieldArgs F, Scratch W, double zref, double level,
                                                            double* __restrict__ part)
{
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    __shared__ double sacc[kAngleVals][kRedThreads];
    const int tid = threadIdx.x;
#define ACC(i) sacc[i][tid]
    for (int i = 0; i < 17; ++i) ACC(i) = 0.0;
    ACC(0) = -1e300;
    float pmax = -3.0e38f, pmin = 3.0e38f;
    const int z0 = (int)floor(zref);
    const double fz = zref - z0;
    const float lf = (float)level;
    const bool lexact = (double)lf == level;
    const float* __restrict__ P = W.rho[0];
    const unsigned nxy = (unsigned)nx * (unsigned)ny;
    // Interface crossings are rare and scattered: a lane that meets one would
    // run the FP64 work of add_crossing alone, at the cost of a whole warp's.
    // So the warp queues its crossings in shared memory, in lane order, and
    // works through them 32 at a time with every lane busy; which lane sums
    // which crossing depends only on the data, so the sums are reproducible.
    __shared__ int4 qpos[kRedThreads / 32][64];     // (x, y, z, axis)
    __shared__ float2 qphi[kRedThreads / 32][64];   // (phi at the node, phi at the neighbour)
    const int lane = tid & 31, warp = tid >> 5;
    int queued = 0;
    auto drain = [&](int n) {  // lanes < n take a queued crossing each, then the queue shifts by n
        __syncwarp();
        if (lane < n) {
            const int4 q = qpos[warp][lane];
            const float2 f = qphi[warp][lane];
            const bool s0 = above(f.x, lf, lexact, level);
            add_crossing(&sacc[0][tid], kRedThreads, q.x, q.y, q.z, q.w, f.x, f.y, level, s0, zref);
        }
        __syncwarp();
        if (lane + n < queued) {  // at most 31 left, read from [n, queued), written to [0, queued - n)
            const int4 q = qpos[warp][lane + n];
            const float2 f = qphi[warp][lane + n];
            qpos[warp][lane] = q;
            qphi[warp][lane] = f;
        }
        __syncwarp();
        queued -= n;
    };
    // a warp takes lattice rows (y, z) = w, w + W, ... (W warps in the grid), its lanes x = lane, lane + 32, ...
    const int rows = ny * nz, nwarps = gridDim.x * (kRedThreads / 32);
    for (int r = blockIdx.x * (kRedThreads / 32) + warp; r < rows; r += nwarps)
    for (int xb = 0; xb < nx; xb += 32) {  // warp-uniform: the queue needs the whole warp
        const int x = xb + lane;
        const bool in = x < nx;
        const int z = r / ny, y = r - z * ny;
        const unsigned i = (unsigned)r * (unsigned)nx + (unsigned)(in ? x : nx - 1);
        // the node and its +x, +y, +z neighbours (the node itself past an edge), loaded together
        const float p0 = P[i];
        const float pn[3] = {P[in && x + 1 < nx ? i + 1 : i], P[y + 1 < ny ? i + nx : i], P[z + 1 < nz ? i + nxy : i]};
        if (in && z == z0 && z0 + 1 < nz) {  // reference plane: every column, solid or not
            const unsigned i1 = x + 1 < nx ? i + 1 : i - x;
            ACC(1) += plane_length(p0, pn[2], P[i1], P[i1 + nxy], fz, level);
        }
        const bool fluid = in && (!F.general ? !(z == 0 || z == nz - 1) : (F.nbmask[F.L.off(x, y, z)] & kSelfSolid) == 0);
        if (fluid) {
            pmax = fmaxf(pmax, p0);
            pmin = fminf(pmin, p0);
        }
        const bool s0 = above(p0, lf, lexact, level);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int x1 = x + (d == 0), y1 = y + (d == 1), z1 = z + (d == 2);
            bool cross = fluid && x1 < nx && y1 < ny && z1 < nz;
            if (cross) cross = !(F.general ? (F.nbmask[F.L.off(x1, y1, z1)] & kSelfSolid) != 0 : z1 == nz - 1);
            if (cross) cross = s0 != above(pn[d], lf, lexact, level);
            const unsigned m = __ballot_sync(0xffffffffu, cross);
            if (cross) {
                const int at = queued + __popc(m & ((1u << lane) - 1u));
                qpos[warp][at] = make_int4(x, y, z, d);
                qphi[warp][at] = make_float2(p0, pn[d]);
            }
            queued += __popc(m);
            if (queued >= 32) drain(32);
        }
    }
    if (queued > 0) drain(queued);
    // block reduction: FP32 maxima by shuffles; FP64 values only in warps that hold some
    __shared__ double sh[kRedThreads / 32][kAngleVals];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pmax = fmaxf(pmax, __shfl_down_sync(0xffffffffu, pmax, o));
        pmin = fminf(pmin, __shfl_down_sync(0xffffffffu, pmin, o));
    }
    if (lane == 0) {
        sh[warp][17] = pmax > -3.0e38f ? (double)pmax : -1e300;
        sh[warp][18] = pmin < 3.0e38f ? -(double)pmin : -1e300;
    }
    for (int v = 0; v < 17; ++v) {
        const bool is_max = v == 0;
        double val = ACC(v);
        // a contribution changed the value's bits from their start (integer test: no FP64 operation)
        const bool held = __double_as_longlong(val) != __double_as_longlong(is_max ? -1e300 : 0.0);
        if (__any_sync(0xffffffffu, held)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double w = __shfl_down_sync(0xffffffffu, val, o);
                val = is_max ? fmax(val, w) : val + w;
            }
        }
        if (lane == 0) sh[warp][v] = val;
    }
#undef ACC
    __syncthreads();
    if (tid < kAngleVals) {
        const bool is_max = (kAngleMaxMask >> tid) & 1u;
        double v = sh[0][tid];
        for (int w = 1; w < kRedThreads / 32; ++w) v = is_max ? fmax(v, sh[w][tid]) : v + sh[w][tid];
        part[(long long)blockIdx.x * kAngleVals + tid] = v;
    }
}

// ---------------------------------------------------------------- pressure tensor
// Pressure tensor of Sec. 4.1 at a node, in FP64 from the FP32 fields:
//   P_ij = sum_a sum_k (c_ki - u_i)(c_kj - u_j) n_k^a
//        + 1/4 sum over the two ordered component pairs (a, abar) of
//          g kappa sum_k G_k [psi^a(x) psi^abar(x+c_k) + psi^abar(x) psi^a(x+c_k)] c_ki c_kj,
// u the moments' velocity (j + F/2)/rho, psi of a solid neighbour the wall
// pseudo-density (the force's reading of the wall). Both ordered pairs give the
// same bracket, so the interaction is 1/2 g kappa sum_k G_k [..] c_ki c_kj.
// Components xx, yy, zz, xy, xz, yz; zero on solid nodes.
template <class S>
__device__ bool node_pressure(const FieldArgs& F, const S* __restrict__ f, const Scratch& W, int x, int y, int z,
                              double (&P)[6])
{
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    for (int c = 0; c < 6; ++c) P[c] = 0.0;
    const long long off = F.L.off(x, y, z);
    if (node_solid(F, x, y, z, off)) return false;
    const long long i = (long long)x + (long long)nx * (y + (long long)ny * z);
    const double u[3] = {W.u[0][i], W.u[1][i], W.u[2][i]};
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < Q; ++k) {
            const double n = decode<S>(f + F.L.at(a, k, off), k, F.P.ref[a]);
            const double d[3] = {cx(k) - u[0], cy(k) - u[1], cz(k) - u[2]};
            P[0] += d[0] * d[0] * n;
            P[1] += d[1] * d[1] * n;
            P[2] += d[2] * d[2] * n;
            P[3] += d[0] * d[1] * n;
            P[4] += d[0] * d[2] * n;
            P[5] += d[1] * d[2] * n;
        }
    const double pr = W.psi[0][i], pb = W.psi[1][i];
    double I[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 1; k < Q; ++k) {
        const long long ip = (long long)wrapi(x + cx(k), nx) + (long long)nx * (wrapi(y + cy(k), ny) + (long long)ny * wrapi(z + cz(k), nz));
        const double G = is_axis(k) ? F.P.Gax : F.P.Gdi;
        const double pair = G * (pr * (double)W.psi[1][ip] + pb * (double)W.psi[0][ip]);
        const double c3[3] = {(double)cx(k), (double)cy(k), (double)cz(k)};
        I[0] += pair * c3[0] * c3[0];
        I[1] += pair * c3[1] * c3[1];
        I[2] += pair * c3[2] * c3[2];
        I[3] += pair * c3[0] * c3[1];
        I[4] += pair * c3[0] * c3[2];
        I[5] += pair * c3[1] * c3[2];
    }
    const double h = 0.5 * (double)F.P.gk;
    for (int c = 0; c < 6; ++c) P[c] += h * I[c];
    return true;
}

// every node: P[c*N + i] (FP64)
template <class S>
__global__ void pressure_field_kernel(FieldArgs F, const S* __restrict__ f, Scratch W, double* __restrict__ out)
{
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        double P[6];
        node_pressure<S>(F, f, W, x, y, z, P);
        for (int c = 0; c < 6; ++c) out[c * N + i] = P[c];
    }
}

// one block per z plane: sums over the plane's fluid nodes of the six
// components, phi = rho_r - rho_b and the count -> out[z*8 + v]
template <class S>
__global__ void __launch_bounds__(kRedThreads) pressure_plane_kernel(FieldArgs F, const S* __restrict__ f, Scratch W,
                                                                     double* __restrict__ out)
{
    const int nx = F.L.nx, ny = F.L.ny, z = blockIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = threadIdx.x; c < nx * ny; c += blockDim.x) {
        const int x = c % nx, y = c / nx;
        double P[6];
        if (!node_pressure<S>(F, f, W, x, y, z, P)) continue;
        const long long i = (long long)c + (long long)nx * ny * z;
        for (int v = 0; v < 6; ++v) acc[v] += P[v];
        acc[6] += (double)W.rho[0][i] - (double)W.rho[1][i];
        acc[7] += 1.0;
    }
    block_reduce<8>(acc, 0u, out);
}

// Radial bins about a centre: per fluid node with z >= zmin at distance
// r > 0 (minimum image along x, y, and z for the mask-driven periodic
// geometry), bin floor(r/dr) < nbins collects P_N = n.P.n,
// P_T = (tr P - P_N)/2, phi and 1. Sums are kept in 64-bit fixed point
// (units of 2^-30) so that the atomic accumulation is exact and the result
// does not depend on the order the nodes are added in.
__global__ void __launch_bounds__(kRedThreads) pressure_radial_kernel(FieldArgs F, const void* f, int prec, Scratch W,
                                                                      double cxx, double cyy, double czz, double dr,
                                                                      int nbins, double zmin,
                                                                      unsigned long long* __restrict__ out)
{
    __shared__ unsigned long long sh[kRadialBinsMax * 4];
    for (int b = threadIdx.x; b < nbins * 4; b += blockDim.x) sh[b] = 0ull;
    __syncthreads();
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long long)nx * ny));
        if (z < zmin) continue;
        double d[3] = {x - cxx, y - cyy, z - czz};
        d[0] -= nx * rint(d[0] / nx);
        d[1] -= ny * rint(d[1] / ny);
        if (F.general) d[2] -= nz * rint(d[2] / nz);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(r > 0)) continue;
        const double bf = floor(r / dr);
        if (bf >= nbins) continue;
        double P[6];
        bool fluid;
        if (prec == 0) fluid = node_pressure<float>(F, (const float*)f, W, x, y, z, P);
        else if (prec == 1) fluid = node_pressure<__half>(F, (const __half*)f, W, x, y, z, P);
        else fluid = node_pressure<__nv_bfloat16>(F, (const __nv_bfloat16*)f, W, x, y, z, P);
        if (!fluid) continue;
        const double n[3] = {d[0] / r, d[1] / r, d[2] / r};
        const double T[3][3] = {{P[0], P[3], P[4]}, {P[3], P[1], P[5]}, {P[4], P[5], P[2]}};
        double pn = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) pn += n[a] * T[a][b] * n[b];
        const double pt = 0.5 * (P[0] + P[1] + P[2] - pn);
        const double phi = (double)W.rho[0][i] - (double)W.rho[1][i];
        const int b = (int)bf;
        atomicAdd(&sh[b * 4 + 0], (unsigned long long)__double2ll_rn(pn * kRadialFix));
        atomicAdd(&sh[b * 4 + 1], (unsigned long long)__double2ll_rn(pt * kRadialFix));
        atomicAdd(&sh[b * 4 + 2], (unsigned long long)__double2ll_rn(phi * kRadialFix));
        atomicAdd(&sh[b * 4 + 3], 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins * 4; b += blockDim.x)
        if (sh[b]) atomicAdd(&out[b], sh[b]);
}

// ---------------------------------------------------------------- population copies
template <class S>
__global__ void get_pop_kernel(FieldArgs F, const S* __restrict__ f, double* __restrict__ out)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N * 2 * Q; i += (long long)gridDim.x * blockDim.x) {
        const int ak = (int)(i / N);
        const long long n = i % N;
        const int a = ak / Q, k = ak % Q;
        const int x = (int)(n % F.L.nx), y = (int)((n / F.L.nx) % F.L.ny), z = (int)(n / ((long long)F.L.nx * F.L.ny));
        const long long off = F.L.off(x, y, z);
        out[i] = decode<S>(f + F.L.at(a, k, off), k, F.P.ref[a]);
    }
}

template <class S>
__global__ void set_pop_kernel(FieldArgs F, S* __restrict__ f, const double* __restrict__ in)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N * 2 * Q; i += (long long)gridDim.x * blockDim.x) {
        const int ak = (int)(i / N);
        const long long n = i % N;
        const int a = ak / Q, k = ak % Q;
        const int x = (int)(n % F.L.nx), y = (int)((n / F.L.nx) % F.L.ny), z = (int)(n / ((long long)F.L.nx * F.L.ny));
        const long long off = F.L.off(x, y, z);
        float v = (float)in[i];
        if constexpr (Codec<S>::kDeviation) v = (float)(in[i] / (double)zeta(k) - (double)F.P.ref[a]);
        put<S>(f + F.L.at(a, k, 0), F.L, x, y, (long long)z * F.L.plane, v);
    }
}

// ---------------------------------------------------------------- launchers

__global__ void clock_set_kernel(uint32_t* clk, uint32_t v)
{
    clk[0] = v;
    clk[1] = 0;
}

cudaError_t launch_clock_set(uint32_t* clk, uint32_t v, cudaStream_t st)
{
    clock_set_kernel<<<1, 1, 0, st>>>(clk, v);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_init(const FieldArgs& F, S* f, const double* rr, const double* rb, cudaStream_t st, int* err)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    init_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, rr, rb, err);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_conservation(const FieldArgs& F, const S* f, unsigned long long* acc, unsigned int* ticket,
                                double* out, cudaStream_t st, float* phi)
{
    // one wave of resident blocks (a grid-stride loop over the nodes): a partial
    // last wave of a fixed grid left most SMs idle at the end
    static int blocks = 0;
    if (!blocks) {
        int dev = 0, nsm = 0, occ = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ==
                                                      cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, cons_kernel<S>, kRedThreads, 0) == cudaSuccess &&
            nsm * occ > 0)
            blocks = nsm * occ < kConsBlocks ? nsm * occ : kConsBlocks;
        else
            blocks = kConsBlocks;
    }
    cons_kernel<S><<<blocks, kRedThreads, 0, st>>>(F, f, acc, ticket, out, phi);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_fields(const FieldArgs& F, const S* f, const Scratch& W, bool velocity, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    fields_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, W);
    if (velocity) velocity_kernel<<<grid_for(N, 256, 65536), 256, 0, st>>>(F, W);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_phi(const FieldArgs& F, const S* f, const Scratch& W, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    phi_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, W);
    return cudaGetLastError();
}

cudaError_t launch_angle(const FieldArgs& F, const Scratch& W, double zref, double level, double* part, double* out,
                         cudaStream_t st)
{
    angle_kernel<<<kAngleBlocks, kRedThreads, 0, st>>>(F, W, zref, level, part);
    finish_rows_kernel<kAngleVals><<<kAngleVals, 256, 0, st>>>(part, kAngleBlocks, kAngleMaxMask, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_get_pop(const FieldArgs& F, const S* f, double* out, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz * 2 * Q;
    get_pop_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_set_pop(const FieldArgs& F, S* f, const double* in, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz * 2 * Q;
    set_pop_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, in);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_pressure_field(const FieldArgs& F, const S* f, const Scratch& W, double* out, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    pressure_field_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, W, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_pressure_planes(const FieldArgs& F, const S* f, const Scratch& W, double* out, cudaStream_t st)
{
    pressure_plane_kernel<S><<<F.L.nz, kRedThreads, 0, st>>>(F, f, W, out);
    return cudaGetLastError();
}

cudaError_t launch_pressure_radial(const FieldArgs& F, const void* f, int prec, const Scratch& W, const double* centre,
                                   double dr, int nbins, double zmin, unsigned long long* out, cudaStream_t st)
{
    if (nbins < 1 || nbins > kRadialBinsMax) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * 4 * nbins, st);
    if (e != cudaSuccess) return e;
    pressure_radial_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(F, f, prec, W, centre[0], centre[1], centre[2], dr,
                                                                nbins, zmin, out);
    return cudaGetLastError();
}

#define LBSC_INST(S)                                                                                  \
    template cudaError_t launch_init<S>(const FieldArgs&, S*, const double*, const double*, cudaStream_t, int*); \
    template cudaError_t launch_conservation<S>(const FieldArgs&, const S*, unsigned long long*, unsigned int*, \
                                                double*, cudaStream_t, float*);                                \
    template cudaError_t launch_fields<S>(const FieldArgs&, const S*, const Scratch&, bool, cudaStream_t); \
    template cudaError_t launch_phi<S>(const FieldArgs&, const S*, const Scratch&, cudaStream_t);      \
    template cudaError_t launch_get_pop<S>(const FieldArgs&, const S*, double*, cudaStream_t);       \
    template cudaError_t launch_set_pop<S>(const FieldArgs&, S*, const double*, cudaStream_t);   \
    template cudaError_t launch_pressure_field<S>(const FieldArgs&, const S*, const Scratch&, double*, cudaStream_t); \
    template cudaError_t launch_pressure_planes<S>(const FieldArgs&, const S*, const Scratch&, double*, cudaStream_t);
LBSC_INST(float)
LBSC_INST(__half)
LBSC_INST(__nv_bfloat16)

}  // namespace lbsc
