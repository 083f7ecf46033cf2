// Non-step kernels: initial equilibrium, FP64 conservation sums, moment
// fields for readback, contact-angle reductions and population copies.
// All reductions are deterministic: fixed grid, fixed per-thread ranges,
// warp shuffles, then a single-block pass over the per-block partials in
// block order.
#include "lb_fields.cuh"

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

// Sum (or max) nblocks partial rows of NV values in block order.
template <int NV>
__global__ void finish_kernel(const double* __restrict__ part, int nblocks, uint32_t is_max, double* __restrict__ out)
{
    const int i = threadIdx.x;
    if (i >= NV) return;
    const bool mx = (is_max >> i) & 1u;
    double v = mx ? -1e300 : 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double p = part[(long long)b * NV + i];
        v = mx ? fmax(v, p) : v + p;
    }
    out[i] = v;
}

template <class S>
__device__ __forceinline__ float decode(const S* p, int k, float ref)
{
    const float v = Codec<S>::load(p);
    if constexpr (Codec<S>::kDeviation) return zeta(k) * (ref + v);
    else return v;
}

__device__ __forceinline__ bool node_solid(const FieldArgs& F, int x, int y, int z, long long off)
{
    if (F.general) return (F.nbmask[off] & kSelfSolid) != 0;
    return z == 0 || z == F.L.nz - 1;
}

// ---------------------------------------------------------------- init
// populations at rest: n_k = zeta_k rho (Eq. Equil at u = 0)
template <class S>
__global__ void init_kernel(FieldArgs F, S* __restrict__ f, const double* __restrict__ rr, const double* __restrict__ rb)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % F.L.nx), y = (int)((i / F.L.nx) % F.L.ny), z = (int)(i / ((long long)F.L.nx * F.L.ny));
        for (int a = 0; a < 2; ++a) {
            const float rho = (float)(a == 0 ? rr[i] : rb[i]);
            for (int k = 0; k < Q; ++k) {
                float v;
                if constexpr (Codec<S>::kDeviation) v = rho - F.P.ref[a];
                else v = zeta(k) * rho;
                put<S>(f + (long long)(a * Q + k) * F.L.slot, F.L, x, y, (long long)z * F.L.plane, v);
            }
        }
    }
}

// ---------------------------------------------------------------- conservation
// cons = {M_r, M_b, Px, Py, Pz, non-finite count, fluid nodes, -}
template <class S>
__global__ void __launch_bounds__(kRedThreads) cons_kernel(FieldArgs F, const S* __restrict__ f, double* __restrict__ part)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % F.L.nx), y = (int)((i / F.L.nx) % F.L.ny), z = (int)(i / ((long long)F.L.nx * F.L.ny));
        const long long off = F.L.off(x, y, z);
        if (node_solid(F, x, y, z, off)) continue;
        acc[6] += 1.0;
        for (int a = 0; a < 2; ++a) {
            float rho = 0.f, j[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < Q; ++k) {
                const float n = decode<S>(f + (long long)(a * Q + k) * F.L.slot + off, k, F.P.ref[a]);
                if (!isfinite(n)) acc[5] += 1.0;
                rho += n;
                j[0] += cx(k) * n;
                j[1] += cy(k) * n;
                j[2] += cz(k) * n;
            }
            acc[a] += rho;
            acc[2] += j[0];
            acc[3] += j[1];
            acc[4] += j[2];
        }
    }
    block_reduce<8>(acc, 0u, part);
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
                    const float n = decode<S>(f + (long long)(a * Q + k) * F.L.slot + off, k, F.P.ref[a]);
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

// ---------------------------------------------------------------- contact angle
// Per column (x, y): top phi = 0 crossing (max), positive length of the
// reference-plane interpolant along x, and sphere-fit sums of interface points.
// acc = {top, area, npts, M00, M01, M02, M03, M11, M12, M13, M22, M23, M33, v0, v1, v2, v3}
__global__ void __launch_bounds__(kRedThreads) angle_kernel(FieldArgs F, Scratch W, double zref, double level,
                                                            double* __restrict__ part)
{
    const int nx = F.L.nx, ny = F.L.ny, nz = F.L.nz;
    double acc[kAngleVals];
    for (int i = 0; i < kAngleVals; ++i) acc[i] = 0.0;
    acc[0] = -1e300;
    const int z0 = (int)floor(zref);
    const double fz = zref - z0;
    auto phi = [&](int x, int y, int z) -> double {
        const long long i = (long long)x + (long long)nx * (y + (long long)ny * z);
        return (double)W.rho[0][i] - (double)W.rho[1][i] - level;
    };
    auto solid = [&](int x, int y, int z) -> bool {
        const long long off = F.L.off(x, y, z);
        return node_solid(F, x, y, z, off);
    };
    const long long ncols = (long long)nx * ny;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncols; c += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)(c / nx);
        for (int z = 0; z + 1 < nz; ++z) {
            if (solid(x, y, z) || solid(x, y, z + 1)) continue;
            const double p0 = phi(x, y, z), p1 = phi(x, y, z + 1);
            if (p0 > 0 && p1 <= 0) acc[0] = fmax(acc[0], z + p0 / (p0 - p1));
        }
        if (z0 >= 0 && z0 + 1 < nz) {
            const int x1 = (x + 1) % nx;
            const double a0 = (1 - fz) * phi(x, y, z0) + fz * phi(x, y, z0 + 1);
            const double a1 = (1 - fz) * phi(x1, y, z0) + fz * phi(x1, y, z0 + 1);
            double len;
            if (a0 > 0 && a1 > 0) len = 1.0;
            else if (a0 <= 0 && a1 <= 0) len = 0.0;
            else if (a0 > 0) len = a0 / (a0 - a1);
            else len = a1 / (a1 - a0);
            acc[1] += len;
        }
        for (int z = 0; z < nz; ++z) {
            if (solid(x, y, z)) continue;
            const double p0 = phi(x, y, z);
            for (int d = 0; d < 3; ++d) {
                const int x1 = x + (d == 0), y1 = y + (d == 1), z1 = z + (d == 2);
                if (x1 >= nx || y1 >= ny || z1 >= nz || solid(x1, y1, z1)) continue;
                const double p1 = phi(x1, y1, z1);
                if ((p0 > 0) == (p1 > 0)) continue;
                const double t = p0 / (p0 - p1);
                const double pxv = x + t * (d == 0), pyv = y + t * (d == 1), pzv = z + t * (d == 2);
                if (pzv < zref) continue;
                const double row[4] = {2 * pxv, 2 * pyv, 2 * pzv, 1.0};
                const double rhs = pxv * pxv + pyv * pyv + pzv * pzv;
                acc[2] += 1.0;
                int m = 3;
                for (int r = 0; r < 4; ++r)
                    for (int q = r; q < 4; ++q) acc[m++] += row[r] * row[q];
                for (int r = 0; r < 4; ++r) acc[13 + r] += row[r] * rhs;
            }
        }
    }
    block_reduce<kAngleVals>(acc, 1u, part);
}

// ---------------------------------------------------------------- ghost images
// Refresh the ghost columns x = -1, nx and rows y = -1, ny (corners
// included) of planes [z0, z1) from the real nodes they mirror.
template <class S>
__global__ void ghost_kernel(Layout L, S* __restrict__ f, int z0, int z1)
{
    const int per_plane = 2 * L.ny + 2 * (L.nx + 2);
    const long long total = (long long)2 * Q * (z1 - z0) * per_plane;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int item = (int)(i % per_plane);
        const long long rest = i / per_plane;
        const int z = z0 + (int)(rest % (z1 - z0));
        const int ak = (int)(rest / (z1 - z0));
        S* p = f + (long long)ak * L.slot;
        int sx, sy, gx, gy;  // source node, ghost position
        if (item < 2 * L.ny) {
            sy = gy = item >> 1;
            gx = (item & 1) ? L.nx : -1;
            sx = (item & 1) ? 0 : L.nx - 1;
        } else {
            const int r = item - 2 * L.ny;
            gx = (r >> 1) - 1;  // -1 .. nx
            sx = wrapi(gx, L.nx);
            gy = (r & 1) ? L.ny : -1;
            sy = (r & 1) ? 0 : L.ny - 1;
        }
        p[L.off(gx, gy, z)] = p[L.off(sx, sy, z)];
    }
}

template <class S>
cudaError_t launch_ghosts(const Layout& L, S* f, int z0, int z1, cudaStream_t st)
{
    if (z1 <= z0) return cudaSuccess;
    const long long total = (long long)2 * Q * (z1 - z0) * (2 * L.ny + 2 * (L.nx + 2));
    long long b = (total + 255) / 256;
    if (b > 4096) b = 4096;
    ghost_kernel<S><<<(int)b, 256, 0, st>>>(L, f, z0, z1);
    return cudaGetLastError();
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
        out[i] = decode<S>(f + (long long)ak * F.L.slot + off, k, F.P.ref[a]);
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
        put<S>(f + (long long)ak * F.L.slot, F.L, x, y, (long long)z * F.L.plane, v);
    }
}

// ---------------------------------------------------------------- launchers
static int grid_for(long long n, int threads, int cap)
{
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

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
cudaError_t launch_init(const FieldArgs& F, S* f, const double* rr, const double* rb, cudaStream_t st)
{
    const long long N = (long long)F.L.nx * F.L.ny * F.L.nz;
    init_kernel<S><<<grid_for(N, 256, 65536), 256, 0, st>>>(F, f, rr, rb);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_conservation(const FieldArgs& F, const S* f, double* part, double* out, cudaStream_t st)
{
    cons_kernel<S><<<kRedBlocks, kRedThreads, 0, st>>>(F, f, part);
    finish_kernel<8><<<1, 32, 0, st>>>(part, kRedBlocks, 0u, out);
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

cudaError_t launch_angle(const FieldArgs& F, const Scratch& W, double zref, double level, double* part, double* out,
                         cudaStream_t st)
{
    angle_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(F, W, zref, level, part);
    finish_kernel<kAngleVals><<<1, 32, 0, st>>>(part, kRedBlocks, 1u, out);
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

#define LBSC_INST(S)                                                                                  \
    template cudaError_t launch_init<S>(const FieldArgs&, S*, const double*, const double*, cudaStream_t); \
    template cudaError_t launch_conservation<S>(const FieldArgs&, const S*, double*, double*, cudaStream_t); \
    template cudaError_t launch_fields<S>(const FieldArgs&, const S*, const Scratch&, bool, cudaStream_t); \
    template cudaError_t launch_get_pop<S>(const FieldArgs&, const S*, double*, cudaStream_t);       \
    template cudaError_t launch_set_pop<S>(const FieldArgs&, S*, const double*, cudaStream_t);   \
    template cudaError_t launch_ghosts<S>(const Layout&, S*, int, int, cudaStream_t);
LBSC_INST(float)
LBSC_INST(__half)
LBSC_INST(__nv_bfloat16)

}  // namespace lbsc
