// Discrete adjoint of the time step (Sec. 2) with respect to the wall
// pseudo-densities (eta_wall_r, eta_wall_b), for the planar-wall geometry.
//
// Forward step at a fluid node y, component a (omega = 1/tau):
//   rho^a = sum_k n_k, j^a = sum_k n_k c_k, psi^a = 1 - exp(-rho^a)
//   F^a   = -g kappa psi^a(y) S^a,  S^a = sum_m G_m psi~^abar(y + c_m) c_m
//           (psi~ = wall pseudo-density eta_abar where y + c_m is solid)
//   u'    = sum_b omega_b j^b / D,  D = sum_b omega_b rho^b
//   u^a   = u' + tau_a F^a / rho^a
//   q_k   = zeta_k rho^a (1 + P_k(u^a)),  n*_k = (1 - omega_a) n_k + omega_a q_k
//   stream: n_k(y + c_k, t+1) = n*_k(y), or n_kbar(y, t+1) = n*_k(y) into a wall
// The adjoint runs these in reverse for lambda = dJ/dn:
//   mu_k(y) = dJ/dn*_k(y) = lambda_k(y + c_k) or lambda_kbar(y) (wall)
//   then back through BGK, the equilibrium, the velocity shift, u', the force
//   and psi, ending in lambda_k(y, t) = (1 - omega) mu_k + rhobar + c_k . jbar.
// The force couples neighbours: node y sends Sbar^a = -g kappa psi^a(y) Fbar^a
// to psi^abar of its 18 neighbours (or to eta_abar where the neighbour is a
// wall); a second pass gathers those contributions.
//
// Adjoint arrays are dense, index x + nx*(y + ny*z), FP32; gradient sums FP64.
#include "lb_fields.cuh"

namespace lbsc {

__device__ __forceinline__ long long didx(int x, int y, int z, int nx, int ny)
{
    return (long long)x + (long long)nx * (y + (long long)ny * z);
}
__device__ __forceinline__ bool wall_z(int z, int nz) { return z == 0 || z == nz - 1; }
// coordinates of dense node index i (32-bit: node counts stay below 2^31)
__device__ __forceinline__ void node_xyz(int i, int nx, int ny, int& x, int& y, int& z)
{
    const int t = i / nx;
    x = i - t * nx;
    z = t / ny;
    y = t - z * ny;
}

// forward rho, j, psi of the stored state (lattice layout L)
template <class S>
__global__ void adj_forward_kernel(Layout L, KParams P, const S* __restrict__ f, AdjFields A)
{
    const long long N = (long long)L.nx * L.ny * L.nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz((int)i, L.nx, L.ny, x, y, z);
        const bool solid = wall_z(z, L.nz);
        const long long off = L.off(x, y, z);
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            float r = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
            if (!solid) {
                #pragma unroll
                for (int k = 0; k < Q; ++k) {
                    float v = Codec<S>::load(f + L.at(a, k, off));
                    if constexpr (Codec<S>::kDeviation) v = zeta(k) * (P.ref[a] + v);
                    r += v;
                    jx += cx(k) * v;
                    jy += cy(k) * v;
                    jz += cz(k) * v;
                }
            }
            A.rho[a][i] = r;
            A.j[a][0][i] = jx;
            A.j[a][1][i] = jy;
            A.j[a][2][i] = jz;
            A.psi[a][i] = solid ? P.eta[a] : -expm1f(-r);
        }
    }
}

// Pass A: per fluid node, mu from lambda(t+1), the local adjoint of BGK,
// equilibrium, shift, u' and force; lambda(t) gets (1 - omega) mu; the wall
// gradient is reduced into part[block][2] (FP64).
__global__ void __launch_bounds__(256)
    adj_local_kernel(AdjArgs G, AdjFields A, const float* __restrict__ lam_next, float* __restrict__ lam_cur,
                     double* __restrict__ part)
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long N = (long long)nx * ny * nz;
    double geta[2] = {0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz((int)i, nx, ny, x, y, z);
        if (wall_z(z, nz)) {
            #pragma unroll
            for (int k = 0; k < 2 * Q; ++k) lam_cur[(long long)k * N + i] = 0.f;
            #pragma unroll
            for (int a = 0; a < 2; ++a) {
                A.rhob[a][i] = 0.f;
                A.psib[a][i] = 0.f;
                #pragma unroll
                for (int d = 0; d < 3; ++d) A.jb[a][d][i] = A.V[a][d][i] = 0.f;
            }
            continue;
        }
        float rho[2], j[2][3], psi[2], S[2][3], F[2][3];
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            rho[a] = A.rho[a][i];
            psi[a] = A.psi[a][i];
            #pragma unroll
            for (int d = 0; d < 3; ++d) j[a][d] = A.j[a][d][i];
        }
        // S^a = sum_m G_m psi~^abar(y + c_m) c_m, wall links flagged
        #pragma unroll
        for (int a = 0; a < 2; ++a) S[a][0] = S[a][1] = S[a][2] = 0.f;
        #pragma unroll
        for (int m = 1; m < Q; ++m) {
            const long long n = didx(wrapi(x + cx(m), nx), wrapi(y + cy(m), ny), z + cz(m), nx, ny);
            #pragma unroll
            for (int a = 0; a < 2; ++a) {
                const float ps = G.G[m] * A.psi[1 - a][n];
                S[a][0] += ps * cx(m);
                S[a][1] += ps * cy(m);
                S[a][2] += ps * cz(m);
            }
        }
        #pragma unroll
        for (int a = 0; a < 2; ++a)
            #pragma unroll
            for (int d = 0; d < 3; ++d) F[a][d] = -G.gk * psi[a] * S[a][d];
        const float D = G.omega[0] * rho[0] + G.omega[1] * rho[1];
        float up[3] = {0.f, 0.f, 0.f};
        if (D > 0.f)
            #pragma unroll
            for (int d = 0; d < 3; ++d) up[d] = (G.omega[0] * j[0][d] + G.omega[1] * j[1][d]) / D;

        float rhob[2] = {0.f, 0.f}, ub[2][3], upb[3] = {0.f, 0.f, 0.f};
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            const bool shift = rho[a] > 1e-12f;
            float u[3];
            #pragma unroll
            for (int d = 0; d < 3; ++d) u[d] = up[d] + (shift ? G.tau[a] * F[a][d] / rho[a] : 0.f);
            const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            ub[a][0] = ub[a][1] = ub[a][2] = 0.f;
            #pragma unroll
            for (int k = 0; k < Q; ++k) {
                // mu_k = lambda_k(y + c_k), or lambda_kbar(y) when y + c_k is a wall
                const int zt = z + cz(k);
                float mu;
                if (wall_z(zt, nz)) mu = lam_next[(long long)(a * Q + opp(k)) * N + i];
                else mu = lam_next[(long long)(a * Q + k) * N + didx(wrapi(x + cx(k), nx), wrapi(y + cy(k), ny), zt, nx, ny)];
                lam_cur[(long long)(a * Q + k) * N + i] = (1.0f - G.omega[a]) * mu;
                const float qb = G.omega[a] * mu;
                const float cu = cx(k) * u[0] + cy(k) * u[1] + cz(k) * u[2];
                const float P = 3.f * cu + 4.5f * cu * cu - 1.5f * usq + 4.5f * cu * cu * cu - 4.5f * usq * cu;
                rhob[a] += qb * zeta(k) * (1.0f + P);
                const float Ak = 3.f + 9.f * cu + 13.5f * cu * cu - 4.5f * usq, Bk = -3.f - 9.f * cu;
                const float w = qb * zeta(k) * rho[a];
                ub[a][0] += w * (cx(k) * Ak + u[0] * Bk);
                ub[a][1] += w * (cy(k) * Ak + u[1] * Bk);
                ub[a][2] += w * (cz(k) * Ak + u[2] * Bk);
            }
            #pragma unroll
            for (int d = 0; d < 3; ++d) upb[d] += ub[a][d];
        }
        float Fb[2][3];
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            const bool shift = rho[a] > 1e-12f;
            float dot = 0.f;
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
                Fb[a][d] = shift ? ub[a][d] * G.tau[a] / rho[a] : 0.f;
                dot += ub[a][d] * F[a][d];
            }
            if (shift) rhob[a] -= dot * G.tau[a] / (rho[a] * rho[a]);
        }
        float jb[2][3];
        if (D > 0.f) {
            const float updot = upb[0] * up[0] + upb[1] * up[1] + upb[2] * up[2];
            #pragma unroll
            for (int a = 0; a < 2; ++a) {
                #pragma unroll
                for (int d = 0; d < 3; ++d) jb[a][d] = G.omega[a] * upb[d] / D;
                rhob[a] -= G.omega[a] * updot / D;
            }
        } else {
            #pragma unroll
            for (int a = 0; a < 2; ++a) jb[a][0] = jb[a][1] = jb[a][2] = 0.f;
        }
        // force: psi^a(y) factor and the neighbour sum
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            float V[3];
            float sdot = 0.f;
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
                V[d] = -G.gk * psi[a] * Fb[a][d];
                sdot += Fb[a][d] * S[a][d];
            }
            A.psib[a][i] = -G.gk * sdot;
            #pragma unroll
            for (int d = 0; d < 3; ++d) {
                A.V[a][d][i] = V[d];
                A.jb[a][d][i] = jb[a][d];
            }
            A.rhob[a][i] = rhob[a];
            // wall links of the neighbour sum feed d J / d eta_abar
            #pragma unroll
            for (int m = 1; m < Q; ++m)
                if (wall_z(z + cz(m), nz)) geta[1 - a] += (double)(G.G[m] * (V[0] * cx(m) + V[1] * cy(m) + V[2] * cz(m)));
        }
    }
    // block reduction of the wall gradient
    __shared__ double sh[8][2];
    #pragma unroll
    for (int a = 0; a < 2; ++a) {
        double v = geta[a];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][a] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        part[blockIdx.x * 2 + threadIdx.x] = v;
    }
}

// Pass B: gather the neighbours' force adjoints into psibar, then finish
// lambda(t) = (1 - omega) mu + rhobar + c . jbar with rhobar including psibar psi'.
__global__ void adj_gather_kernel(AdjArgs G, AdjFields A, float* __restrict__ lam_cur)
{
    const int nx = G.nx, ny = G.ny, nz = G.nz;
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz((int)i, nx, ny, x, y, z);
        if (wall_z(z, nz)) continue;
        #pragma unroll
        for (int a = 0; a < 2; ++a) {
            // psi^a(x) is used by F^abar(x - c_m) for every fluid x - c_m
            float pb = A.psib[a][i];
            #pragma unroll
            for (int m = 1; m < Q; ++m) {
                const int zs = z - cz(m);
                if (wall_z(zs, nz)) continue;
                const long long s = didx(wrapi(x - cx(m), nx), wrapi(y - cy(m), ny), zs, nx, ny);
                pb += G.G[m] * (A.V[1 - a][0][s] * cx(m) + A.V[1 - a][1][s] * cy(m) + A.V[1 - a][2][s] * cz(m));
            }
            const float rb = A.rhob[a][i] + pb * expf(-A.rho[a][i]);
            const float jb[3] = {A.jb[a][0][i], A.jb[a][1][i], A.jb[a][2][i]};
            #pragma unroll
            for (int k = 0; k < Q; ++k)
                lam_cur[(long long)(a * Q + k) * N + i] += rb + cx(k) * jb[0] + cy(k) * jb[1] + cz(k) * jb[2];
        }
    }
}

// Observable J of the densities and its gradient lambda(T) = dJ/drho (FP64 sums).
// obs 0: centre-of-mass height of rho_r above the wall plane, sum (z - 1/2) rho_r / sum rho_r
// obs 1: the same with weight sigma(phi / eps), phi = rho_r - rho_b (the droplet, softly)
// obs 2: wetted area, sum over the first fluid layer of sigma(phi / eps)
__device__ __forceinline__ double sigmoid(double s) { return 1.0 / (1.0 + exp(-s)); }

__global__ void obs_sums_kernel(int nx, int ny, int nz, int obs, double eps, const float* __restrict__ rr,
                                const float* __restrict__ rb, double* __restrict__ part)
{
    const long long N = (long long)nx * ny * nz;
    double s0 = 0, s1 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / ((long long)nx * ny));
        if (wall_z(z, nz)) continue;
        const double h = z - 0.5;
        if (obs == 0) {
            s0 += rr[i];
            s1 += h * rr[i];
        } else {
            const double w = sigmoid(((double)rr[i] - (double)rb[i]) / eps);
            if (obs == 1) {
                s0 += w;
                s1 += h * w;
            } else if (z == 1) {
                s0 += w;
            }
        }
    }
    __shared__ double sh[8][2];
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5][0] = s0;
        sh[threadIdx.x >> 5][1] = s1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[w][threadIdx.x];
        part[blockIdx.x * 2 + threadIdx.x] = v;
    }
}

// sums[0..1] = reduced (s0, s1); J = s1/s0 (obs 0, 1) or s0 (obs 2), written to sums[2]
__global__ void obs_finish_kernel(const double* __restrict__ part, int nblocks, int obs, double* __restrict__ sums)
{
    if (threadIdx.x != 0) return;
    double s0 = 0, s1 = 0;
    for (int b = 0; b < nblocks; ++b) {
        s0 += part[2 * b];
        s1 += part[2 * b + 1];
    }
    sums[0] = s0;
    sums[1] = s1;
    sums[2] = obs == 2 ? s0 : s1 / s0;
}

__global__ void obs_grad_kernel(int nx, int ny, int nz, int obs, double eps, const float* __restrict__ rr,
                                const float* __restrict__ rb, const double* __restrict__ sums, float* __restrict__ lam)
{
    const long long N = (long long)nx * ny * nz;
    const double s0 = sums[0], J = sums[2];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(i / ((long long)nx * ny));
        double gr = 0, gb = 0;
        if (!wall_z(z, nz)) {
            const double h = z - 0.5;
            if (obs == 0) {
                gr = (h - J) / s0;
            } else {
                const double w = sigmoid(((double)rr[i] - (double)rb[i]) / eps);
                const double dw = w * (1.0 - w) / eps;  // d w / d phi
                double gphi = 0;
                if (obs == 1) gphi = (h - J) * dw / s0;
                else if (z == 1) gphi = dw;
                gr = gphi;
                gb = -gphi;
            }
        }
        #pragma unroll
        for (int k = 0; k < Q; ++k) {
            lam[(long long)k * N + i] = (float)gr;
            lam[(long long)(Q + k) * N + i] = (float)gb;
        }
    }
}

// accumulate the per-block wall gradient of one backward step into acc[2] (block order)
__global__ void adj_acc_kernel(const double* __restrict__ part, int nblocks, double* __restrict__ acc)
{
    const int a = threadIdx.x;
    if (a >= 2) return;
    double v = 0;
    for (int b = 0; b < nblocks; ++b) v += part[2 * b + a];
    acc[a] += v;
}

template <class S>
cudaError_t launch_adj_forward(const Layout& L, const KParams& P, const S* f, const AdjFields& A, cudaStream_t st)
{
    adj_forward_kernel<S><<<kAdjBlocks, 256, 0, st>>>(L, P, f, A);
    return cudaGetLastError();
}

cudaError_t launch_adj_backstep(const AdjArgs& G, const AdjFields& A, const float* lam_next, float* lam_cur,
                                double* part, double* acc, cudaStream_t st)
{
    adj_local_kernel<<<kAdjBlocks, 256, 0, st>>>(G, A, lam_next, lam_cur, part);
    adj_gather_kernel<<<kAdjBlocks, 256, 0, st>>>(G, A, lam_cur);
    adj_acc_kernel<<<1, 32, 0, st>>>(part, kAdjBlocks, acc);
    return cudaGetLastError();
}

cudaError_t launch_observable(int nx, int ny, int nz, int obs, double eps, const float* rr, const float* rb,
                              double* part, double* sums, float* lam, cudaStream_t st)
{
    obs_sums_kernel<<<kAdjBlocks, 256, 0, st>>>(nx, ny, nz, obs, eps, rr, rb, part);
    obs_finish_kernel<<<1, 32, 0, st>>>(part, kAdjBlocks, obs, sums);
    if (lam) obs_grad_kernel<<<kAdjBlocks, 256, 0, st>>>(nx, ny, nz, obs, eps, rr, rb, sums, lam);
    return cudaGetLastError();
}

template cudaError_t launch_adj_forward<float>(const Layout&, const KParams&, const float*, const AdjFields&, cudaStream_t);
template cudaError_t launch_adj_forward<__half>(const Layout&, const KParams&, const __half*, const AdjFields&, cudaStream_t);
template cudaError_t launch_adj_forward<__nv_bfloat16>(const Layout&, const KParams&, const __nv_bfloat16*,
                                                       const AdjFields&, cudaStream_t);

}  // namespace lbsc
