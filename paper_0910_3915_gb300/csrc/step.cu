// Fused time step of the two-component Shan-Chen D3Q19 model (Sec. 2):
// moments -> psi = 1 - exp(-rho) -> Shan-Chen and wall force (Eq. SCforce)
// -> force-shifted cubic equilibrium (Eq. Equil) -> BGK -> push streaming with
// mid-grid bounce-back (Eq. LBeqs), in one kernel.
//
// Design: populations are double-buffered (read src, write dst), structure of
// arrays, one 32-node row segment per warp. A CTA owns a tile of 32 x TY
// columns and a range of z planes and marches upward in z. At each plane it
// loads the next plane's populations, reduces them to rho, j and psi, and
// keeps psi for three planes (tile plus a one-node ring) in shared memory; the
// ring nodes' psi comes from their populations in src, which no CTA writes
// during the step. psi therefore never travels through HBM and HBM traffic
// is one read and one write of every population per step.
#include "lb_fields.cuh"

namespace lbsc {

// rho and j of one component from its 19 stored values v_k: FP32 stores n_k;
// 16-bit formats store e_k with n_k = zeta_k (rho_ref + e_k). The same routine
// serves a tile's own nodes and its ring, so both see bit-identical rho.
template <class S>
__device__ __forceinline__ float rho_of(const float (&v)[Q], float ref)
{
    if constexpr (Codec<S>::kDeviation) {
        float ax = 0.f, di = 0.f;
#pragma unroll
        for (int k = 1; k <= 6; ++k) ax += v[k];
#pragma unroll
        for (int k = 7; k < Q; ++k) di += v[k];
        return ref + (v[0] * (1.0f / 3.0f) + (ax * (1.0f / 18.0f) + di * (1.0f / 36.0f)));
    } else {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < Q; ++k) s += v[k];
        return s;
    }
}

template <class S>
__device__ __forceinline__ void mom_of(const float (&v)[Q], float (&j)[3])
{
    float ax[3] = {0.f, 0.f, 0.f}, di[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        float* acc = is_axis(k) ? ax : di;
        if (cx(k)) acc[0] += cx(k) * v[k];
        if (cy(k)) acc[1] += cy(k) * v[k];
        if (cz(k)) acc[2] += cz(k) * v[k];
    }
    if constexpr (Codec<S>::kDeviation) {
#pragma unroll
        for (int d = 0; d < 3; ++d) j[d] = ax[d] * (1.0f / 18.0f) + di[d] * (1.0f / 36.0f);
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) j[d] = ax[d] + di[d];
    }
}

// psi = 1 - exp(-rho), evaluated as -expm1(-rho) to keep precision at small rho
__device__ __forceinline__ float psi_of(float rho) { return -expm1f(-rho); }

template <class S>
__device__ __forceinline__ void load_comp(const S* __restrict__ p, long long slot, float (&v)[Q])
{
#pragma unroll
    for (int k = 0; k < Q; ++k) v[k] = Codec<S>::load(p + k * slot);
}

template <class S, int TY, bool kGeneral, bool kTauOne>
__global__ void __launch_bounds__(32 * TY) step_kernel(const StepArgs<S> A)
{
    constexpr int TX = 32, NT = TX * TY, HX = TX + 2, HY = TY + 2;
    constexpr int RING = 2 * HX + 2 * TY;           // ring nodes around the tile
    constexpr int NIT = (2 * RING + NT - 1) / NT;   // ring items (node, component) per thread
    __shared__ float sp[4][2][HY][HX];              // psi of 4 planes, slot = z & 3

    const int nx = A.L.nx, ny = A.L.ny, nz = A.L.nz, px = A.L.px;
    const long long plane = A.L.plane, slot = A.L.slot;
    const S* __restrict__ src = A.src;
    S* __restrict__ dst = A.dst;
    const uint32_t* __restrict__ nbmask = A.nbmask;
    const float eta[2] = {A.P.eta[0], A.P.eta[1]};
    const float ref[2] = {A.P.ref[0], A.P.ref[1]};
    const float tau[2] = {A.P.tau[0], A.P.tau[1]};
    const float itau[2] = {A.P.itau[0], A.P.itau[1]};
    const float gk = A.P.gk, Gax = A.P.Gax, Gdi = A.P.Gdi;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int ncol = A.tiles_x * A.tiles_y;
    const int nzf = A.zhi - A.zlo;

    for (int item = blockIdx.x; item < ncol * A.nseg; item += gridDim.x) {
        const int col = item % ncol, seg = item / ncol;
        const int za = A.zlo + (int)((long long)seg * nzf / A.nseg);
        const int zb = A.zlo + (int)((long long)(seg + 1) * nzf / A.nseg);
        if (za >= zb) continue;
        const int x0 = (col % A.tiles_x) * TX, y0 = (col / A.tiles_x) * TY;
        const int gx = x0 + tx, gy = y0 + ty;
        const bool valid = gx < nx && gy < ny;
        const int ox = gx % nx, oy = gy % ny;  // ragged tiles: wrapped copy of a real column
        const long long own = (long long)oy * px + ox;

        // this thread's ring items: smem position, plane offset of the node, component
        int it_sm[NIT], it_a[NIT];
        long long it_off[NIT];
#pragma unroll
        for (int i = 0; i < NIT; ++i) {
            const int it = tid + i * NT;
            it_a[i] = -1;
            if (it < 2 * RING) {
                const int a = it >= RING, r = it - a * RING;
                int ix, iy;
                if (r < HX) { ix = r; iy = 0; }
                else if (r < 2 * HX) { ix = r - HX; iy = HY - 1; }
                else if (r < 2 * HX + TY) { ix = 0; iy = r - 2 * HX + 1; }
                else { ix = HX - 1; iy = r - 2 * HX - TY + 1; }
                const int hx = ((x0 - 1 + ix) % nx + nx) % nx, hy = ((y0 - 1 + iy) % ny + ny) % ny;
                it_a[i] = a;
                it_sm[i] = iy * HX + ix;
                it_off[i] = (long long)hy * px + hx;
            }
        }

        // Fill psi of plane zp (tile + ring) into its slot; return own moments.
        // Own populations stay in v when the collision needs them (tau != 1).
        auto fill = [&](int zp, float (&rho)[2], float (&j)[2][3], float (&v)[2][Q]) {
            const int zw = kGeneral ? wrapi(zp, nz) : zp;
            const long long zoff = (long long)zw * plane;
            float* spl = &sp[zp & 3][0][0][0];
            bool solid;
            if constexpr (kGeneral) solid = (__ldg(nbmask + zoff + own) & kSelfSolid) != 0;
            else solid = (zp == 0 || zp == nz - 1);
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                float ps = eta[a];
                rho[a] = 0.f;
                j[a][0] = j[a][1] = j[a][2] = 0.f;
                if (!solid) {
                    float w[Q];
                    load_comp<S>(src + (long long)a * Q * slot + zoff + own, slot, w);
                    rho[a] = rho_of<S>(w, ref[a]);
                    mom_of<S>(w, j[a]);
                    ps = psi_of(rho[a]);
                    if constexpr (!kTauOne) {
#pragma unroll
                        for (int k = 0; k < Q; ++k) v[a][k] = w[k];
                    }
                }
                spl[(a * HY + ty + 1) * HX + tx + 1] = ps;
            }
#pragma unroll
            for (int i = 0; i < NIT; ++i) {
                if (it_a[i] < 0) continue;
                const int a = it_a[i];
                bool hsolid;
                if constexpr (kGeneral) hsolid = (__ldg(nbmask + zoff + it_off[i]) & kSelfSolid) != 0;
                else hsolid = solid;
                float ps = eta[a];
                if (!hsolid) {
                    float w[Q];
                    load_comp<S>(src + (long long)a * Q * slot + zoff + it_off[i], slot, w);
                    ps = psi_of(rho_of<S>(w, ref[a]));
                }
                spl[a * HY * HX + it_sm[i]] = ps;
            }
        };

        float rc[2], jc[2][3], vc[2][Q];
        float rn[2], jn[2][3], vn[2][Q];
        __syncthreads();  // the previous item's readers are done with the ring
        fill(za - 1, rn, jn, vn);
        fill(za, rc, jc, vc);

        const int xm = wrapi(gx - 1, nx), xp = wrapi(gx + 1, nx);
        const long long ym = (long long)wrapi(gy - 1, ny) * px, yc = (long long)gy * px,
                        yp = (long long)wrapi(gy + 1, ny) * px;

        for (int z = za; z < zb; ++z) {
            fill(z + 1, rn, jn, vn);
            __syncthreads();

            bool self_solid = false;
            uint32_t nb = 0;
            if constexpr (kGeneral) {
                if (valid) {
                    nb = __ldg(nbmask + (long long)z * plane + own);
                    self_solid = (nb & kSelfSolid) != 0;
                }
            }
            if (valid && !self_solid) {
                const float* s0 = &sp[(z - 1) & 3][0][0][0];
                const float* s1 = &sp[z & 3][0][0][0];
                const float* s2 = &sp[(z + 1) & 3][0][0][0];
                // Eq. SCforce: S^a = sum_k G_k psi^abar(x + c_k) c_k, F^a = -g kappa psi^a(x) S^a
                float F[2][3];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int ab = 1 - a;
                    float ax[3] = {0.f, 0.f, 0.f}, di[3] = {0.f, 0.f, 0.f};
#pragma unroll
                    for (int k = 1; k < Q; ++k) {
                        const float* sl = cz(k) < 0 ? s0 : (cz(k) > 0 ? s2 : s1);
                        const float ps = sl[(ab * HY + ty + 1 + cy(k)) * HX + tx + 1 + cx(k)];
                        float* acc = is_axis(k) ? ax : di;
                        if (cx(k)) acc[0] += cx(k) * ps;
                        if (cy(k)) acc[1] += cy(k) * ps;
                        if (cz(k)) acc[2] += cz(k) * ps;
                    }
                    const float pre = -gk * s1[(a * HY + ty + 1) * HX + tx + 1];
#pragma unroll
                    for (int d = 0; d < 3; ++d) F[a][d] = pre * (Gax * ax[d] + Gdi * di[d]);
                }
                // common velocity u' = sum_a j^a/tau^a / sum_a rho^a/tau^a
                const float den = rc[0] * itau[0] + rc[1] * itau[1];
                const float iden = den > 0.f ? 1.0f / den : 0.f;
                float up[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) up[d] = (jc[0][d] * itau[0] + jc[1][d] * itau[1]) * iden;

                long long zo[3];
                if constexpr (kGeneral) {
                    zo[0] = (long long)wrapi(z - 1, nz) * plane;
                    zo[1] = (long long)z * plane;
                    zo[2] = (long long)wrapi(z + 1, nz) * plane;
                } else {
                    zo[0] = (long long)(z - 1) * plane;
                    zo[1] = (long long)z * plane;
                    zo[2] = (long long)(z + 1) * plane;
                }
                const long long yo[3] = {ym, yc, yp};
                const int xo[3] = {xm, gx, xp};
                const long long self = zo[1] + yc + gx;
                const bool bot = !kGeneral && z - 1 == 0, top = !kGeneral && z + 1 == nz - 1;

#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const float r = rc[a];
                    float u[3];
                    const float sh = r > 1e-12f ? tau[a] / r : 0.f;  // shift tau F / rho
#pragma unroll
                    for (int d = 0; d < 3; ++d) u[d] = up[d] + sh * F[a][d];
                    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                    // Eq. Equil with c_s^2 = 1/3:
                    // n^eq_k = zeta_k rho [1 + 3 cu + 4.5 cu^2 - 1.5 u^2 + 4.5 cu^3 - 4.5 u^2 cu]
                    const float A0 = 3.0f - 4.5f * usq, B0 = -1.5f * usq;
                    const float dref = r - ref[a];
                    S* dbase = dst + (long long)a * Q * slot;
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const float cu = (cx(k) ? cx(k) * u[0] : 0.f) + (cy(k) ? cy(k) * u[1] : 0.f) +
                                         (cz(k) ? cz(k) * u[2] : 0.f);
                        const float P = cu * (A0 + 4.5f * cu * (1.0f + cu)) + B0;
                        float q;  // equilibrium in storage form
                        if constexpr (Codec<S>::kDeviation) q = dref + r * P;
                        else q = zeta(k) * r * (1.0f + P);
                        float s;
                        if constexpr (kTauOne) s = q;
                        else s = vc[a][k] + (q - vc[a][k]) * itau[a];
                        bool wall;
                        if constexpr (kGeneral) wall = (nb >> k) & 1u;
                        else wall = (cz(k) < 0 && bot) || (cz(k) > 0 && top);
                        const long long dst_off = wall ? (long long)opp(k) * slot + self
                                                       : (long long)k * slot + zo[cz(k) + 1] + yo[cy(k) + 1] +
                                                             xo[cx(k) + 1];
                        Codec<S>::store(dbase + dst_off, s);
                    }
                }
            }
            // rotate: next plane becomes current
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                rc[a] = rn[a];
#pragma unroll
                for (int d = 0; d < 3; ++d) jc[a][d] = jn[a][d];
                if constexpr (!kTauOne) {
#pragma unroll
                    for (int k = 0; k < Q; ++k) vc[a][k] = vn[a][k];
                }
            }
        }
    }
}

template <class S, int TY, bool G, bool T1>
static cudaError_t launch_one(const StepArgs<S>& A, cudaStream_t st)
{
    const int items = A.tiles_x * A.tiles_y * A.nseg;
    step_kernel<S, TY, G, T1><<<items, 32 * TY, 0, st>>>(A);
    return cudaGetLastError();
}

template <class S, int TY>
static cudaError_t launch_ty(const StepArgs<S>& A, bool general, bool tau_one, cudaStream_t st)
{
    if (general) return tau_one ? launch_one<S, TY, true, true>(A, st) : launch_one<S, TY, true, false>(A, st);
    return tau_one ? launch_one<S, TY, false, true>(A, st) : launch_one<S, TY, false, false>(A, st);
}

template <class S>
cudaError_t launch_step(const StepArgs<S>& A, int tile_y, bool general, bool tau_one, cudaStream_t st)
{
    switch (tile_y) {
    case 4: return launch_ty<S, 4>(A, general, tau_one, st);
    case 8: return launch_ty<S, 8>(A, general, tau_one, st);
    case 16: return launch_ty<S, 16>(A, general, tau_one, st);
    default: return cudaErrorInvalidValue;
    }
}

template <class S, int TY>
static int occ_ty(bool general, bool tau_one)
{
    int n = 0;
    cudaError_t e;
    if (general)
        e = tau_one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<S, TY, true, true>, 32 * TY, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<S, TY, true, false>, 32 * TY, 0);
    else
        e = tau_one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<S, TY, false, true>, 32 * TY, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_kernel<S, TY, false, false>, 32 * TY, 0);
    return e == cudaSuccess ? n : 1;
}

template <class S>
static int occ_s(int tile_y, bool general, bool tau_one)
{
    switch (tile_y) {
    case 4: return occ_ty<S, 4>(general, tau_one);
    case 8: return occ_ty<S, 8>(general, tau_one);
    default: return occ_ty<S, 16>(general, tau_one);
    }
}

// resident CTAs per SM of the step kernel for this configuration
int step_occupancy(int precision, int tile_y, bool general, bool tau_one)
{
    switch (precision) {
    case 0: return occ_s<float>(tile_y, general, tau_one);
    case 1: return occ_s<__half>(tile_y, general, tau_one);
    default: return occ_s<__nv_bfloat16>(tile_y, general, tau_one);
    }
}

template cudaError_t launch_step<float>(const StepArgs<float>&, int, bool, bool, cudaStream_t);
template cudaError_t launch_step<__half>(const StepArgs<__half>&, int, bool, bool, cudaStream_t);
template cudaError_t launch_step<__nv_bfloat16>(const StepArgs<__nv_bfloat16>&, int, bool, bool, cudaStream_t);

}  // namespace lbsc
