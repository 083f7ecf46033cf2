// Per-node arithmetic of the time step, shared by the step kernels:
// moments (Sec. 2), psi = 1 - exp(-rho), the Shan-Chen and wall force
// (Eq. SCforce), the force-shifted cubic equilibrium (Eq. Equil), BGK, and
// the push of the post-collision populations with mid-grid bounce-back
// (Eq. LBeqs).
#pragma once

#include "lb_internal.cuh"

namespace lbsc {

// rho of one component from its 19 stored values v_k: FP32 stores n_k;
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

// j = sum_k n_k c_k
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

// Eq. SCforce on the psi ring: s0, s1, s2 are the planes z-1, z, z+1 of a
// [2][HY][HX] psi array, the node at row ty+1, column tx+1.
// S^a = sum_k G_k psi^abar(x + c_k) c_k ;  F^a = -g kappa psi^a(x) S^a
template <int HX, int HY>
__device__ __forceinline__ void sc_force(const float* s0, const float* s1, const float* s2, int ty, int tx, float gk,
                                         float Gax, float Gdi, float (&F)[2][3])
{
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
}

// Where the node's populations go: neighbours (wrapped), the planes of z-1,
// z, z+1, and which links end on a wall.
// Ghost images are not written here: the TMA path refreshes them in a
// separate pass (ghost_kernel) after each step. Addresses are a warp-uniform
// slot base plus a 32-bit per-thread offset.
struct Dest {
    int xo[3], yo[3];  // x-1, x, x+1 and y-1, y, y+1, wrapped
    int ro[3];         // row offsets of y-1, y, y+1 (incl. the left padding)
    int zo[3];         // plane offsets of z-1, z, z+1 (offsets stay below 2^31: slot < 2^31)
    bool bot, top;     // planar walls: solid plane below / above
    uint32_t nb;       // general geometry: bit k = link k ends on a solid node

    // per-thread part that stays fixed while the thread marches in z
    __device__ __forceinline__ void set_column(const Layout& L, int x, int y)
    {
        xo[0] = wrapi(x - 1, L.nx);
        xo[1] = x;
        xo[2] = wrapi(x + 1, L.nx);
        yo[0] = wrapi(y - 1, L.ny);
        yo[1] = y;
        yo[2] = wrapi(y + 1, L.ny);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) ro[dy] = (yo[dy] + 1) * L.px + L.gx;
        nb = 0;
    }
    template <class S>
    __device__ __forceinline__ void store(S* __restrict__ p, const Layout&, int dx, int dy, int dz, float v) const
    {
        Codec<S>::store(p + zo[dz + 1] + ro[dy + 1] + xo[dx + 1], v);
    }
};

// BGK with the force-shifted cubic equilibrium and the push with mid-grid
// bounce-back, for both components of one node. rc, jc: moments; vc: the
// stored values (used when tau != 1); F: Shan-Chen force.
// The 18 moving populations follow Eq. Equil; the rest population takes the
// remainder of the node's mass, which Eq. Equil and BGK leave unchanged, so
// that rounded lattice weights (1/3 + 6/18 + 12/36 != 1 in FP32) and 16-bit
// rounding of the stored values do not bias the mass.
template <class S, bool kGeneral, bool kTauOne>
__device__ __forceinline__ void collide_store(const float (&rc)[2], const float (&jc)[2][3], const float (&vc)[2][Q],
                                              const float (&F)[2][3], const float (&tau)[2], const float (&itau)[2],
                                              const float (&ref)[2], S* __restrict__ dst, const Layout& L, int x, int y,
                                              const Dest& D)
{
    // common velocity u' = sum_a j^a/tau^a / sum_a rho^a/tau^a
    const float den = rc[0] * itau[0] + rc[1] * itau[1];
    const float iden = den > 0.f ? 1.0f / den : 0.f;
    float up[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) up[d] = (jc[0][d] * itau[0] + jc[1][d] * itau[1]) * iden;

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
        S* dbase = dst + (long long)a * Q * L.slot;
        float sum = 0.f, sax = 0.f, sdi = 0.f;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const float cu = (cx(k) ? cx(k) * u[0] : 0.f) + (cy(k) ? cy(k) * u[1] : 0.f) + (cz(k) ? cz(k) * u[2] : 0.f);
            const float P = cu * (A0 + 4.5f * cu * (1.0f + cu)) + B0;
            float q;  // equilibrium in storage form
            if constexpr (Codec<S>::kDeviation) q = dref + r * P;
            else q = zeta(k) * r * (1.0f + P);
            float s;
            if constexpr (kTauOne) s = q;
            else s = vc[a][k] + (q - vc[a][k]) * itau[a];
            if constexpr (Codec<S>::kDeviation) {
                const float sr = Codec<S>::round(s);
                if (is_axis(k)) sax += sr;
                else sdi += sr;
            } else {
                sum += s;
            }
            bool wall;
            if constexpr (kGeneral) wall = (D.nb >> k) & 1u;
            else wall = (cz(k) < 0 && D.bot) || (cz(k) > 0 && D.top);
            if (wall) D.store<S>(dbase + (long long)opp(k) * L.slot, L, 0, 0, 0, s);
            else D.store<S>(dbase + (long long)k * L.slot, L, cx(k), cy(k), cz(k), s);
        }
        float s0;
        if constexpr (Codec<S>::kDeviation) s0 = 3.0f * (dref - (sax * (1.0f / 18.0f) + sdi * (1.0f / 36.0f)));
        else s0 = r - sum;
        D.store<S>(dbase, L, 0, 0, 0, s0);
    }
}

}  // namespace lbsc
