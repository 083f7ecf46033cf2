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
//
// For 16-bit storage, m36 = 36 (rho - rho_ref) = 12 e_0 + 2 sum_axis e_k + sum_diag e_k
// is also returned: the values are 16-bit numbers, so these FP32 sums are exact
// (their bits span far less than 24), and the collision balances the node's
// mass in this exact form rather than through the rounded rho.
template <class S>
__device__ __forceinline__ float rho_of(const float (&v)[Q], float ref, float* m36 = nullptr)
{
    // opposite velocities come in pairs (k, k+1), k odd: sum each pair first
    if constexpr (Codec<S>::kDeviation) {
        const float ax = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
        const float di = (((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14]))) +
                         ((v[15] + v[16]) + (v[17] + v[18]));
        const float m = fmaf(12.0f, v[0], fmaf(2.0f, ax, di));
        if (m36) *m36 = m;
        return ref + m * (1.0f / 36.0f);
    } else {
        const float ax = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
        const float di = (((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14]))) +
                         ((v[15] + v[16]) + (v[17] + v[18]));
        return (v[0] + ax) + di;
    }
}

// j = sum_k n_k c_k, from the differences of opposite pairs: d = n_k - n_kbar
// (k odd), j = sum over pairs of c_k d
template <class S>
__device__ __forceinline__ void mom_of(const float (&v)[Q], float (&j)[3])
{
    float d[Q / 2 + 1];
#pragma unroll
    for (int k = 1; k < Q; k += 2) d[(k + 1) / 2] = v[k] - v[k + 1];
    float ax[3] = {0.f, 0.f, 0.f}, di[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float dk = d[(k + 1) / 2];
        float* acc = is_axis(k) ? ax : di;
        if (cx(k)) acc[0] = cx(k) > 0 ? acc[0] + dk : acc[0] - dk;
        if (cy(k)) acc[1] = cy(k) > 0 ? acc[1] + dk : acc[1] - dk;
        if (cz(k)) acc[2] = cz(k) > 0 ? acc[2] + dk : acc[2] - dk;
    }
    if constexpr (Codec<S>::kDeviation) {
#pragma unroll
        for (int q = 0; q < 3; ++q) j[q] = ax[q] * (1.0f / 18.0f) + di[q] * (1.0f / 36.0f);
    } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) j[q] = ax[q] + di[q];
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
        auto psi_at = [&](int k) {
            const float* sl = cz(k) < 0 ? s0 : (cz(k) > 0 ? s2 : s1);
            return sl[(ab * HY + ty + 1 + cy(k)) * HX + tx + 1 + cx(k)];
        };
        // opposite neighbours in pairs: psi(x + c_k) - psi(x - c_k), k odd
        float ax[3] = {0.f, 0.f, 0.f}, di[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 1; k < Q; k += 2) {
            const float dk = psi_at(k) - psi_at(k + 1);
            float* acc = is_axis(k) ? ax : di;
            if (cx(k)) acc[0] = cx(k) > 0 ? acc[0] + dk : acc[0] - dk;
            if (cy(k)) acc[1] = cy(k) > 0 ? acc[1] + dk : acc[1] - dk;
            if (cz(k)) acc[2] = cz(k) > 0 ? acc[2] + dk : acc[2] - dk;
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
    int* err;          // status word (bounds-checked build only)

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
// Loop order: velocity k outer, component inner, so each destination address
// is formed once and both components' slots are reached by a uniform offset.
// For 16-bit storage the rest value, which balances the node's mass (taken
// exactly from m36 and the stored moving values), is rounded stochastically:
// round-to-nearest of nearly equal bulk values would bias the mass of every
// bulk node the same way, step after step. BF16 (8 significant bits) rounds
// the moving values stochastically too. The random bits come from a hash of
// the node and the lattice's step counter `clk`: fresh every step, and the
// same again when a checkpoint is replayed.
template <class S, bool kGeneral, bool kTauOne>
__device__ __forceinline__ void collide_store(const float (&rc)[2], const float (&jc)[2][3], const float (&vc)[2][Q],
                                              const float (&F)[2][3], const float (&tau)[2], const float (&itau)[2],
                                              const float (&ref)[2], S* __restrict__ dst, const Layout& L, int x, int y,
                                              const Dest& D, const float (&m36)[2], uint32_t clk = 0)
{
    // common velocity u' = sum_a j^a/tau^a / sum_a rho^a/tau^a
    const float den = rc[0] * itau[0] + rc[1] * itau[1];
    const float iden = den > 0.f ? __frcp_rn(den) : 0.f;
    float up[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) up[d] = (jc[0][d] * itau[0] + jc[1][d] * itau[1]) * iden;

    // per component: equilibrium velocity u' + tau F / rho and the polynomial
    // coefficients of Eq. Equil with c_s^2 = 1/3:
    // n^eq_k = zeta_k rho [1 + P_k],  P = cu (3 - 4.5 u^2 + 4.5 cu (1 + cu)) - 1.5 u^2
    float u[2][3], A0[2], B0[2], w1[2], w2[2], base[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const float r = rc[a];
        const float sh = r > 1e-12f ? tau[a] * __frcp_rn(r) : 0.f;  // shift tau F / rho
#pragma unroll
        for (int d = 0; d < 3; ++d) u[a][d] = fmaf(sh, F[a][d], up[d]);
        const float usq = u[a][0] * u[a][0] + u[a][1] * u[a][1] + u[a][2] * u[a][2];
        A0[a] = fmaf(-4.5f, usq, 3.0f);
        B0[a] = -1.5f * usq;
        if constexpr (Codec<S>::kDeviation) {
            w1[a] = w2[a] = r;          // e* = (rho - rho_ref) + rho P
            base[a] = r - ref[a];
        } else {
            w1[a] = r * (1.0f / 18.0f);  // n* = zeta rho + zeta rho P
            w2[a] = r * (1.0f / 36.0f);
            base[a] = 0.f;
        }
    }
    const long long slot = L.slot;
    const int self = D.zo[1] + D.ro[1] + D.xo[1];
    float sum[2] = {0.f, 0.f}, sax[2] = {0.f, 0.f}, sdi[2] = {0.f, 0.f};
    uint32_t hsh = 0;
    if constexpr (Codec<S>::kDitherMoving) hsh = node_hash((uint32_t)self, clk);
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        bool wall;
        if constexpr (kGeneral) wall = (D.nb >> k) & 1u;
        else wall = (cz(k) < 0 && D.bot) || (cz(k) > 0 && D.top);
        // destination: the neighbour x + c_k, or slot kbar of this node (bounce-back)
        const int qo = wall ? self : D.zo[cz(k) + 1] + D.ro[cy(k) + 1] + D.xo[cx(k) + 1];
        if constexpr (kCheckBounds)
            if (!in_bounds(qo, slot, D.err)) continue;
        S* q = dst + qo;
        const long long so = (long long)(wall ? opp(k) : k) * slot;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const float cu = (cx(k) ? cx(k) * u[a][0] : 0.f) + (cy(k) ? cy(k) * u[a][1] : 0.f) +
                             (cz(k) ? cz(k) * u[a][2] : 0.f);
            const float P = fmaf(cu, fmaf(cu, fmaf(4.5f, cu, 4.5f), A0[a]), B0[a]);
            const float w = is_axis(k) ? w1[a] : w2[a];
            const float qk = fmaf(w, P, Codec<S>::kDeviation ? base[a] : w);  // equilibrium, storage form
            float s;
            if constexpr (kTauOne) s = qk;
            else s = fmaf(qk - vc[a][k], itau[a], vc[a][k]);
            if constexpr (Codec<S>::kDeviation) {
                S h;
                if constexpr (Codec<S>::kDitherMoving) h = Codec<S>::sr(s, rand16(hsh, a * Q + k));
                else h = Codec<S>::rn(s);
                if (is_axis(k)) sax[a] += Codec<S>::val(h);
                else sdi[a] += Codec<S>::val(h);
                q[so + (long long)a * Q * slot] = h;
            } else {
                sum[a] += s;
                Codec<S>::store(q + so + (long long)a * Q * slot, s);
            }
        }
    }
    if constexpr (kCheckBounds)
        if (!in_bounds(self, slot, D.err)) return;
    S* q0 = dst + self;
    uint32_t hrest = 0;
    if constexpr (Codec<S>::kDitherMoving) hrest = node_hash(hsh, 0x632BE5ABu);  // a second full mixing round
    else if constexpr (Codec<S>::kDeviation) hrest = node_hash((uint32_t)self, clk);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if constexpr (Codec<S>::kDeviation) {
            // 12 e_0* = m36 - 2 sum_axis e_k* - sum_diag e_k*, the right side exact in FP32
            // the residual step makes the quotient round as x/12 itself would;
            // the rounded reciprocal alone scales every rest value by 1 + 3e-8
            const float x0 = m36[a] - fmaf(2.0f, sax[a], sdi[a]);
            float s0 = x0 * (1.0f / 12.0f);
            s0 = fmaf(fmaf(-12.0f, s0, x0), 1.0f / 12.0f, s0);
            q0[(long long)a * Q * slot] = Codec<S>::sr(s0, rand16(hrest, a));
        } else {
            Codec<S>::store(q0 + (long long)a * Q * slot, rc[a] - sum[a]);
        }
    }
}

}  // namespace lbsc
