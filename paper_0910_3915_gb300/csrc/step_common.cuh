// Per-node arithmetic of the time step, shared by the step kernels:
// moments (Sec. 2), psi = 1 - exp(-rho), the Shan-Chen and wall force
// (Eq. SCforce), the force-shifted cubic equilibrium (Eq. Equil), BGK, and
// the push of the post-collision populations with mid-grid bounce-back
// (Eq. LBeqs).
#pragma once

#include "lb_internal.cuh"

namespace lbsc {

// The two components go through the same arithmetic, so a node's moments,
// force and collision run on (red, blue) pairs in the packed FP32
// instructions (FADD2/FMUL2/FFMA2): each lane rounds exactly as the scalar
// operation would, so pairing halves the instruction count without changing
// a value. Subtraction is a fused multiply-add with -1 (exact product, one
// rounding).
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 sp2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, sp2(-1.0f), a); }
__device__ __forceinline__ float2 neg2(float2 a) { return __fmul2_rn(a, sp2(-1.0f)); }

// Accumulate signed terms into a sum that starts with its first term
// (whose sign is positive for every sum formed here).
__device__ __forceinline__ void acc_signed(float2& acc, bool& has, float2 t, int sign)
{
    if (!has) acc = sign > 0 ? t : neg2(t);
    else acc = sign > 0 ? add2(acc, t) : sub2(acc, t);
    has = true;
}

// rho of one component from its 19 stored values v_k: FP32 stores n_k;
// 16-bit formats store e_k with n_k = zeta_k (rho_ref + e_k). This routine
// (one component of a ring node, load-from-global kernel) and rho2_of (both
// components in packed lanes: a ring node of the TMA kernel, and every
// tile's own nodes through moments2) perform the same operations in the same
// order, so every kernel sees bit-identical rho for a node.
//
// For 16-bit storage, m36 = 36 (rho - rho_ref) = 12 e_0 + 2 sum_axis e_k + sum_diag e_k
// is also returned: the values are 16-bit numbers, so these FP32 sums are exact
// (their bits span far less than 24), and the collision balances the node's
// mass in this exact form rather than through the rounded rho.
template <class S>
__device__ __forceinline__ float rho_of(const float (&v)[Q], float ref, float* m36 = nullptr)
{
    // opposite velocities come in pairs (k, k+1), k odd: sum each pair first
    const float ax = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
    const float di = (((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14]))) +
                     ((v[15] + v[16]) + (v[17] + v[18]));
    if constexpr (Codec<S>::kDeviation) {
        const float m = fmaf(12.0f, v[0], fmaf(2.0f, ax, di));
        if (m36) *m36 = m;
        return fmaf(m, 1.0f / 36.0f, ref);
    } else {
        return (v[0] + ax) + di;
    }
}

// Both components' rho of one node from its 19 pairs of stored values, in
// the packed lanes: the operations of rho_of in the same order, so each lane
// is the bits rho_of gives for that component. m36 as in rho_of.
template <class S>
__device__ __forceinline__ float2 rho2_of(const float2 (&p)[Q], float2 ref, float2& m36)
{
    const float2 ax = add2(add2(add2(p[1], p[2]), add2(p[3], p[4])), add2(p[5], p[6]));
    const float2 di = add2(add2(add2(add2(p[7], p[8]), add2(p[9], p[10])), add2(add2(p[11], p[12]), add2(p[13], p[14]))),
                           add2(add2(p[15], p[16]), add2(p[17], p[18])));
    if constexpr (Codec<S>::kDeviation) {
        m36 = fma2(sp2(12.0f), p[0], fma2(sp2(2.0f), ax, di));
        return fma2(m36, sp2(1.0f / 36.0f), ref);
    } else {
        return add2(add2(p[0], ax), di);
    }
}

// Both components' rho (as rho_of), m36 (16-bit storage) and
// j = sum_k n_k c_k, the latter from the differences of opposite pairs:
// d = n_k - n_kbar (k odd), j = sum over pairs of c_k d.
template <class S>
__device__ __forceinline__ void moments2(const float (&v)[2][Q], const float (&ref)[2], float (&rho)[2],
                                         float (&j)[2][3], float (&m36)[2])
{
    float2 p[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) p[k] = f2(v[0][k], v[1][k]);
    float2 m = sp2(0.f);
    const float2 r = rho2_of<S>(p, f2(ref[0], ref[1]), m);
    rho[0] = r.x;
    rho[1] = r.y;
    m36[0] = m.x;
    m36[1] = m.y;

    float2 jax[3], jdi[3];
    bool hax[3] = {false, false, false}, hdi[3] = {false, false, false};
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float2 dk = sub2(p[k], p[k + 1]);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int c = q == 0 ? cx(k) : (q == 1 ? cy(k) : cz(k));
            if (!c) continue;
            if (is_axis(k)) acc_signed(jax[q], hax[q], dk, c);
            else acc_signed(jdi[q], hdi[q], dk, c);
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float2 jq;
        if constexpr (Codec<S>::kDeviation) jq = fma2(jax[q], sp2(1.0f / 18.0f), mul2(jdi[q], sp2(1.0f / 36.0f)));
        else jq = add2(jax[q], jdi[q]);
        j[0][q] = jq.x;
        j[1][q] = jq.y;
    }
}

// psi = 1 - exp(-rho) (Sec. 2), evaluated without cancellation at small rho
// and without a library call. Cody and Waite's reduction: rho = k ln2 + r,
// k = rint(rho / ln2), |r| <= ln2/2, with ln2 split as kLn2Hi (16 significant
// bits, so k kLn2Hi is exact for |k| < 2^8) plus kLn2Lo; then
//   1 - exp(-rho) = (1 - 2^-k) + 2^-k (r + r q(r)),
// where r + r q(r) = 1 - exp(-r), i.e. q is the Taylor series of
// (1 - e^-r)/r - 1 = sum_n (-r)^n / (n+1)!, n = 1..6, whose remainder is
// below 2^-26 relative for |r| <= ln2/2. The leading r is added in the last
// fused multiply-add, 1 - 2^-k and the scaling by 2^-k are exact, so the
// result stays within about 1 ulp of -expm1(-rho) (the GPU self-test checks
// it against the exact value and against expm1f). rho is
// clamped to [-80, 80] (psi is -5.5e34 .. 1 there); NaN passes through.
// psi_of and psi2_of (both components in packed lanes) perform the same
// operations, so a node's psi is the same bits whether it is computed as a
// tile's own node or as a ring node of the neighbouring tile.
constexpr float kInvLn2 = 1.44269502162933350f;
constexpr float kLn2Hi = 0.693145751953125f;
constexpr float kLn2Lo = 1.42860676533018700e-06f;
constexpr float kPsiC1 = -0.5f, kPsiC2 = 1.0f / 6.0f, kPsiC3 = -1.0f / 24.0f, kPsiC4 = 1.0f / 120.0f,
                kPsiC5 = -1.0f / 720.0f, kPsiC6 = 1.0f / 5040.0f;

__device__ __forceinline__ float psi_clamp(float rho) { return rho > 80.0f ? 80.0f : (rho < -80.0f ? -80.0f : rho); }
__device__ __forceinline__ float pow2_neg(float kf) { return __int_as_float((127 - (int)kf) << 23); }  // 2^-k

__device__ __forceinline__ float psi_of(float rho)
{
    const float x = psi_clamp(rho);
    const float kf = rintf(x * kInvLn2);
    const float r = fmaf(kf, -kLn2Lo, fmaf(kf, -kLn2Hi, x));
    float t = fmaf(kPsiC6, r, kPsiC5);
    t = fmaf(t, r, kPsiC4);
    t = fmaf(t, r, kPsiC3);
    t = fmaf(t, r, kPsiC2);
    t = fmaf(t, r, kPsiC1);
    const float q = r * t;
    const float sc = pow2_neg(kf);
    return fmaf(sc, fmaf(r, q, r), 1.0f - sc);
}

__device__ __forceinline__ float2 psi2_of(float2 rho)
{
    const float2 x = f2(psi_clamp(rho.x), psi_clamp(rho.y));
    const float2 xk = mul2(x, sp2(kInvLn2));
    const float2 kf = f2(rintf(xk.x), rintf(xk.y));
    const float2 r = fma2(kf, sp2(-kLn2Lo), fma2(kf, sp2(-kLn2Hi), x));
    float2 t = fma2(sp2(kPsiC6), r, sp2(kPsiC5));
    t = fma2(t, r, sp2(kPsiC4));
    t = fma2(t, r, sp2(kPsiC3));
    t = fma2(t, r, sp2(kPsiC2));
    t = fma2(t, r, sp2(kPsiC1));
    const float2 q = mul2(r, t);
    const float2 sc = f2(pow2_neg(kf.x), pow2_neg(kf.y));
    return fma2(sc, fma2(r, q, r), sub2(sp2(1.0f), sc));
}

// Eq. SCforce on the psi ring: s0, s1, s2 are the planes z-1, z, z+1 of a
// [HY][HX] ring of pairs (psi^b, psi^r) (psi_pair), the node at row ty+1,
// column tx+1. S^a = sum_k G_k psi^abar(x + c_k) c_k ;  F^a = -g kappa psi^a(x) S^a.
// A neighbour's pair is one 8-byte shared-memory load, and its lanes are
// already the other component's psi for each lane a of the force.
template <int HX, int HY>
__device__ __forceinline__ void sc_force(const float2* s0, const float2* s1, const float2* s2, int ty, int tx,
                                         float gk, float Gax, float Gdi, float (&F)[2][3])
{
    auto psi_at = [&](int k) {
        const float2* sl = cz(k) < 0 ? s0 : (cz(k) > 0 ? s2 : s1);
        return sl[(ty + 1 + cy(k)) * HX + tx + 1 + cx(k)];
    };
    // opposite neighbours in pairs: psi(x + c_k) - psi(x - c_k), k odd
    float2 ax[3], di[3];
    bool hax[3] = {false, false, false}, hdi[3] = {false, false, false};
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        const float2 dk = sub2(psi_at(k), psi_at(k + 1));
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int c = q == 0 ? cx(k) : (q == 1 ? cy(k) : cz(k));
            if (!c) continue;
            if (is_axis(k)) acc_signed(ax[q], hax[q], dk, c);
            else acc_signed(di[q], hdi[q], dk, c);
        }
    }
    const float2 own = s1[(ty + 1) * HX + tx + 1];
    const float2 pre = mul2(sp2(-gk), f2(own.y, own.x));  // (psi^r, psi^b) of the node
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float2 Fd = mul2(pre, fma2(sp2(Gax), ax[d], mul2(sp2(Gdi), di[d])));
        F[0][d] = Fd.x;
        F[1][d] = Fd.y;
    }
}

// The ring stores each node's pair as (psi^b, psi^r): the value of component a
// sits in lane 1 - a.
__device__ __forceinline__ float2 psi_pair(float psi_r, float psi_b) { return make_float2(psi_b, psi_r); }
__device__ __forceinline__ float* psi_lane(float2* node, int a) { return (float*)node + (1 - a); }

// Where the node's populations go: neighbours (wrapped), the planes of z-1,
// z, z+1, and which links end on a wall. Only real nodes are written (no
// periodic images are stored). Addresses are a warp-uniform slot base plus a
// 32-bit per-thread offset.
struct Dest {
    int xo[3], yo[3];  // x-1, x, x+1 and y-1, y, y+1, wrapped
    int ro[3];         // row offsets of y-1, y, y+1 (incl. the left padding)
    int zo[3];         // plane offsets of z-1, z, z+1 (offsets stay below 2^31: slot < 2^31)
    bool bot, top;     // planar walls: solid plane below / above
    uint32_t nb;       // general geometry: bit k = link k ends on a solid node
    uint32_t hoff;     // added to the node's offset in the dither hash (0 unless the lattice is a z slab)
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
        hoff = 0;
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
// The two components are the lanes of packed pairs and are stored side by
// side, so each destination takes one paired store per velocity; opposite
// velocities are taken together (c_kbar.u = -c_k.u).
// For 16-bit storage the rest value, which balances the node's mass (taken
// exactly from m36 and the stored moving values), is rounded stochastically:
// round-to-nearest of nearly equal bulk values would bias the mass of every
// bulk node the same way, step after step. BF16 (8 significant bits) rounds
// the moving values stochastically too, a velocity's two values from the two
// halves of one 32-bit random word. The random bits come from a hash of
// the node and the lattice's step counter `clk`: fresh every step, and the
// same again when a checkpoint is replayed.
template <class S, bool kGeneral, bool kTauOne>
__device__ __forceinline__ void collide_store(const float (&rc)[2], const float (&jc)[2][3], const float (&vc)[2][Q],
                                              const float (&F)[2][3], const float (&tau)[2], const float (&itau)[2],
                                              const float (&ref)[2], S* __restrict__ dst, const Layout& L, int x, int y,
                                              const Dest& D, const float (&m36)[2], uint32_t clk = 0)
{
    // common velocity u' = sum_a j^a/tau^a / sum_a rho^a/tau^a
    const float den = fmaf(rc[1], itau[1], rc[0] * itau[0]);
    const float iden = den > 0.f ? __frcp_rn(den) : 0.f;
    float up[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) up[d] = fmaf(jc[1][d], itau[1], jc[0][d] * itau[0]) * iden;

    // per component (the two lanes): equilibrium velocity u' + tau F / rho and
    // the polynomial coefficients of Eq. Equil with c_s^2 = 1/3:
    // n^eq_k = zeta_k rho [1 + P_k],  P = cu (3 - 4.5 u^2 + 4.5 cu (1 + cu)) - 1.5 u^2
    float sh[2];
#pragma unroll
    for (int a = 0; a < 2; ++a) sh[a] = rc[a] > 1e-12f ? tau[a] * __frcp_rn(rc[a]) : 0.f;  // shift tau F / rho
    float2 u[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) u[d] = fma2(f2(sh[0], sh[1]), f2(F[0][d], F[1][d]), sp2(up[d]));
    const float2 usq = fma2(u[2], u[2], fma2(u[1], u[1], mul2(u[0], u[0])));
    const float2 A0 = fma2(sp2(-4.5f), usq, sp2(3.0f));
    const float2 B0 = mul2(sp2(-1.5f), usq);
    const float2 R = f2(rc[0], rc[1]);
    float2 w1, w2, base;
    if constexpr (Codec<S>::kDeviation) {
        w1 = w2 = R;  // e* = (rho - rho_ref) + rho P
        base = sub2(R, f2(ref[0], ref[1]));
    } else {
        w1 = mul2(R, sp2(1.0f / 18.0f));  // n* = zeta rho + zeta rho P
        w2 = mul2(R, sp2(1.0f / 36.0f));
        base = sp2(0.f);
    }
    const long long slot = L.slot;
    const int self = D.zo[1] + D.ro[1] + D.xo[1];
    float2 sum = sp2(0.f), sax = sp2(0.f), sdi = sp2(0.f);
    uint32_t hsh = 0;
    if constexpr (Codec<S>::kDitherMoving) hsh = node_hash((uint32_t)self + D.hoff, clk);
    // opposite velocities in pairs: c_{k+1} = -c_k (k odd, the first nonzero
    // component of c_k positive), so c_{k+1}.u = -(c_k.u) exactly
#pragma unroll
    for (int k = 1; k < Q; k += 2) {
        float2 cuk;
        if (is_axis(k)) {
            cuk = u[(k - 1) / 2];
        } else {
            const int d1 = cz(k) ? 2 : 1;                    // second nonzero component
            const int s1 = d1 == 2 ? cz(k) : cy(k);
            const float2 u0 = cx(k) ? u[0] : u[1];           // first nonzero component (+1)
            cuk = s1 > 0 ? add2(u0, u[d1]) : sub2(u0, u[d1]);
        }
        // P(+-cu) = E +- O with the even part E = 4.5 cu^2 + B0 and the odd
        // part O = cu (A0 + 4.5 cu^2), so the pair's equilibria in storage form
        // are T +- U with T = w E + base and U = w O
        const float2 w = is_axis(k) ? w1 : w2;
        const float2 c2 = mul2(cuk, cuk);
        const float2 T = fma2(w, fma2(sp2(4.5f), c2, B0), Codec<S>::kDeviation ? base : w);
        const float2 U = mul2(w, mul2(cuk, fma2(sp2(4.5f), c2, A0)));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int kk = k + h;
            const float2 qk = h ? sub2(T, U) : add2(T, U);  // equilibrium, storage form
            float2 s;
            if constexpr (kTauOne) {
                s = qk;
            } else {
                const float2 v = f2(vc[0][kk], vc[1][kk]);
                s = fma2(sub2(qk, v), f2(itau[0], itau[1]), v);
            }
            bool wall;
            if constexpr (kGeneral) wall = (D.nb >> kk) & 1u;
            else wall = (cz(kk) < 0 && D.bot) || (cz(kk) > 0 && D.top);
            // destination: the neighbour x + c_k, or slot kbar of this node (bounce-back)
            const int qo = wall ? self : D.zo[cz(kk) + 1] + D.ro[cy(kk) + 1] + D.xo[cx(kk) + 1];
            if constexpr (kCheckBounds)
                if (!in_bounds(qo, slot, D.err)) continue;
            S* q = dst + 2 * (qo + (long long)(wall ? opp(kk) : kk) * slot);  // the pair of both components
            if constexpr (Codec<S>::kDeviation) {
                // round both components' values into one pair; hv: the stored values in FP32
                float2 hv;
                typename Codec<S>::Pair h;
                if constexpr (Codec<S>::kDitherMoving) h = Codec<S>::sr2(s, rand32(hsh, kk), hv);
                else h = Codec<S>::rn2(s, hv);
                if (is_axis(kk)) sax = add2(sax, hv);
                else sdi = add2(sdi, hv);
                *(typename Codec<S>::Pair*)q = h;
            } else {
                sum = add2(sum, s);
                Codec<S>::store2(q, s.x, s.y);
            }
        }
    }
    if constexpr (kCheckBounds)
        if (!in_bounds(self, slot, D.err)) return;
    S* q0 = dst + 2 * (long long)self;
    if constexpr (Codec<S>::kDeviation) {
        uint32_t hrest;
        if constexpr (Codec<S>::kDitherMoving) hrest = node_hash(hsh, 0x632BE5ABu);  // a second full mixing round
        else hrest = node_hash((uint32_t)self + D.hoff, clk);
        // 12 e_0* = m36 - 2 sum_axis e_k* - sum_diag e_k*, the right side exact in FP32
        // the residual step makes the quotient round as x/12 itself would;
        // the rounded reciprocal alone scales every rest value by 1 + 3e-8
        const float2 x0 = sub2(f2(m36[0], m36[1]), fma2(sp2(2.0f), sax, sdi));
        float2 s0 = mul2(x0, sp2(1.0f / 12.0f));
        s0 = fma2(fma2(sp2(-12.0f), s0, x0), sp2(1.0f / 12.0f), s0);
        float2 unused;
        *(typename Codec<S>::Pair*)q0 = Codec<S>::sr2(s0, rand32(hrest, 0), unused);
    } else {
        const float2 r0 = sub2(R, sum);
        Codec<S>::store2(q0, r0.x, r0.y);
    }
}

}  // namespace lbsc
