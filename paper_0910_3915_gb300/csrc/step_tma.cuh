// Fused time step (Sec. 2) for the planar-wall geometry, with the next
// planes' populations staged into shared memory by TMA.
//
// A CTA owns a 32 x TY tile of columns and a z segment, as in the
// load-from-global kernel, but one thread streams whole planes of the tile
// plus its one-node ring (all 19 slots of paired values, one 4-D tensor box
// per plane) into an NS-deep ring of shared-memory stages with
// cp.async.bulk.tensor, completion tracked by one mbarrier per stage. The
// compute warps reduce a landed plane to rho, j and psi out of shared memory
// while the following planes are in flight, then collide and push the plane
// below. The periodic images come from small extra boxes of real nodes: two
// 16-byte column strips at the x edges, one row at the y edges (the row
// across the periodic boundary) and 16-byte corner pieces of that row, so no
// image of any node is ever stored. Every wait is bounded: a wait that gives
// up writes an error status, drains the CTA's copies in flight and leaves the
// kernel.
#pragma once

#include <cuda.h>

#include "lb_fields.cuh"
#include "step_common.cuh"

namespace lbsc {

constexpr uint32_t kSpinLimit = 1u << 22;  // try_wait rounds before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the completion of the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Geometry of one stage. The tensor maps order a buffer as (x values, storage
// row, plane, slot k), so a box of R rows and W columns lands in shared
// memory as [k][r][c][a]: element (k, r, c, a) at 2 ((k R + r) W + c) + a.
// (Ordering the slot before the row would make the layouts of all regions
// alike, but the copies would then walk the 19 slots, hundreds of megabytes
// apart, row by row: measured 16% slower.) Regions, each 128-byte aligned:
//   main     HY rows x BX columns: x = x0 - cofs + c (16 bytes of columns on
//            each side of the tile; edge tiles shift the box inward, see the
//            kernel), rows from the tile's row window;
//   xl, xr   HY rows x SX columns (16 bytes), the same rows: the left strip
//            holds the columns around x = nx - 1 (the images of x = -1), the
//            right strip x = 0 .. SX - 1 (the images of x >= nx); loaded only by
//            the tiles at the x edges;
//   ys       one row x BX columns: the row across the periodic y boundary
//            (y = ny - 1 for the first row of tiles, y = 0 for the last);
//   cl, cr   one row x SX columns: the x-edge pieces of that row.
// Element offsets count values (two per node).
template <class S, int TY>
struct TmaGeom {
    static constexpr int TX = 32, HX = TX + 2, HY = TY + 2;
    static constexpr int GX = edge_x<S>();                    // nodes in 16 bytes
    static constexpr int BX = TX + 2 * GX;                   // the box's nodes per row: 16 bytes of columns each side
    static constexpr int SX = GX;                            // strip width: 16 bytes of columns
    static constexpr int al(int elems) { return (elems * (int)sizeof(S) + 127) / 128 * 128 / (int)sizeof(S); }
    static constexpr int MAIN_ELEMS = 2 * Q * HY * BX;
    static constexpr int XS_ELEMS = 2 * Q * HY * SX;
    static constexpr int YS_ELEMS = 2 * Q * BX;
    static constexpr int CS_ELEMS = 2 * Q * SX;
    static constexpr int XL = al(MAIN_ELEMS), XR = XL + al(XS_ELEMS), YS = XR + al(XS_ELEMS);
    static constexpr int CL = YS + al(YS_ELEMS), CR = CL + al(CS_ELEMS);
    static constexpr int STAGE_ELEMS = CR + al(CS_ELEMS);
    static constexpr uint32_t MAIN_BYTES = MAIN_ELEMS * sizeof(S);
    static constexpr uint32_t XS_BYTES = XS_ELEMS * sizeof(S);
    static constexpr uint32_t YS_BYTES = YS_ELEMS * sizeof(S);
    static constexpr uint32_t CS_BYTES = CS_ELEMS * sizeof(S);
    static constexpr uint32_t STAGE_BYTES = STAGE_ELEMS * sizeof(S);
    static constexpr int PSI_FLOATS = 4 * 2 * HY * HX;
    static constexpr size_t smem(int NS) { return 128 + (size_t)NS * STAGE_BYTES + PSI_FLOATS * 4 + NS * 8; }
};

// Resident CTAs per SM the registers are held to (tau = 1): for 8-row tiles
// three FP32 CTAs (shared memory admits no more) and four 16-bit CTAs (64
// registers, a few words spilled: 32 warps per SM measured faster than 24);
// five CTAs of 4-row tiles; other variants take the compiler's choice.
template <class S, int TY, bool kTauOne>
constexpr int kTmaCtas = !kTauOne ? 1 : (TY == 8 ? (sizeof(S) == 2 ? 4 : 3) : (TY == 4 ? 5 : 1));

// The four tensor maps of one buffer and tile height: main box, x-edge strip,
// y-edge row, corner piece (boxes HY x BX, HY x SX, 1 x BX, 1 x SX nodes).
struct TmaMaps {
    CUtensorMap m[4];
};

// One work item: tile column `col` of the lattice A (tile row col / tiles_x,
// x tile col % tiles_x), fluid planes [za, zb), with the maps of A's source
// buffer. `stages`, `sp` and `bar` are the CTA's shared stages, psi ring and
// stage barriers; g counts the planes the CTA has consumed so far (the
// barriers' phases run on across items). Returns false when a wait gave up
// (the status word is set and the CTA's copies in flight are drained).
template <class S, int TY, int NS, bool kTauOne>
__device__ __forceinline__ bool tma_item(const TmaMaps& maps, const StepArgs<S>& A, int col, int za, int zb, S* stages,
                                         float* sp, uint64_t* bar, uint32_t& g, uint32_t clk)
{
    using G = TmaGeom<S, TY>;
    constexpr int TX = 32, NT = TX * TY, HX = G::HX, HY = G::HY, GX = G::GX, BX = G::BX, SX = G::SX;
    constexpr int RING = 2 * HX + 2 * TY;
    constexpr int NIT = (RING + NT - 1) / NT;
    using P2 = typename Codec<S>::Pair;

    const Layout L = A.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const long long plane = L.plane;
    S* __restrict__ dst = A.dst;
    const float eta[2] = {A.P.eta[0], A.P.eta[1]};
    const float ref[2] = {A.P.ref[0], A.P.ref[1]};
    const float tau[2] = {A.P.tau[0], A.P.tau[1]};
    const float itau[2] = {A.P.itau[0], A.P.itau[1]};
    const float gk = A.P.gk, Gax = A.P.Gax, Gdi = A.P.Gdi;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;

    // rows [y0, y0 + hgt) of an even split of ny (hgt <= TY); a row past hgt is an idle warp
    const int tyi = col / A.tiles_x;
    const int x0 = (col - tyi * A.tiles_x) * TX;
    const int y0 = tile_row(tyi, ny, A.tiles_y), hgt = tile_row(tyi + 1, ny, A.tiles_y) - y0;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = ty < hgt;
    const bool valid = active && gx < nx;
    const int np = zb - za + 2;  // planes za-1 .. zb
    // x edges: the periodic images come from the strips (column of x = nx - 1 in the left strip)
    const bool left_edge = x0 == 0, right_edge = x0 + TX >= nx;
    // the box's column of node x0: GX (16 bytes of ring columns on each
    // side); an edge tile takes its outer ring column from a strip, so its
    // box is shifted inward and reads no padding columns beyond the lattice
    // (0 at the left edge, 2 GX at the right edge)
    const int cofs = left_edge ? 0 : (right_edge ? 2 * GX : GX);
    const int sl = (L.gx + nx - 1) / SX * SX, ol = L.gx + nx - 1 - sl;
    // y edges: the row window of the box, given by the box row of node row
    // y0 (rofs). A middle tile's box holds rows y0 - 1 .. y0 + TY; the first
    // row of tiles' rows 0 .. HY - 1 and the last row's the HY rows ending at
    // its last own row, the ring row across the boundary coming from the
    // y-edge row (ys, with its corner pieces). With a single row of tiles
    // (ny <= TY) the box holds every row and the ring rows wrap inside it.
    const bool single = A.tiles_y == 1;
    const bool first = tyi == 0 && !single, last = tyi == A.tiles_y - 1 && !single;
    const int rofs = (first || single) ? 0 : (last ? HY - hgt : 1);
    const int yrow = first ? ny - 1 : 0;  // the real row in ys (first or last row of tiles)
    // own node: the main box; lanes past x = nx - 1 of a ragged last tile
    // hold the periodic images x - nx from the right strip (the one at
    // x = nx is the +x neighbour of x = nx - 1), as far as the strip reaches
    const bool own_strip = gx >= nx;
    const bool own_rd = active && gx - nx < SX;
    const int own_off = own_strip ? G::XR + 2 * ((ty + rofs) * SX + gx - nx) : 2 * ((ty + rofs) * BX + tx + cofs);
    // the copies' coordinates: x of the main box and of the left strip in
    // values (two per node; 16-byte aligned, as the copy requires), storage
    // row (real row + 1) of the box's first row and of the y-edge row (-1: none)
    const int xb = 2 * (x0 + L.gx - cofs), xs = 2 * sl;
    const int yb = y0 - rofs + 1, ysr = (first || last) ? yrow + 1 : -1;

    // ring items (one per ring node, both components): shared-memory
    // position, stage position of the node's slot-0 pair, and its region's
    // slot stride: 0 main box (2 HY BX), 1 x strip (2 HY SX), 2 y-edge row
    // (2 BX), 3 corner piece (2 SX)
    // (packed in one word: stage position in bits 0-16, shared-memory position in
    // bits 17-26, stride class in bits 27-28; -1 for no item)
    static_assert(G::STAGE_ELEMS <= (1 << 17) && HY * HX <= (1 << 10), "ring item fields fit their bits");
    int it_code[NIT];
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int r = tid + i * NT;
        it_code[i] = -1;
        if (r < RING) {
            int it_sm, it_base, it_cls;
            int ix, iy;
            if (r < HX) { ix = r; iy = 0; }
            else if (r < 2 * HX) { ix = r - HX; iy = hgt + 1; }
            else if (r < 2 * HX + TY) { ix = 0; iy = r - 2 * HX + 1; }
            else { ix = HX - 1; iy = r - 2 * HX - TY + 1; }
            const bool on = r < 2 * HX || iy <= hgt;  // side columns: the tile's own rows only
            it_sm = iy * HX + ix;
            const int xr = x0 - 1 + ix, yr = y0 - 1 + iy;  // the ring node (unwrapped)
            const bool across = (first && yr < 0) || (last && yr >= ny);  // in the y-edge row
            const int row = wrapi(yr, ny) - y0 + rofs;                   // box row otherwise
            if (xr < 0) {  // x = -1: the image of x = nx - 1
                it_cls = across ? 3 : 1;
                it_base = across ? G::CL + 2 * ol : G::XL + 2 * (row * SX + ol);
            } else if (xr >= nx && xr - nx < SX) {  // x >= nx: the images of x - nx
                it_cls = across ? 3 : 1;
                it_base = across ? G::CR + 2 * (xr - nx) : G::XR + 2 * (row * SX + xr - nx);
            } else {
                it_cls = across ? 2 : 0;
                it_base = across ? G::YS + 2 * (ix - 1 + cofs) : 2 * (row * BX + ix - 1 + cofs);
            }
            if (on) it_code[i] = it_base | (it_sm << 17) | (it_cls << 27);
        }
    }

    auto issue = [&](int zp, uint32_t gi) {
        uint64_t* b = &bar[gi % NS];
        if ((zp == 0 && !(A.halo & 1)) || (zp == nz - 1 && !(A.halo & 2))) {
            mbar_arrive(b);  // a wall plane: nothing to load (a z slab's halo plane is loaded like fluid)
        } else {
            S* stg = stages + (size_t)(gi % NS) * G::STAGE_ELEMS;
            const bool ye = ysr >= 0;
            fence_proxy_async();
            mbar_expect_tx(b, G::MAIN_BYTES + (left_edge ? G::XS_BYTES : 0u) + (right_edge ? G::XS_BYTES : 0u) +
                                  (ye ? G::YS_BYTES + (left_edge ? G::CS_BYTES : 0u) +
                                            (right_edge ? G::CS_BYTES : 0u)
                                      : 0u));
            tma_load_4d(stg, &maps.m[0], b, xb, yb, zp, 0);
            if (left_edge) tma_load_4d(stg + G::XL, &maps.m[1], b, xs, yb, zp, 0);
            if (right_edge) tma_load_4d(stg + G::XR, &maps.m[1], b, 2 * L.gx, yb, zp, 0);
            if (ye) {
                tma_load_4d(stg + G::YS, &maps.m[2], b, xb, ysr, zp, 0);
                if (left_edge) tma_load_4d(stg + G::CL, &maps.m[3], b, xs, ysr, zp, 0);
                if (right_edge) tma_load_4d(stg + G::CR, &maps.m[3], b, 2 * L.gx, ysr, zp, 0);
            }
        }
    };

    // wait for plane i of the item, reduce it to psi (tile + ring) and own
    // moments, then refill its stage with plane i + NS
    auto consume = [&](int i, float (&rho)[2], float (&j)[2][3], float (&v)[2][Q], float (&m)[2]) -> bool {
        const int zp = za - 1 + i;
        const uint32_t gi = g + i;
        const bool ok = mbar_wait(&bar[gi % NS], (gi / NS) & 1u);
        float2* spl = (float2*)sp + (zp & 3) * (HY * HX);
        const bool solid = (zp == 0 && !(A.halo & 1)) || (zp == nz - 1 && !(A.halo & 2));
        if (ok) {
            const S* st = stages + (size_t)(gi % NS) * G::STAGE_ELEMS;
            float ps[2] = {eta[0], eta[1]};
            rho[0] = rho[1] = m[0] = m[1] = 0.f;
#pragma unroll
            for (int a = 0; a < 2; ++a) j[a][0] = j[a][1] = j[a][2] = 0.f;
            if (!solid && own_rd) {
                float w[2][Q];
                // both components of velocity k in one shared-memory load
                const P2* so = (const P2*)(st + own_off);
                if (!own_strip) {
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const float2 t = Codec<S>::val2(so[k * HY * BX]);
                        w[0][k] = t.x;
                        w[1][k] = t.y;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const float2 t = Codec<S>::val2(so[k * HY * SX]);
                        w[0][k] = t.x;
                        w[1][k] = t.y;
                    }
                }
                moments2<S>(w, ref, rho, j, m);
                const float2 p2 = psi2_of(f2(rho[0], rho[1]));
                ps[0] = p2.x;
                ps[1] = p2.y;
                if constexpr (!kTauOne) {
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int k = 0; k < Q; ++k) v[a][k] = w[a][k];
                }
            }
            if (active) {
                spl[(ty + 1) * HX + tx + 1] = psi_pair(ps[0], ps[1]);
            }
#pragma unroll
            for (int q = 0; q < NIT; ++q) {
                const int code = it_code[q];
                if (code < 0) continue;
                const int it_sm = (code >> 17) & 0x3FF;
                float2 pr = f2(eta[0], eta[1]);
                if (!solid) {
                    // both components of velocity k in one shared-memory load
                    float2 w[Q];
                    const P2* si = (const P2*)(st + (code & 0x1FFFF));
                    const int cls = (code >> 27) & 3;
                    if (cls == 0) {
#pragma unroll
                        for (int k = 0; k < Q; ++k) w[k] = Codec<S>::val2(si[k * HY * BX]);
                    } else if (cls == 1) {
#pragma unroll
                        for (int k = 0; k < Q; ++k) w[k] = Codec<S>::val2(si[k * HY * SX]);
                    } else if (cls == 2) {
#pragma unroll
                        for (int k = 0; k < Q; ++k) w[k] = Codec<S>::val2(si[k * BX]);
                    } else {
#pragma unroll
                        for (int k = 0; k < Q; ++k) w[k] = Codec<S>::val2(si[k * SX]);
                    }
                    float2 unused;
                    pr = psi2_of(rho2_of<S>(w, f2(ref[0], ref[1]), unused));
                }
                spl[it_sm] = psi_pair(pr.x, pr.y);
            }
        }
        const bool bad = __syncthreads_or(!ok);
        if (bad) {
            if (tid == 0) {
                atomicOr(A.err, kErrWait);
                for (int k2 = i; k2 < np && k2 < i + NS; ++k2) mbar_wait(&bar[(g + k2) % NS], ((g + k2) / NS) & 1u);
            }
            return false;
        }
        if (tid == 0 && i + NS < np) issue(zp + NS, gi + NS);
        return true;
    };

    float rc[2], jc[2][3], vc[2][Q], mc[2];
    float rn[2], jn[2][3], vn[2][Q], mn[2];
    __syncthreads();  // the previous item's collide is done with the psi ring
    if (tid == 0)
        for (int i = 0; i < NS && i < np; ++i) issue(za - 1 + i, g + i);
    if (!consume(0, rn, jn, vn, mn) || !consume(1, rc, jc, vc, mc)) return false;

    Dest D;
    D.set_column(L, valid ? gx : 0, valid ? gy : 0);
    D.err = A.err;
    D.hoff = A.hkey;

    for (int z = za; z < zb; ++z) {
        if (!consume(z - za + 2, rn, jn, vn, mn)) return false;
        if (valid) {
            float F[2][3];
            const float2* ring = (const float2*)sp;
            sc_force<HX, HY>(ring + ((z - 1) & 3) * (HY * HX), ring + (z & 3) * (HY * HX),
                             ring + ((z + 1) & 3) * (HY * HX), ty, tx, gk, Gax, Gdi, F);
            D.zo[0] = (int)((z - 1) * plane);
            D.zo[1] = (int)(z * plane);
            D.zo[2] = (int)((z + 1) * plane);
            D.bot = z - 1 == 0 && !(A.halo & 1);  // a halo plane takes pushes like fluid
            D.top = z + 1 == nz - 1 && !(A.halo & 2);
            if constexpr (Codec<S>::kDeviation) {
                // rho = rho_ref + m36 / 36, as moments2 forms it: not held across the plane
                const float2 r = fma2(f2(mc[0], mc[1]), sp2(1.0f / 36.0f), f2(ref[0], ref[1]));
                const float rr[2] = {r.x, r.y};
                collide_store<S, false, kTauOne>(rr, jc, vc, F, tau, itau, ref, dst, L, gx, gy, D, mc, clk);
            } else {
                collide_store<S, false, kTauOne>(rc, jc, vc, F, tau, itau, ref, dst, L, gx, gy, D, mc, clk);
            }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            if constexpr (!Codec<S>::kDeviation) rc[a] = rn[a];
            mc[a] = mn[a];
#pragma unroll
            for (int d = 0; d < 3; ++d) jc[a][d] = jn[a][d];
            if constexpr (!kTauOne) {
#pragma unroll
                for (int k = 0; k < Q; ++k) vc[a][k] = vn[a][k];
            }
        }
    }
    g += np;
    return true;
}

template <class S, int TY, int NS, bool kTauOne>
__global__ void __launch_bounds__(32 * TY, (kTmaCtas<S, TY, kTauOne>))
    step_tma_kernel(const __grid_constant__ TmaMaps maps, const StepArgs<S> A)
{
    using G = TmaGeom<S, TY>;
    static_assert(G::STAGE_BYTES % 128 == 0 && (G::XL * sizeof(S)) % 128 == 0 && (G::YS * sizeof(S)) % 128 == 0 &&
                      (G::CL * sizeof(S)) % 128 == 0 && (G::CR * sizeof(S)) % 128 == 0,
                  "stages and their regions stay 128-byte aligned");
    static_assert((2 * G::BX * sizeof(S)) % 16 == 0 && (2 * G::SX * sizeof(S)) % 16 == 0,
                  "box rows are whole 16-byte units");
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    S* stages = (S*)base;
    float* sp = (float*)(base + (size_t)NS * G::STAGE_BYTES);  // psi ring [4][HY][HX] of pairs (psi^b, psi^r)
    uint64_t* bar = (uint64_t*)(sp + G::PSI_FLOATS);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t g = 0;  // planes this CTA has issued and consumed so far
    uint32_t clk = 0;
    if constexpr (Codec<S>::kDeviation) clk = clock_read(A.clock);
    const int ncol = A.tiles_x * A.tiles_y;
    const int nzf = A.zhi - A.zlo;
    for (int item = blockIdx.x; item < ncol * A.nseg; item += gridDim.x) {
        const int col = item % ncol, seg = item / ncol;
        const int za = A.zlo + (int)((long long)seg * nzf / A.nseg);
        const int zb = A.zlo + (int)((long long)(seg + 1) * nzf / A.nseg);
        if (za >= zb) continue;
        if (!tma_item<S, TY, NS, kTauOne>(maps, A, col, za, zb, stages, sp, bar, g, clk)) break;
    }
    if constexpr (Codec<S>::kDeviation) clock_tick(A.clock);
}

// Batched TMA step: a persistent grid walks a work list of (box, tile column,
// first plane, end plane) items over many planar-wall lattices with their own
// sizes and parameters; args[2 box + parity] and maps[2 box + parity] describe
// box `box` for this step (the maps live in global memory, written by the host
// before the launch). The last CTA out advances every box's step counter.
template <class S, int TY, int NS, bool kTauOne>
__global__ void __launch_bounds__(32 * TY, (kTmaCtas<S, TY, kTauOne>))
    batch_tma_kernel(const TmaMaps* __restrict__ maps, const StepArgs<S>* __restrict__ args,
                     const int4* __restrict__ items, int nitems, int parity, int nbox, uint32_t* done)
{
    using G = TmaGeom<S, TY>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    S* stages = (S*)base;
    float* sp = (float*)(base + (size_t)NS * G::STAGE_BYTES);
    uint64_t* bar = (uint64_t*)(sp + G::PSI_FLOATS);
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint32_t g = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const StepArgs<S>& A = args[2 * w.x + parity];
        const TmaMaps& M = maps[2 * w.x + parity];
        if (threadIdx.x == 0)
            for (int i = 0; i < 4; ++i)  // the maps were written through the generic proxy
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&M.m[i]) : "memory");
        uint32_t clk = 0;
        if constexpr (Codec<S>::kDeviation) clk = clock_read(A.clock);
        if (!tma_item<S, TY, NS, kTauOne>(M, A, w.y, w.z, w.w, stages, sp, bar, g, clk)) break;
    }
    if constexpr (Codec<S>::kDeviation) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(done, 1u) == gridDim.x - 1) {
                atomicExch(done, 0u);
                for (int b = 0; b < nbox; ++b) atomicAdd(args[2 * b].clock, 1u);
            }
        }
    }
}

template <class S, int TY, int NS, bool T1>
static cudaError_t tma_launch_one(const CUtensorMap* m, const StepArgs<S>& A, cudaStream_t st)
{
    const size_t smem = TmaGeom<S, TY>::smem(NS);
    const int items = A.tiles_x * A.tiles_y * A.nseg;
    TmaMaps maps;
    for (int i = 0; i < 4; ++i) maps.m[i] = m[i];
    step_tma_kernel<S, TY, NS, T1><<<items, 32 * TY, smem, st>>>(maps, A);
    return cudaGetLastError();
}

template <class S, int TY, int NS, bool T1>
static cudaError_t tma_prepare_one()
{
    return cudaFuncSetAttribute(step_tma_kernel<S, TY, NS, T1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)TmaGeom<S, TY>::smem(NS));
}

template <class S, int TY, int NS, bool T1>
static int tma_occ_one()
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, step_tma_kernel<S, TY, NS, T1>, 32 * TY,
                                                      TmaGeom<S, TY>::smem(NS)) != cudaSuccess)
        return 1;
    return n;
}

// Dispatch over the built (tile height, stages, tau == 1) combinations.
// op 0: launch; op 1: set the shared-memory attribute; op 2: occupancy.
template <class S>
static long long tma_dispatch(int op, int ty, int ns, bool t1, const CUtensorMap* m, const StepArgs<S>* A,
                              cudaStream_t st)
{
#define LBSC_TMA_CASE(TY_, NS_)                                                                       \
    if (ty == TY_ && ns == NS_) {                                                                     \
        if (op == 0) return t1 ? tma_launch_one<S, TY_, NS_, true>(m, *A, st)                         \
                               : tma_launch_one<S, TY_, NS_, false>(m, *A, st);                       \
        if (op == 1) {                                                                                \
            cudaError_t e = tma_prepare_one<S, TY_, NS_, true>();                                     \
            return e != cudaSuccess ? e : tma_prepare_one<S, TY_, NS_, false>();                      \
        }                                                                                             \
        return t1 ? tma_occ_one<S, TY_, NS_, true>() : tma_occ_one<S, TY_, NS_, false>();             \
    }
    LBSC_TMA_CASE(4, 1)
    LBSC_TMA_CASE(4, 2)
    LBSC_TMA_CASE(4, 3)
    LBSC_TMA_CASE(8, 1)
    LBSC_TMA_CASE(8, 2)
    LBSC_TMA_CASE(8, 3)
    if constexpr (sizeof(S) == 2) {
        LBSC_TMA_CASE(16, 1)
        LBSC_TMA_CASE(16, 2)
    }
#undef LBSC_TMA_CASE
    return op == 2 ? 0 : (long long)cudaErrorInvalidValue;
}

// The batched TMA kernel for one stage and 4- or 8-row tiles: op 0 launches
// on `grid` CTAs (returns a cudaError_t), op 1 sets the shared-memory
// attribute, op 2 returns resident CTAs per SM (0 if not built).
template <class S, int TY, bool T1>
static long long tma_batch_one(int op, const TmaMaps* maps, const StepArgs<S>* args, const int4* items, int nitems,
                               int parity, int nbox, uint32_t* done, int grid, cudaStream_t st)
{
    const size_t smem = TmaGeom<S, TY>::smem(1);
    if (op == 0) {
        batch_tma_kernel<S, TY, 1, T1><<<grid, 32 * TY, smem, st>>>(maps, args, items, nitems, parity, nbox, done);
        return cudaGetLastError();
    }
    if (op == 1)
        return cudaFuncSetAttribute(batch_tma_kernel<S, TY, 1, T1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_tma_kernel<S, TY, 1, T1>, 32 * TY, smem) !=
        cudaSuccess)
        return 0;
    return n;
}

template <class S>
static long long tma_batch_dispatch(int op, int ty, bool t1, const void* maps, const StepArgs<S>* args,
                                    const int4* items, int nitems, int parity, int nbox, uint32_t* done, int grid,
                                    cudaStream_t st)
{
    const TmaMaps* m = (const TmaMaps*)maps;
    if (ty == 4)
        return t1 ? tma_batch_one<S, 4, true>(op, m, args, items, nitems, parity, nbox, done, grid, st)
                  : tma_batch_one<S, 4, false>(op, m, args, items, nitems, parity, nbox, done, grid, st);
    if (ty == 8)
        return t1 ? tma_batch_one<S, 8, true>(op, m, args, items, nitems, parity, nbox, done, grid, st)
                  : tma_batch_one<S, 8, false>(op, m, args, items, nitems, parity, nbox, done, grid, st);
    return op == 2 ? 0 : (long long)cudaErrorInvalidValue;
}

}  // namespace lbsc
