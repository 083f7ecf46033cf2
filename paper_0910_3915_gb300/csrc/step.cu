// Fused time step of the two-component Shan-Chen D3Q19 model (Sec. 2),
// load-from-global variant: any solid mask (general geometry) and any tile.
//
// Design: populations are double-buffered (read src, write dst), structure of
// arrays, one 32-node row segment per warp. A CTA owns a tile of 32 x TY
// columns and a range of z planes and marches upward in z. For plane z it
// collides, with psi of planes z-1..z+1 (tile plus a one-node ring) held in a
// four-plane shared-memory ring; the ring nodes' psi comes from their
// populations in src, which no CTA writes during the step, so psi never
// travels through HBM. Loads run two planes ahead of the collision: the raw
// populations of plane z+2 are requested into registers before plane z is
// collided and reduced to rho, j and psi one iteration later, so memory
// latency overlaps the arithmetic of the plane below.
#include "lb_fields.cuh"
#include "step_common.cuh"

namespace lbsc {

// One work item: tile column `col` of the lattice A, fluid planes [za, zb).
// sp: the CTA's psi ring, [4][TY+2][34] pairs (psi^b, psi^r).
template <class S, int TY, bool kGeneral, bool kTauOne>
__device__ __forceinline__ void step_item(const StepArgs<S>& A, int col, int za, int zb,
                                          float2 (&sp)[4][TY + 2][34], uint32_t clk)
{
    constexpr int TX = 32, NT = TX * TY, HX = TX + 2, HY = TY + 2;
    constexpr int RING = 2 * HX + 2 * TY;          // ring nodes around the tile
    constexpr int NIT = (2 * RING + NT - 1) / NT;  // ring items (node, component) per thread

    const Layout L = A.L;
    const int nx = L.nx, ny = L.ny, nz = L.nz, px = L.px;
    const int plane = (int)L.plane;
    const long long slot = L.slot;
    const S* __restrict__ src = A.src;
    S* __restrict__ dst = A.dst;
    const uint32_t* __restrict__ nbmask = A.nbmask;
    const float eta[2] = {A.P.eta[0], A.P.eta[1]};
    const float ref[2] = {A.P.ref[0], A.P.ref[1]};
    const float tau[2] = {A.P.tau[0], A.P.tau[1]};
    const float itau[2] = {A.P.itau[0], A.P.itau[1]};
    const float gk = A.P.gk, Gax = A.P.Gax, Gdi = A.P.Gdi;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;

    // tile rows [y0, y0 + hgt): the tiles_y tiles split the ny rows evenly
    // (hgt <= TY); one warp per row, so a row past hgt is an idle warp
    const int tyi = col / A.tiles_x;
    const int x0 = (col - tyi * A.tiles_x) * TX;
    const int y0 = tile_row(tyi, ny, A.tiles_y), hgt = tile_row(tyi + 1, ny, A.tiles_y) - y0;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool active = ty < hgt;
    const bool valid = active && gx < nx;
    const int ox = gx % nx;  // ragged x: a wrapped copy of a real column (the +x neighbour's psi)
    const int own = (gy + 1) * px + ox + L.gx;

    // this thread's ring items: smem position, plane offset of the node, component
    int it_sm[NIT], it_a[NIT], it_off[NIT];
#pragma unroll
    for (int i = 0; i < NIT; ++i) {
        const int it = tid + i * NT;
        it_a[i] = -1;
        it_sm[i] = 0;
        it_off[i] = 0;
        if (it < 2 * RING) {
            const int a = it >= RING, r = it - a * RING;
            int ix, iy;
            if (r < HX) { ix = r; iy = 0; }
            else if (r < 2 * HX) { ix = r - HX; iy = hgt + 1; }
            else if (r < 2 * HX + TY) { ix = 0; iy = r - 2 * HX + 1; }
            else { ix = HX - 1; iy = r - 2 * HX - TY + 1; }
            const int hx = ((x0 - 1 + ix) % nx + nx) % nx, hy = ((y0 - 1 + iy) % ny + ny) % ny;
            if (r < 2 * HX || iy <= hgt) it_a[i] = a;  // side columns: the tile's own rows only
            it_sm[i] = iy * HX + ix;
            it_off[i] = (hy + 1) * px + hx + L.gx;
        }
    }

    // raw populations of the plane in flight (own node, ring items) and
    // whether each node is solid
    float ro_[2][Q], ri_[NIT][Q];
    bool so_ = false, si_[NIT];

    // request plane zp into the raw registers
    auto issue = [&](int zp) {
        const int zw = kGeneral ? wrapi(zp, nz) : zp;
        const int zoff = zw * plane;
        const bool wall_plane = !kGeneral && ((zp == 0 && !(A.halo & 1)) || (zp == nz - 1 && !(A.halo & 2)));
        if (!active) so_ = true;  // idle row: no loads, no psi
        // bounds-checked build: every slot of a node lies in the buffer iff its offset in the slot does
        else if (kCheckBounds && !in_bounds((long long)zoff + own, L.slot, A.err)) so_ = true;
        else if constexpr (kGeneral) so_ = (__ldg(nbmask + zoff + own) & kSelfSolid) != 0;
        else so_ = wall_plane;
        if (!so_) {
            const S* p = src + 2 * (long long)(zoff + own);  // per-thread node pointer, uniform slot offsets
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float2 t = Codec<S>::load2(p + 2 * k * slot);  // both components of velocity k
                ro_[0][k] = t.x;
                ro_[1][k] = t.y;
            }
        }
#pragma unroll
        for (int i = 0; i < NIT; ++i) {
            if (it_a[i] < 0) continue;
            if (kCheckBounds && !in_bounds((long long)zoff + it_off[i], L.slot, A.err)) si_[i] = true;
            else if constexpr (kGeneral) si_[i] = (__ldg(nbmask + zoff + it_off[i]) & kSelfSolid) != 0;
            else si_[i] = wall_plane;
            if (!si_[i]) {
                const S* p = src + 2 * (long long)(zoff + it_off[i]) + it_a[i];  // one component of the ring node
#pragma unroll
                for (int k = 0; k < Q; ++k) ri_[i][k] = Codec<S>::load(p + 2 * k * slot);
            }
        }
    };
    // reduce the raw registers of plane zp: psi into its ring slot, own moments out
    auto reduce = [&](int zp, float (&rho)[2], float (&j)[2][3], float (&v)[2][Q], float (&m)[2]) {
        float2* spl = &sp[zp & 3][0][0];
        float ps[2] = {eta[0], eta[1]};
        rho[0] = rho[1] = m[0] = m[1] = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a) j[a][0] = j[a][1] = j[a][2] = 0.f;
        if (!so_) {
            moments2<S>(ro_, ref, rho, j, m);
            const float2 p2 = psi2_of(f2(rho[0], rho[1]));
            ps[0] = p2.x;
            ps[1] = p2.y;
            if constexpr (!kTauOne) {
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int k = 0; k < Q; ++k) v[a][k] = ro_[a][k];
            }
        }
        if (active) {
            spl[(ty + 1) * HX + tx + 1] = psi_pair(ps[0], ps[1]);
        }
#pragma unroll
        for (int i = 0; i < NIT; ++i) {
            if (it_a[i] < 0) continue;
            const int a = it_a[i];
            // select, not index: a runtime index would put eta and ref in local memory
            const float eta_a = a ? eta[1] : eta[0], ref_a = a ? ref[1] : ref[0];
            *psi_lane(&spl[it_sm[i]], a) = si_[i] ? eta_a : psi_of(rho_of<S>(ri_[i], ref_a));
        }
    };

    float rc[2], jc[2][3], vc[2][Q], mc[2];
    float rn[2], jn[2][3], vn[2][Q], mn[2];
    __syncthreads();  // the previous item's readers are done with the ring
    issue(za - 1);
    reduce(za - 1, rn, jn, vn, mn);
    issue(za);
    reduce(za, rc, jc, vc, mc);
    issue(za + 1);

    Dest D;
    D.set_column(L, valid ? gx : 0, valid ? gy : 0);
    D.err = A.err;
    D.hoff = A.hkey;

    for (int z = za; z < zb; ++z) {
        reduce(z + 1, rn, jn, vn, mn);
        if (z + 2 <= zb) issue(z + 2);
        __syncthreads();

        bool self_solid = false;
        if constexpr (kGeneral) {
            if (valid) {
                D.nb = __ldg(nbmask + z * plane + own);
                self_solid = (D.nb & kSelfSolid) != 0;
            }
        }
        if (valid && !self_solid) {
            float F[2][3];
            sc_force<HX, HY>(&sp[(z - 1) & 3][0][0], &sp[z & 3][0][0], &sp[(z + 1) & 3][0][0], ty, tx,
                             gk, Gax, Gdi, F);
            if constexpr (kGeneral) {
                D.zo[0] = wrapi(z - 1, nz) * plane;
                D.zo[2] = wrapi(z + 1, nz) * plane;
            } else {
                D.zo[0] = (z - 1) * plane;
                D.zo[2] = (z + 1) * plane;
            }
            D.zo[1] = z * plane;
            D.bot = !kGeneral && z - 1 == 0 && !(A.halo & 1);  // a halo plane takes pushes like fluid
            D.top = !kGeneral && z + 1 == nz - 1 && !(A.halo & 2);
            collide_store<S, kGeneral, kTauOne>(rc, jc, vc, F, tau, itau, ref, dst, L, gx, gy, D, mc, clk);
        }
        // rotate: next plane becomes current
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            rc[a] = rn[a];
            mc[a] = mn[a];
#pragma unroll
            for (int d = 0; d < 3; ++d) jc[a][d] = jn[a][d];
            if constexpr (!kTauOne) {
#pragma unroll
                for (int k = 0; k < Q; ++k) vc[a][k] = vn[a][k];
            }
        }
    }
}

// Resident CTAs per SM the register budget is sized for (tau = 1 kernels, which
// keep no pre-collision populations): the FP32 kernel with 8-row tiles fits 128
// registers without spilling (two CTAs of 256 threads), 4-row tiles are held to
// three CTAs of 128 threads (168 registers). Other variants: one CTA.
template <class S, int TY, bool kTauOne>
constexpr int kMinCtas = !kTauOne ? 1 : (TY == 4 ? 3 : ((sizeof(S) == 4 && TY == 8) ? 2 : 1));

template <class S, int TY, bool kGeneral, bool kTauOne>
__global__ void __launch_bounds__(32 * TY, (kMinCtas<S, TY, kTauOne>)) step_kernel(const StepArgs<S> A)
{
    __shared__ float2 sp[4][TY + 2][34];  // psi pairs of 4 planes, slot = z & 3
    const int ncol = A.tiles_x * A.tiles_y;
    const int nzf = A.zhi - A.zlo;
    uint32_t clk = 0;
    if constexpr (Codec<S>::kDeviation) clk = clock_read(A.clock);
    for (int item = blockIdx.x; item < ncol * A.nseg; item += gridDim.x) {
        const int col = item % ncol, seg = item / ncol;
        const int za = A.zlo + (int)((long long)seg * nzf / A.nseg);
        const int zb = A.zlo + (int)((long long)(seg + 1) * nzf / A.nseg);
        if (za >= zb) continue;
        step_item<S, TY, kGeneral, kTauOne>(A, col, za, zb, sp, clk);
    }
    if constexpr (Codec<S>::kDeviation) clock_tick(A.clock);
}

// Batched step: a persistent grid walks a work list of (box, tile column,
// first plane, end plane) items over many lattices with their own sizes and
// parameters; args[2*box + parity] describes box `box` for this step.
template <class S, int TY, bool kTauOne>
__global__ void __launch_bounds__(32 * TY)
    batch_step_kernel(const StepArgs<S>* __restrict__ args, const int4* __restrict__ items, int nitems, int parity,
                      int nbox, uint32_t* done)
{
    __shared__ float2 sp[4][TY + 2][34];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];
        const StepArgs<S> A = args[2 * w.x + parity];
        uint32_t clk = 0;
        if constexpr (Codec<S>::kDeviation) clk = clock_read(A.clock);
        step_item<S, TY, false, kTauOne>(A, w.y, w.z, w.w, sp, clk);
    }
    if constexpr (Codec<S>::kDeviation) {
        // the last CTA out advances every box's step counter
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

// resident CTAs per SM of the load-from-global step kernel
int step_occupancy(int precision, int tile_y, bool general, bool tau_one)
{
    switch (precision) {
    case 0: return occ_s<float>(tile_y, general, tau_one);
    case 1: return occ_s<__half>(tile_y, general, tau_one);
    default: return occ_s<__nv_bfloat16>(tile_y, general, tau_one);
    }
}

template <class S, int TY>
static cudaError_t batch_ty(const StepArgs<S>* args, const int4* items, int nitems, int parity, bool tau_one,
                            int grid, int nbox, uint32_t* done, cudaStream_t st)
{
    if (tau_one) batch_step_kernel<S, TY, true><<<grid, 32 * TY, 0, st>>>(args, items, nitems, parity, nbox, done);
    else batch_step_kernel<S, TY, false><<<grid, 32 * TY, 0, st>>>(args, items, nitems, parity, nbox, done);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_batch_step(const StepArgs<S>* args, const int4* items, int nitems, int parity, int tile_y,
                              bool tau_one, int grid, int nbox, uint32_t* done, cudaStream_t st)
{
    switch (tile_y) {
    case 4: return batch_ty<S, 4>(args, items, nitems, parity, tau_one, grid, nbox, done, st);
    case 8: return batch_ty<S, 8>(args, items, nitems, parity, tau_one, grid, nbox, done, st);
    case 16: return batch_ty<S, 16>(args, items, nitems, parity, tau_one, grid, nbox, done, st);
    default: return cudaErrorInvalidValue;
    }
}

// resident CTAs per SM of the batched kernel
template <class S>
int batch_occupancy(int tile_y, bool tau_one)
{
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (tile_y) {
    case 4:
        e = tau_one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 4, true>, 128, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 4, false>, 128, 0);
        break;
    case 8:
        e = tau_one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 8, true>, 256, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 8, false>, 256, 0);
        break;
    default:
        e = tau_one ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 16, true>, 512, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_step_kernel<S, 16, false>, 512, 0);
    }
    return e == cudaSuccess && n > 0 ? n : 1;
}

// Self-test of psi: out[i] = psi_of(rho[i]); the packed lanes of
// psi2_of(rho[i], rho[n-1-i]) in out[n + i] and out[2n + i]; and
// out[3n + i] = -expm1f(-rho[i]) from the CUDA math library.
__global__ void psi_probe_kernel(const float* __restrict__ rho, int n, float* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[i] = psi_of(rho[i]);
        const float2 p = psi2_of(f2(rho[i], rho[n - 1 - i]));
        out[n + i] = p.x;
        out[2 * n + i] = p.y;
        out[3 * n + i] = -expm1f(-rho[i]);
    }
}

cudaError_t launch_psi_probe(const float* rho, int n, float* out, cudaStream_t st)
{
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    psi_probe_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(rho, n, out);
    return cudaGetLastError();
}

// Self-test of the 16-bit stochastic rounding: out[i] = the stored pair
// (as its 32-bit word) that Codec<S>::sr2 makes of (v[2i], v[2i+1]) with the
// random word m[i]; out[n + i] and out[2n + i] = the FP32 values it reports
// back for the mass balance, as bit patterns.
template <class S>
__global__ void round_probe_kernel(const float* __restrict__ v, const uint32_t* __restrict__ m, int n,
                                   uint32_t* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float2 back;
        const typename Codec<S>::Pair h = Codec<S>::sr2(make_float2(v[2 * i], v[2 * i + 1]), m[i], back);
        out[i] = *(const uint32_t*)&h;
        out[n + i] = __float_as_uint(back.x);
        out[2 * n + i] = __float_as_uint(back.y);
    }
}

cudaError_t launch_round_probe(int precision, const float* v, const uint32_t* m, int n, uint32_t* out,
                               cudaStream_t st)
{
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    if (precision == 1) round_probe_kernel<__half><<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(v, m, n, out);
    else round_probe_kernel<__nv_bfloat16><<<blocks < 1 ? 1 : blocks, 256, 0, st>>>(v, m, n, out);
    return cudaGetLastError();
}

#define LBSC_BATCH_INST(S)                                                                                     \
    template cudaError_t launch_batch_step<S>(const StepArgs<S>*, const int4*, int, int, int, bool, int, int, uint32_t*, \
                                              cudaStream_t);                                                 \
    template int batch_occupancy<S>(int, bool);
LBSC_BATCH_INST(float)
LBSC_BATCH_INST(__half)
LBSC_BATCH_INST(__nv_bfloat16)

template cudaError_t launch_step<float>(const StepArgs<float>&, int, bool, bool, cudaStream_t);
template cudaError_t launch_step<__half>(const StepArgs<__half>&, int, bool, bool, cudaStream_t);
template cudaError_t launch_step<__nv_bfloat16>(const StepArgs<__nv_bfloat16>&, int, bool, bool, cudaStream_t);

}  // namespace lbsc
