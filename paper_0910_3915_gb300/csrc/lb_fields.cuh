// Declarations shared by the kernels' translation units and the C-ABI layer.
#pragma once

#include <cuda.h>

#include "lb_internal.cuh"

namespace lbsc {

constexpr int kRedThreads = 256;  // threads per reduction block
constexpr int kRedBlocks = 512;   // fixed grid of the reductions: fixed summation order
constexpr int kConsBlocks = 2048;   // most blocks of the conservation sums (one wave of resident blocks is used)
constexpr int kAngleBlocks = 1216;  // fixed grid of the contact-angle reduction
constexpr int kAngleVals = 19;    // contact-angle partial sums per block
constexpr int kPartRows = kConsBlocks > kAngleBlocks ? kConsBlocks : kAngleBlocks;  // rows of the partials area
constexpr uint32_t kAngleMaxMask = (1u << 0) | (1u << 17) | (1u << 18);  // max-reduced entries of the 19

// Geometry and parameters for the non-step kernels.
struct FieldArgs {
    Layout L;
    KParams P;
    int general;                    // 0: solid layers z = 0 and z = nz-1; 1: nbmask
    const uint32_t* nbmask;
};

// Unpadded float fields (index x + nx*(y + ny*z)) used by readback kernels.
struct Scratch {
    float* rho[2];
    float* j[3];
    float* psi[2];
    float* u[3];
};

// Dense FP32 fields of the adjoint (index x + nx*(y + ny*z)).
struct AdjFields {
    float* rho[2];   // forward: densities
    float* psi[2];   // forward: psi (wall pseudo-density on solid nodes)
    float* j[2][3];  // forward: momenta
    float* rhob[2];  // adjoint of rho before the psi term
    float* jb[2][3]; // adjoint of j
    float* V[2][3];  // adjoint of the neighbour sum S^a: -g kappa psi^a Fbar^a
    float* psib[2];  // adjoint of psi^a from the node's own force
};
struct AdjArgs {
    int nx, ny, nz;
    float gk, G[Q];  // G[k]: neighbour weight of link k (G[0] unused)
    float tau[2], omega[2];
    float eta[2];
};
constexpr int kAdjBlocks = 512;
template <class S>
cudaError_t launch_adj_forward(const Layout& L, const KParams& P, const S* f, const AdjFields& A, cudaStream_t st);
cudaError_t launch_adj_backstep(const AdjArgs& G, const AdjFields& A, const float* lam_next, float* lam_cur,
                                double* part, double* acc, cudaStream_t st);
cudaError_t launch_observable(int nx, int ny, int nz, int obs, double eps, const float* rr, const float* rb,
                              double* part, double* sums, float* lam, cudaStream_t st);

template <class S>
cudaError_t launch_step(const StepArgs<S>& A, int tile_y, bool general, bool tau_one, cudaStream_t st);
// TMA-staged step for planar walls: op 0 launches (returns a cudaError_t),
// op 1 sets the kernels' shared-memory attribute, op 2 returns resident CTAs
// per SM (0 if the (tile_y, stages) pair is not built for S).
template <class S>
long long tma_step(int op, int tile_y, int stages, bool tau_one, const CUtensorMap* map, const StepArgs<S>* args,
                   cudaStream_t stream);
template <class S>
cudaError_t launch_batch_step(const StepArgs<S>* args, const int4* items, int nitems, int parity, int tile_y,
                              bool tau_one, int grid, int nbox, uint32_t* done, cudaStream_t st);
// Batched TMA-staged step (planar walls, one stage, 4- or 8-row tiles): maps
// is a device array of 2 nbox groups of the four tensor maps (box i, source
// buffer p at 2 i + p, 64-byte aligned); ops as for tma_step (op 0 launches
// on `grid` CTAs).
template <class S>
long long tma_batch(int op, int tile_y, bool tau_one, const void* maps, const StepArgs<S>* args, const int4* items,
                    int nitems, int parity, int nbox, uint32_t* done, int grid, cudaStream_t stream);
template <class S>
int batch_occupancy(int tile_y, bool tau_one);
// bounded-wait self-test: a wait nothing satisfies, limit try_wait rounds
cudaError_t launch_wait_probe(int* err, unsigned limit, cudaStream_t st);
cudaError_t launch_psi_probe(const float* rho, int n, float* out, cudaStream_t st);
// 16-bit rounding self-test (precision 1 = FP16, 2 = BF16)
cudaError_t launch_round_probe(int precision, const float* v, const uint32_t* m, int n, uint32_t* out,
                               cudaStream_t st);
// set a lattice's device step counter to v (and its done-ticket to 0)
cudaError_t launch_clock_set(uint32_t* clk, uint32_t v, cudaStream_t st);
template <class S>
cudaError_t launch_init(const FieldArgs& F, S* f, const double* rr, const double* rb, cudaStream_t st,
                        int* err = nullptr);
// FP64 conservation sums into out[0..7] through 64-bit fixed-point accumulators
// acc[0..6] and a block ticket, both zero between calls (the kernel clears them)
constexpr float kConsFix = 268435456.0f;  // 2^28: the accumulators' unit is 2^-28
// phi (optional): also write phi = rho_r - rho_b of every node, as launch_phi does
template <class S>
cudaError_t launch_conservation(const FieldArgs& F, const S* f, unsigned long long* acc, unsigned int* ticket,
                                double* out, cudaStream_t st, float* phi = nullptr);
template <class S>
cudaError_t launch_fields(const FieldArgs& F, const S* f, const Scratch& W, bool velocity, cudaStream_t st);
// phi = rho_r - rho_b of every node into W.rho[0] (the contact angle's input)
template <class S>
cudaError_t launch_phi(const FieldArgs& F, const S* f, const Scratch& W, cudaStream_t st);
cudaError_t launch_angle(const FieldArgs& F, const Scratch& W, double zref, double level, double* part, double* out,
                         cudaStream_t st);
// pressure tensor of Sec. 4.1 (after launch_fields with velocity): every node,
// per-plane sums, and fixed-point radial bins (see fields.cu)
template <class S>
cudaError_t launch_pressure_field(const FieldArgs& F, const S* f, const Scratch& W, double* out, cudaStream_t st);
template <class S>
cudaError_t launch_pressure_planes(const FieldArgs& F, const S* f, const Scratch& W, double* out, cudaStream_t st);
constexpr int kRadialBinsMax = 1024;
constexpr double kRadialFix = 1073741824.0;  // fixed-point unit of the radial sums: 2^-30
cudaError_t launch_pressure_radial(const FieldArgs& F, const void* f, int prec, const Scratch& W, const double* centre,
                                   double dr, int nbins, double zmin, unsigned long long* out, cudaStream_t st);
// z-slab face messages (halo.cu): 38 entries of nx*ny values per face
constexpr int kHaloEntries = 38;
// face 0 = below (planes 0, 1), 1 = above (planes nz-2, nz-1); unpack 0 packs
// the lattice's outgoing message into msg, 1 applies the neighbour's message
cudaError_t launch_halo_copy(const Layout& L, void* f, size_t elem, void* msg, int face, int unpack, cudaStream_t st);
// both messages of the face between slab A (below) and B (above), lattice to lattice
cudaError_t launch_halo_exchange(const Layout& LA, void* fa, const Layout& LB, void* fb, size_t elem, cudaStream_t st);
template <class S>
cudaError_t launch_get_pop(const FieldArgs& F, const S* f, double* out, cudaStream_t st);
template <class S>
cudaError_t launch_set_pop(const FieldArgs& F, S* f, const double* in, cudaStream_t st);

}  // namespace lbsc
