/*
 * lbsc: two-component Shan-Chen lattice Boltzmann (D3Q19) on one GB300 GPU.
 *
 * The method is that of Schmieschek & Harting, "Contact angle determination
 * in multicomponent lattice Boltzmann simulations":
 *   - Sec. 2, Eq. LBeqs     evolution n_k(x + c_k, t+1) - n_k(x, t) = Omega_k
 *   - Sec. 2                BGK collision Omega_k = -(n_k - n_k^eq)/tau
 *   - Sec. 2, Eq. Equil     cubic equilibrium n_k^eq(rho, u)
 *   - Sec. 2, Eq. SCforce   F^a = -psi^a g sum_{x'} psi^abar(x') (x' - x),
 *                           psi = 1 - exp(-rho), velocity shift tau F / rho
 *   - Sec. 2                walls: mid-grid bounce-back, and the wall acting as
 *                           an extra species with a pseudo-density
 *   - Sec. 3, Eq. geoCA     geometric contact angle from base, height, radius
 *
 * Conventions shared by every entry point:
 *   - Status: every function returns LB_OK (0) or a negative LB_ERR_* code and
 *     never throws; lb_last_error() gives the message of the last failure.
 *   - Host arrays are owned by the caller and are only read or written during
 *     the call. Field arrays hold nx*ny*nz values indexed x + nx*(y + ny*z).
 *   - Device memory is owned by the context (allocated in lb_init, released
 *     by lb_free) unless the caller passes its own buffer to lb_init_external.
 *   - Work is queued on the CUDA stream given at init, in order. lb_step is
 *     asynchronous; device-side errors surface at the next call that waits
 *     (lb_moments, lb_contact_angle, lb_save, lb_sync).
 *   - Lattice units throughout. x and y are periodic; z is periodic unless
 *     walled off by solid nodes. The default geometry has solid layers at
 *     z = 0 and z = nz - 1, i.e. mid-grid wall planes at z = 0.5 and
 *     z = nz - 1.5.
 */
#ifndef LBSC_H
#define LBSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LB_OK 0
#define LB_ERR_ARG (-1)              /* invalid argument (null pointer, bad size or value) */
#define LB_ERR_CUDA (-2)             /* a CUDA call failed (out of memory, launch failure) */
#define LB_ERR_NAN (-3)              /* the state holds non-finite populations */
#define LB_ERR_BARRIER_TIMEOUT (-4)  /* a bounded device-side wait gave up */
#define LB_ERR_STATE (-5)            /* call not valid in the context's current state */
#define LB_ERR_UNSUPPORTED (-6)      /* combination of options not built */

/* population storage */
#define LB_F32 0   /* populations in FP32 */
#define LB_F16 1   /* FP16 deviations e_k = n_k/zeta_k - rho_ref, FP32 arithmetic */
#define LB_BF16 2  /* BF16 deviations, as above */

/* step kernel variants (lb_set_step_variant) */
#define LB_STEP_AUTO 0  /* the TMA kernel with one stage where it applies, else load-from-global */
#define LB_STEP_LDG 1   /* every plane loaded from global memory by the compute threads */
#define LB_STEP_TMA 2   /* planes staged into shared memory by TMA (planar walls only) */

/* neighbour weights G_k of the Shan-Chen force sum */
#define LB_WEIGHTS_UNIT 0  /* G_k = 1 for the 18 neighbours, as Eq. SCforce is printed */
#define LB_WEIGHTS_W36 1   /* G_k = 36 zeta_k: 2 on axes, 1 on diagonals */

typedef struct lb_ctx lb_ctx;

/* Model parameters (Sec. 2).
 *   tau_r, tau_b   BGK relaxation times, > 0.5 (kinematic viscosity (2 tau - 1)/6)
 *   g_br           inter-component coupling g_{r b}, > 0 repulsive
 *   eta_wall_r     wall pseudo-density standing in for psi^r at solid nodes (felt by b)
 *   eta_wall_b     wall pseudo-density standing in for psi^b at solid nodes (felt by r)
 *                  A signed wettability w maps to (eta_wall_r, eta_wall_b) = (-w, +w):
 *                  w > 0 repels the r droplet.
 *   force_weights  LB_WEIGHTS_UNIT or LB_WEIGHTS_W36
 *   force_scale    multiplier kappa on every force term (1 = the printed force) */
typedef struct {
    double tau_r, tau_b, g_br, eta_wall_r, eta_wall_b;
    int force_weights;
    double force_scale;
} lb_params;

/* Geometric droplet measurement (Sec. 3). */
typedef struct {
    double theta_deg;     /* contact angle from Eq. geoCA, read as atan2(b/2, r - h) */
    double theta_fit_deg; /* contact angle of a least-squares sphere through interface points */
    double h;             /* apex height of the phi = 0 surface above the wall plane z = 0.5 */
    double b;             /* base diameter at the wall, from r and h */
    double r;             /* sphere radius from the cap above the reference plane */
    double base_ref;      /* equivalent-circle diameter of {phi > 0} at the reference plane */
    double xc, yc, zc;    /* fitted sphere centre */
    double r_fit;         /* fitted sphere radius */
    int ok;               /* 1 if theta_deg, h, b, r are defined (status == LB_DROP_OK) */
    int n_points;         /* interface points in the sphere fit */
    double phi_max;       /* max of rho_r - rho_b over fluid nodes (the droplet phase's contrast) */
    double phi_min;       /* min of rho_r - rho_b over fluid nodes */
    int status;           /* LB_DROP_*: why theta is missing, checked in this order */
} lb_droplet;

/* lb_droplet.status (the interface is phi = rho_r - rho_b = level) */
#define LB_DROP_OK 0         /* a cap with its apex above the reference plane and a base there */
#define LB_DROP_BAD_PLANE 1  /* the reference plane wall + offset (and the plane above it) is outside the lattice */
#define LB_DROP_NO_PHASE 2   /* no fluid node has phi > level: the droplet phase has dissolved */
#define LB_DROP_NO_APEX 3    /* phi > level somewhere, but never below a node with phi <= level */
#define LB_DROP_LOW_APEX 4   /* the apex is not above the reference plane: a cap flatter than the offset */
#define LB_DROP_NO_BASE 5    /* no phi > level area at the reference plane: the drop is detached */

/* Create a context on the current CUDA device.
 * nx, ny, nz >= 1 (nz >= 3 with the default walls), and one population plane
 * set (padded rows times ny+2 rows times nz) below 2^31 elements, i.e. up to
 * about 1.9e9 nodes; precision LB_F32/LB_F16/LB_BF16.
 * rho_r, rho_b: host arrays (nx*ny*nz doubles) of initial densities; populations
 * start at rest equilibrium n_k = zeta_k rho (Eq. Equil at u = 0). Values on
 * solid nodes are ignored. For 16-bit storage the deviation reference rho_ref
 * of each component is the mean of its initial density over fluid nodes.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which all work
 * of this context is queued. Parameters start as tau = 1, g_br = 0, no wall
 * force, unit weights, force_scale 1. On error *out is NULL. */
int lb_init(lb_ctx** out, int nx, int ny, int nz, int precision,
            const double* rho_r, const double* rho_b, void* cuda_stream);

/* Re-initialise an existing context from new initial densities (host arrays
 * of nx*ny*nz doubles, as lb_init), without allocating: populations at rest
 * equilibrium, step count and device step counter back to 0. Geometry,
 * parameters, schedule and (16-bit storage) the deviation references of
 * lb_init stay. The densities are checked on the GPU: LB_ERR_ARG if one is
 * negative or not finite (the populations are then undefined until the next
 * successful reset). Host arrays in pinned memory copy asynchronously; the
 * call synchronises the context's stream before it returns. */
int lb_reset(lb_ctx* ctx, const double* rho_r, const double* rho_b);

/* ------------------------------------------------------------ z-slab decomposition
 * The update of a node needs only its nearest neighbours (Sec. 2), so a
 * lattice splits into slabs of whole z planes with one exchange per step.
 * A slab is a context of nx x ny x nz planes whose planes 1..nz-2 it owns.
 * Plane 0 and plane nz-1 are either the solid wall layers of the whole
 * lattice or halo planes: copies of the neighbouring slab's boundary plane,
 * read for psi (the force at the owned boundary plane) and pushed into like
 * fluid nodes, never updated by the slab's own step. After every step the
 * two slabs of a face exchange one message each way (lb_halo_pack /
 * lb_halo_unpack, or lb_halo_exchange lattice to lattice): the 5 crossing
 * populations per component per face node and the 28 boundary-plane values
 * the neighbour's halo plane takes; then the slabs' owned planes hold exactly
 * what the whole lattice holds (bitwise: each node's arithmetic is the same).
 * Stepping a slab further without the exchange leaves its boundary planes
 * stale. A slab with neighbours on both faces owns at least two planes (the
 * plane it sends must be final after its own step). Slabs always use the
 * load-from-global step kernel and planar walls. */
#define LB_HALO_BELOW 1 /* plane 0 is a halo plane (a neighbour below) */
#define LB_HALO_ABOVE 2 /* plane nz-1 is a halo plane (a neighbour above) */

/* Create a slab: as lb_init on the slab's nz planes (rho_r, rho_b: host,
 * nx*ny*nz doubles, including the halo planes' initial densities, i.e. the
 * neighbours' boundary planes). halo: LB_HALO_BELOW | LB_HALO_ABOVE as the
 * slab has neighbours. zbase: index in the whole lattice of the slab's plane
 * 0 (it keys 16-bit storage's rounding dither by the node's position in the
 * whole lattice). ref: NULL, or the whole lattice's 16-bit deviation
 * references {rho_ref_r, rho_ref_b} (its mean initial densities over fluid
 * nodes), which every slab must share. */
int lb_init_slab(lb_ctx** out, int nx, int ny, int nz, int precision, const double* rho_r, const double* rho_b,
                 void* cuda_stream, int halo, int zbase, const double* ref);

/* Bytes of one face message: 38 * nx * ny values in the storage format. */
int lb_halo_bytes(lb_ctx* ctx, size_t* bytes);

/* Enqueue (on the context's stream) the copy of this slab's outgoing message
 * for face 0 (below) or 1 (above) into msg (device memory of lb_halo_bytes
 * bytes): entries 0..9 the crossing populations (component a, i-th of the
 * crossing velocities: entry 5a + i), entries 10..37 the boundary plane's
 * values with c_z of that direction or 0 (entry 10 + 14a + i), x fastest.
 * LB_ERR_STATE if the slab has no halo plane on that face. */
int lb_halo_pack(lb_ctx* ctx, int face, void* msg);

/* Enqueue the application of the neighbour's message (its lb_halo_pack of
 * the facing side) on face 0 (below) or 1 (above). */
int lb_halo_unpack(lb_ctx* ctx, int face, const void* msg);

/* Both messages of one face, lattice to lattice, in one kernel: `below` has
 * a halo plane above, `above` one below; same nx, ny, precision and stream
 * (the same device, or devices with peer access to each other's memory). */
int lb_halo_exchange(lb_ctx* below, lb_ctx* above);

/* nsteps steps of a lattice split into nslab slabs (ordered bottom to top,
 * halo planes exactly on their inner faces, one stream): each step steps
 * every slab and then exchanges every face. */
int lb_slabs_step(lb_ctx* const* slabs, int nslab, int nsteps);

/* Bytes of device memory lb_init_external needs for this lattice. */
int lb_required_bytes(int nx, int ny, int nz, int precision, size_t* bytes);

/* As lb_init, but the populations and scratch live in a caller-owned device
 * buffer of at least lb_required_bytes bytes, 256-byte aligned, that must
 * outlive the context. The context allocates no population memory itself. */
int lb_init_external(lb_ctx** out, int nx, int ny, int nz, int precision,
                     const double* rho_r, const double* rho_b, void* cuda_stream,
                     void* device_buffer, size_t buffer_bytes);

/* Set the solid mask: host array of nx*ny*nz bytes, 1 = solid (mid-grid
 * bounce-back, Sec. 2; the wall pseudo-densities act from solid nodes).
 * A mask with solid layers exactly at z = 0 and z = nz - 1 selects the
 * planar-wall kernels; any other mask the general kernels. Must leave at
 * least one fluid node. Populations already on solid nodes are discarded. */
int lb_set_geometry(lb_ctx* ctx, const uint8_t* solid);

/* Set the model parameters (copied). LB_ERR_ARG if tau <= 0.5, a value is
 * not finite, or force_weights is unknown. */
int lb_set_params(lb_ctx* ctx, const lb_params* params);

/* Advance nsteps >= 0 time steps of Eq. LBeqs (moments, psi, Shan-Chen and
 * wall force, force-shifted cubic equilibrium, BGK, streaming with mid-grid
 * bounce-back) on the context's stream. Asynchronous. The steps run as
 * launches of CUDA graphs of 2^i steps (one per set bit of nsteps, and one
 * per 32 steps); the first call after the schedule, the parameters or the
 * geometry changed captures those graphs (on a private stream) before it
 * launches. */
int lb_step(lb_ctx* ctx, int nsteps);

/* Wait for the stream and report a device-side failure, if any. */
int lb_sync(lb_ctx* ctx);

/* Failure-detection self-test (a library facility; the paper has no
 * counterpart). Runs the bounded device-side wait used by the TMA-staged step
 * on an mbarrier that nothing completes, with spin_limit try_wait rounds
 * (1 .. 2^20). The wait gives up, the kernel records the failure in the
 * context's device status word and returns without faulting. Returns
 * LB_ERR_BARRIER_TIMEOUT (the expected outcome); the context stays usable. */
int lb_selftest_bounded_wait(lb_ctx* ctx, unsigned spin_limit);

/* Self-test of the step's pseudopotential psi = 1 - exp(-rho) (Sec. 2; the
 * library evaluates it by its own range reduction and series, not by a
 * math-library call). rho: n host floats (1 <= n <= 2^24). out: 4n host
 * floats, written with
 *   out[i]        psi as the step computes it for a ring node,
 *   out[n + i]    psi of rho[i] in the first lane of the packed (two-component)
 *                 evaluation of the pair (rho[i], rho[n-1-i]),
 *   out[2n + i]   psi of rho[n-1-i] in the second lane of that evaluation,
 *   out[3n + i]   -expm1f(-rho[i]) from the CUDA math library, for comparison.
 * Runs on the current device with temporary device memory (synchronous).
 * LB_ERR_ARG for NULL arrays or n out of range, LB_ERR_CUDA on a CUDA error
 * (messages via lb_last_error(NULL)). */
int lb_selftest_psi(const float* rho, int n, float* out);

/* Self-test of the stochastic rounding of 16-bit storage (a design choice
 * of this library, not of the paper: the values stored are rounded so that
 * each rounds up with probability equal to its discarded fraction).
 * precision: LB_F16 or LB_BF16. v: 2n host floats, pairs (v[2i], v[2i+1]) as
 * the step stores a velocity's two components; m: n random words, one per
 * pair. out: 3n host words, written with
 *   out[i]        the stored pair as a 32-bit word (first value in the low half),
 *   out[n + i]    the first stored value converted back to FP32, as bits,
 *   out[2n + i]   the second, likewise (the values the mass balance uses).
 * 1 <= n <= 2^24. Runs on the current device with temporary device memory
 * (synchronous). LB_ERR_ARG for another precision, NULL arrays or n out of
 * range, LB_ERR_CUDA on a CUDA error (messages via lb_last_error(NULL)). */
int lb_selftest_round(int precision, const float* v, const unsigned* m, int n, unsigned* out);

/* Read densities and conservation sums (Sec. 2, moments). Any output may be NULL.
 * rho_r, rho_b: nx*ny*nz doubles. u: 3*nx*ny*nz doubles (component-major),
 * the barycentric velocity (sum_a j^a + F/2)/sum_a rho^a with F the total
 * Shan-Chen force. cons[8] = {mass_r, mass_b, Px, Py, Pz (sum of j over
 * nodes and components), non-finite population count, fluid nodes, steps
 * taken}, summed in FP64 on the device in a fixed order.
 * Returns LB_ERR_NAN (after filling the outputs) if any population is not finite. */
int lb_moments(lb_ctx* ctx, double* rho_r, double* rho_b, double* u, double cons[8]);

/* Conservation sums only (cons as in lb_moments), without field copies. */
int lb_conservation(lb_ctx* ctx, double cons[8]);

/* Contact angle of the r droplet on the bottom wall (Sec. 3): phi = rho_r -
 * rho_b = 0 located by linear interpolation, apex height h, base b' at the
 * reference plane `offset` above the wall plane (the paper uses 5 l.u.),
 * sphere radius r from that cap, base b at the wall from r and h, then theta.
 * Needs the default wall at z = 0 and offset >= 0. out->ok = 0 (and LB_OK)
 * when no cap is found. */
int lb_contact_angle(lb_ctx* ctx, double offset, lb_droplet* out);

/* As lb_contact_angle with the interface at phi = level instead of phi = 0.
 * Fig. 4 of the paper draws its error bars from the interface at half the
 * maximum |phi|: level = +max(phi)/2 and level = min(phi)/2. */
int lb_contact_angle_at(lb_ctx* ctx, double offset, double level, lb_droplet* out);

/* The conservation sums (as lb_conservation, into cons[8]) and the droplet's
 * geometric contact angle at level 0 (as lb_contact_angle, into out) of the
 * current state, in one read of the populations: the sums' pass also forms
 * phi = rho_r - rho_b for the angle. The results are those of the two calls
 * made one after the other. Synchronous. Errors as lb_conservation and
 * lb_contact_angle (LB_ERR_ARG for NULL arguments or an offset that is
 * negative or not finite). */
int lb_measure(lb_ctx* ctx, double cons[8], double offset, lb_droplet* out);

/* ------------------------------------------------------------ pressure tensor and surface tension
 * The pressure tensor of Sec. 4.1 at a fluid node x:
 *   P_ij = sum_a sum_k (c_ki - u_i)(c_kj - u_j) n_k^a
 *        + 1/4 sum_(a, abar) g kappa sum_k G_k [psi^a(x) psi^abar(x+c_k) + psi^abar(x) psi^a(x+c_k)] c_ki c_kj
 * with u the velocity lb_moments reports, G_k and kappa the force's weights and
 * scale, and psi of a solid neighbour the wall pseudo-density (as in the
 * force). Solid nodes contribute nothing. Evaluated in FP64 from the stored
 * populations. Components are ordered xx, yy, zz, xy, xz, yz. Each call
 * allocates and frees its device scratch and synchronises the stream. */

/* P: host, 6*nx*ny*nz doubles, P[c*N + idx] (zeros on solid nodes). */
int lb_pressure_tensor(lb_ctx* ctx, double* P);

/* Plane averages along z (Eq. gammaMechDef with the interface normal to z):
 * prof (host, nz*8 doubles): prof[z*8 + v] = mean over the fluid nodes of
 * plane z of P_xx, P_yy, P_zz, P_xy, P_xz, P_yz and phi = rho_r - rho_b,
 * then the fluid count (zeros for a solid plane). gamma_sum (may be NULL):
 * sum over planes with fluid of P_N - P_T, P_N = P_zz, P_T = (P_xx + P_yy)/2;
 * a box with m identical interfaces holds m gamma. The per-plane sums are
 * deterministic (one block per plane, fixed order). */
int lb_pressure_profile(lb_ctx* ctx, double* prof, double* gamma_sum);

/* Radial profile about centre[3] (x, y, z lattice coordinates; distances use
 * the minimum image along x and y, and along z for a mask geometry) for
 * Eq. mechRadGamma: fluid nodes with z >= zmin at r > 0 fall in bin
 * floor(r/dr) (1 <= nbins <= 1024, dr > 0); bins (host, nbins*4 doubles) gets
 * per bin the mean P_N = n.P.n (n the unit vector from the centre), the mean
 * P_T = (tr P - P_N)/2, the mean phi and the count. R_s (may be NULL) is the
 * radius where the bin-mean phi first changes sign going outward, by linear
 * interpolation between bin centres r_b = (b + 1/2) dr (NaN if it never
 * does); gamma (may be NULL) = sum over bins with r_b <= r_max of
 * (r_b/R_s)^2 (P_N - P_T) dr (0 without R_s). Sums are accumulated in 64-bit
 * fixed point (2^-30 units), so the result does not depend on thread order. */
int lb_pressure_radial(lb_ctx* ctx, const double* centre, double dr, int nbins, double zmin, double r_max,
                       double* bins, double* gamma, double* R_s);

/* Young's equation (Eq. young): cos theta = (gamma_SG - gamma_SL)/gamma_LG,
 * theta in degrees, clamped to 0 or 180 outside [-1, 1] (complete wetting or
 * drying). LB_ERR_ARG for non-finite tensions or gamma_LG <= 0 (message via
 * lb_last_error(NULL)). Host only. */
int lb_young_theta(double gamma_sg, double gamma_sl, double gamma_lg, double* theta_deg);

/* Huang's closed form (Eq. huangSigmaLG) for the r droplet, with the same
 * coupling g for fluid-fluid and fluid-wall pairs (which cancels):
 * cos theta = (G_ads,b - G_ads,r) / (g (rho_in - rho_out)/2), where
 * G_ads,r = g eta_wall_b and G_ads,b = g eta_wall_r are the wall
 * interactions each component feels, and rho_in > rho_out the r densities
 * inside and outside the drop. Degrees, clamped as above. Host only. */
int lb_huang_theta(double eta_wall_r, double eta_wall_b, double rho_in, double rho_out, double* theta_deg);

/* Checkpoint: bytes of the state, and copies to / from a host buffer of that
 * size. The state is the population array plus the step counter; params and
 * geometry are not part of it. */
int lb_state_bytes(lb_ctx* ctx, size_t* bytes);
int lb_save(lb_ctx* ctx, void* host, size_t bytes);
int lb_load(lb_ctx* ctx, const void* host, size_t bytes);

/* Copy the populations to a host array of 2*19*nx*ny*nz doubles laid out
 * [component][k][z][y][x], decoded to n_k. Velocity order: k = 0 rest,
 * 1..6 = +x,-x,+y,-y,+z,-z, 7..18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),
 * (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1). */
int lb_get_populations(lb_ctx* ctx, double* n);

/* Replace the populations from a host array laid out as in lb_get_populations. */
int lb_set_populations(lb_ctx* ctx, const double* n);

/* Build properties: LB_BUILD_BOUNDS_CHECKED is set in a library compiled
 * with LBSC_DEBUG_BOUNDS, whose step kernels check every population index
 * against its buffer, skip an access that falls outside and report
 * LB_ERR_STATE at the next lb_sync or readback (a stand-in for a memory
 * checker: no access leaves the buffer, no trap). */
#define LB_BUILD_BOUNDS_CHECKED 1
int lb_build_flags(int* flags);

/* Choose the step kernel's tile height (4, 8 or 16 rows of 32 nodes) and the
 * number of z segments per tile column (0 = automatic). */
int lb_set_schedule(lb_ctx* ctx, int tile_y, int z_segments);

/* The same, with the ny rows split evenly into y_tiles tiles of at most
 * tile_y rows (0 = ceil(ny / tile_y)), so that the count of (tile column,
 * z segment) work items can be matched to the GPU's resident CTAs.
 * LB_ERR_ARG if a tile would need more than tile_y rows or y_tiles > ny.
 * Like every schedule choice it changes no value of the result. */
int lb_set_tiling(lb_ctx* ctx, int tile_y, int y_tiles, int z_segments);

/* Choose the step kernel: LB_STEP_AUTO, LB_STEP_LDG or LB_STEP_TMA, and for
 * the TMA kernel the number of shared-memory stages, i.e. planes in flight
 * (1, 2 or 3; 0 = automatic: 1 for LB_STEP_AUTO, else 3, else 2). One stage
 * leaves room for more resident CTAs per SM (measured the fastest on GB300).
 * Every variant computes bit-identical results. LB_STEP_AUTO and LB_STEP_TMA
 * with a non-planar geometry, or a (tile height, stages) pair that
 * is not built for the precision, fall back to LB_STEP_LDG. */
int lb_set_step_variant(lb_ctx* ctx, int variant, int stages);

/* ------------------------------------------------------------ adjoint
 * Observables of the final densities (phi = rho_r - rho_b, sigma the logistic
 * function, eps = 0.05, sums over fluid nodes, heights above the wall plane):
 *   LB_OBS_COM       sum (z - 1/2) rho_r / sum rho_r
 *   LB_OBS_COM_SOFT  sum (z - 1/2) sigma(phi/eps) / sum sigma(phi/eps)  (droplet centre height)
 *   LB_OBS_WETTED    sum over the first fluid layer of sigma(phi/eps)    (wetted area) */
#define LB_OBS_COM 0
#define LB_OBS_COM_SOFT 1
#define LB_OBS_WETTED 2

/* Advance nsteps time steps (the context ends at step nsteps, as after
 * lb_step) and return J = observable of the final state and the exact
 * gradient of J with respect to the wall pseudo-densities,
 * dJ_deta[0] = dJ/d eta_wall_r, dJ_deta[1] = dJ/d eta_wall_b, computed by the
 * discrete adjoint of the step (Sec. 2: the reverse of streaming with
 * bounce-back, BGK with Eq. Equil, the velocity shift and Eq. SCforce with
 * the wall as a species). States are checkpointed every ckpt_every steps
 * and recomputed one segment at a time (device memory: nsteps/ckpt_every + 1
 * + ckpt_every states). Planar walls only (LB_ERR_UNSUPPORTED otherwise).
 * The paper calibrates the wall parameter by repeated runs; the gradient
 * replaces that search. J may be NULL. */
int lb_step_backward(lb_ctx* ctx, int nsteps, int ckpt_every, int observable, double* dJ_deta, double* J);

/* The observable of the current state (no stepping). */
int lb_observable(lb_ctx* ctx, int observable, double* J);

/* ------------------------------------------------------------ batches
 * Many independent droplet lattices, each with its own size and parameters,
 * advanced together: one persistent kernel launch per time step walks a work
 * list of (lattice, tile column, z range) items, and runs of 32 steps are
 * replayed as a captured CUDA graph. This is the paper's kind of parameter
 * sweep (Sec. 4: theta against system size and wall parameter) done in one
 * launch per step instead of one run per parameter set. Every box uses the
 * default walls (solid layers z = 0 and z = nz - 1). */
typedef struct lb_batch lb_batch;

/* Create a batch of nbox lattices on the current device. dims: 3*nbox ints
 * (nx, ny, nz per box, nz >= 3). rho_r, rho_b: the boxes' initial densities
 * concatenated in box order (each nx*ny*nz doubles, x fastest). params: nbox
 * parameter sets. All boxes share one precision and one stream. */
int lb_batch_create(lb_batch** out, int nbox, const int* dims, const double* rho_r, const double* rho_b,
                    const lb_params* params, int precision, void* cuda_stream);

/* Replace the parameters of box i. */
int lb_batch_set_params(lb_batch* b, int i, const lb_params* params);

/* Work split: tile height (4, 8, 16), z planes per work item, CTAs per SM of
 * the persistent grid (0 = as many as fit). Results do not depend on it. */
int lb_batch_set_schedule(lb_batch* b, int tile_y, int planes_per_item, int ctas_per_sm);

/* Choose the batch's step kernel: LB_STEP_AUTO (default) and LB_STEP_TMA take
 * the TMA-staged persistent kernel (one stage; tile heights 4 and 8, else the
 * load-from-global one), LB_STEP_LDG the load-from-global persistent kernel.
 * Both compute bit-identical results. LB_ERR_ARG for an unknown variant. */
int lb_batch_set_step_variant(lb_batch* b, int variant);

/* Advance every box by nsteps (asynchronous). LB_ERR_STATE if a box was
 * stepped on its own in between. */
int lb_batch_step(lb_batch* b, int nsteps);

/* The context of box i, borrowed: valid until lb_batch_free, usable with
 * lb_moments, lb_contact_angle, lb_save and the other readers. Do not step
 * it or free it on its own. */
int lb_batch_box(lb_batch* b, int i, lb_ctx** out);

/* Conservation sums (as lb_conservation) of every box: 8*nbox doubles. */
int lb_batch_conservation(lb_batch* b, double* cons);

/* Contact angle (as lb_contact_angle) of every box: nbox records. */
int lb_batch_contact_angles(lb_batch* b, double offset, lb_droplet* out);

/* Message of the last failure on this batch (NULL: of the last failed
 * lb_batch_create on this thread). Never NULL. */
const char* lb_batch_last_error(const lb_batch* b);

/* Release the batch, its boxes and their device memory. NULL is a no-op. */
void lb_batch_free(lb_batch* b);

/* FP64 conservation sums of a population field, for callers that cannot
 * allocate device memory. (The paper has no counterpart; this is a library
 * facility.) Some callers may not allocate at the point where they want the
 * sums: code running while its stream is being captured into a CUDA graph,
 * code inside a latency-critical or memory-budgeted section where an
 * allocation may block, fail or be forbidden by the host application's
 * allocator policy. This entry point allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine): its per-block partial sums live
 * in a fixed 64 KiB device array that the library defines at file scope.
 *   populations  device pointer, 2*19*nx*ny*nz doubles laid out as in
 *                lb_get_populations ([component][k][z][y][x]), caller-owned
 *   solid        device pointer to nx*ny*nz bytes (1 = solid, skipped), or NULL
 *   cons         device pointer to 8 doubles, caller-owned; receives
 *                {mass_r, mass_b, Px, Py, Pz, non-finite count, fluid nodes, 0}
 *   cuda_stream  stream the two kernels are queued on; the call is asynchronous
 * At most 67,108,864 nodes (the scratch holds 1024 block rows of 65,536
 * nodes each); larger lattices return LB_ERR_ARG with a message. The first
 * call on each device looks up the scratch array's device address (a
 * cudaGetSymbolAddress call), so make that first call before any stream
 * capture. Every call shares the one scratch array on a device: calls whose
 * kernels overlap on the GPU (different streams, no ordering) race and may
 * return wrong sums. Errors: LB_ERR_ARG (NULL pointer, bad or too large
 * dimensions), LB_ERR_CUDA (launch failure); message via lb_last_error(NULL). */
int lb_conservation_static(const double* populations, const uint8_t* solid, int nx, int ny, int nz,
                           double* cons, void* cuda_stream);

/* Message of the last failure on this context (or, when ctx is NULL, of the
 * last failed lb_init or context-free call on this thread). Never NULL. */
const char* lb_last_error(const lb_ctx* ctx);

/* Release the context and the device memory it owns. NULL is a no-op. */
void lb_free(lb_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBSC_H */
