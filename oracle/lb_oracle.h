/*
 * FP64 CPU oracle for the two-component Shan-Chen lattice Boltzmann step
 * (Schmieschek & Harting, "Contact angle determination in multicomponent
 * lattice Boltzmann simulations", Sec. 2-4).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may include, link or
 * call this code: only the test-suite, the smoke check and the CPU baseline
 * leg of the benchmark use it. It shares no code, header, table or constant
 * with the CUDA library; the two agree only through the paper.
 *
 * Conventions (all quantities in lattice units):
 *   - node index  idx = x + nx*(y + ny*z), all three axes periodic; walls are
 *     solid nodes given by a uint8 mask (1 = solid).
 *   - populations n[(a*19 + k)*N + idx], a = 0 ("r", droplet) or 1 ("b").
 *   - velocity ordering: k = 0 rest, 1..6 = +-x, +-y, +-z, 7..18 = the twelve
 *     diagonals in opposite pairs.
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBO_Q 19

typedef struct {
    double tau[2];      /* BGK relaxation times tau^r, tau^b (Sec. 2, collision operator) */
    double g;           /* inter-component coupling g_{r b} > 0, repulsive (Eq. SCforce) */
    double eta_wall[2]; /* wall pseudo-density: [0] acts as component r (felt by b),
                           [1] acts as component b (felt by r) (Sec. 2, wall as a species) */
    double force_scale; /* multiplier kappa on every Shan-Chen force term (1 = as printed) */
    int weights;        /* neighbour weights G_k: 0 = all 1 (as printed), 1 = 36*zeta_k */
} lbo_params;

typedef struct {
    double theta_deg;     /* geometric contact angle, Eq. geoCA with the cap relation */
    double theta_fit_deg; /* contact angle of a least-squares sphere through interface points */
    double h;             /* apex height above the wall plane */
    double b;             /* base diameter at the wall (recomputed from r and h) */
    double r;             /* sphere radius from the reference-plane base and height */
    double base_ref;      /* base diameter measured at the reference plane */
    double xc, yc, zc;    /* fitted sphere centre */
    double r_fit;         /* fitted sphere radius */
    int ok;               /* 1 when every quantity above is defined */
    int n_points;         /* interface points used by the sphere fit */
} lbo_droplet;

/* D3Q19 table: velocities, weights zeta_k, opposite index. */
void lbo_lattice(int* cx, int* cy, int* cz, double* zeta, int* opp);

/* Cubic equilibrium of Eq. Equil at density rho and velocity u. */
void lbo_equilibrium(double rho, const double* u, double* neq);

/* Populations at rest equilibrium n_k = zeta_k rho for every fluid node, 0 on solid. */
void lbo_init_equilibrium(int nx, int ny, int nz, const uint8_t* solid,
                          const double* rho_r, const double* rho_b, double* n);

/* Densities rho^a and momenta j^a = sum_k n_k c_k of every fluid node
 * (rho: 2*N, j: 2*3*N as j[(a*3 + d)*N + idx]); zero on solid nodes. */
void lbo_density(int nx, int ny, int nz, const uint8_t* solid, const double* n,
                 double* rho, double* j);

/* Shan-Chen plus wall force F^a (2*3*N) of the state n. */
void lbo_force(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
               const double* n, double* F);

/* Advance n in place by `steps` time steps. Returns 0, or -1 on a bad argument. */
int lbo_run(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
            double* n, int steps);

/* Densities, force-corrected barycentric velocity u = (sum j + F/2)/sum rho
 * (3*N, may be NULL) and conservation sums
 * cons = {M_r, M_b, Px, Py, Pz, non-finite count, fluid nodes, 0}. */
void lbo_moments(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
                 const double* n, double* rho_r, double* rho_b, double* u, double* cons);

/* Geometric contact angle of the r droplet sitting on the wall plane z = 0.5. */
int lbo_contact_angle(int nx, int ny, int nz, const uint8_t* solid,
                      const double* rho_r, const double* rho_b, double offset,
                      lbo_droplet* out);

/* The same with the interface at phi = level (Fig. 4 error bars: half max |phi|). */
int lbo_contact_angle_level(int nx, int ny, int nz, const uint8_t* solid,
                            const double* rho_r, const double* rho_b, double offset, double level,
                            lbo_droplet* out);

/* Pressure tensor of Sec. 4.1 per node: P[(c)*N + idx], c = xx, yy, zz, xy, xz, yz. */
void lbo_pressure_tensor(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
                         const double* n, double* P);

#ifdef __cplusplus
}
#endif

#endif
