/*
 * FP64 CPU oracle for the two-component Shan-Chen D3Q19 lattice Boltzmann
 * step, written from Schmieschek & Harting, "Contact angle determination in
 * multicomponent lattice Boltzmann simulations" (Sec. 2 and 3, Sec. 4.1).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * CPU baseline of the benchmark, never by the product path. It is a plain,
 * slow, step-by-step restatement: one pass per stage of the method, in the
 * paper's order, every quantity in double precision.
 *
 * Readings of points the paper leaves open (the CUDA library takes the same):
 *   - "rho = sum_k eta_k" (Sec. 2) is read as rho = sum_k n_k, and "n^{r eq}"
 *     in the collision operator as n^{eq}.
 *   - D3Q19 weights zeta_k and c_s^2 are not printed; the standard values
 *     1/3, 1/18, 1/36 and c_s^2 = 1/3 are used.
 *   - the velocity in the equilibrium is the common Shan-Chen velocity
 *     u' = sum_a (j^a/tau^a) / sum_a (rho^a/tau^a), shifted per component by
 *     delta u^a = tau^a F^a / rho^a (Sec. 2, Eq. after SCforce); the shift is
 *     skipped where rho^a <= 1e-12.
 *   - the wall is an extra species (Sec. 2): a solid neighbour x' contributes
 *     the wall pseudo-density in place of psi(x') in Eq. SCforce. eta_wall[0]
 *     stands in for psi^r (felt by b), eta_wall[1] for psi^b (felt by r). The
 *     coupling is the fluid-fluid g (Sec. 4.1, Huang comparison).
 *   - Eq. SCforce sums over the 18 nearest neighbours without weights
 *     (weights = 0); weights = 1 gives G_k = 36 zeta_k. force_scale multiplies
 *     every force term.
 *   - mid-grid bounce-back (Sec. 2): a population that would stream into a
 *     solid node returns to its origin with reversed velocity.
 */
#include "lb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q LBO_Q

static const double PI = 3.14159265358979323846;

/* D3Q19: rest, six axis directions, twelve face diagonals in opposite pairs. */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static const double CS2 = 1.0 / 3.0; /* speed of sound squared */

/* zeta_k by speed: rest 1/3, axis 1/18, diagonal 1/36 */
static double zeta_of(int k)
{
    int c2 = CX[k] * CX[k] + CY[k] * CY[k] + CZ[k] * CZ[k];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* index of the velocity opposite to c_k, found by search */
static int opposite_of(int k)
{
    for (int m = 0; m < Q; ++m)
        if (CX[m] == -CX[k] && CY[m] == -CY[k] && CZ[m] == -CZ[k]) return m;
    return -1;
}

/* neighbour weight G_k of the force sum */
static double weight_of(int weights, int k)
{
    return weights == 1 ? 36.0 * zeta_of(k) : 1.0;
}

static int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static size_t node(int x, int y, int z, int nx, int ny)
{
    return (size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z);
}

void lbo_lattice(int* cx, int* cy, int* cz, double* zeta, int* opp)
{
    for (int k = 0; k < Q; ++k) {
        if (cx) cx[k] = CX[k];
        if (cy) cy[k] = CY[k];
        if (cz) cz[k] = CZ[k];
        if (zeta) zeta[k] = zeta_of(k);
        if (opp) opp[k] = opposite_of(k);
    }
}

/* Eq. Equil: n_k^eq = zeta_k rho [1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u^2/(2 cs2)
 *                                  + (c.u)^3/(6 cs2^3) - u^2 (c.u)/(2 cs2^2)] */
void lbo_equilibrium(double rho, const double* u, double* neq)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < Q; ++k) {
        double cu = CX[k] * u[0] + CY[k] * u[1] + CZ[k] * u[2];
        neq[k] = zeta_of(k) * rho *
                 (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2) +
                  cu * cu * cu / (6.0 * CS2 * CS2 * CS2) - usq * cu / (2.0 * CS2 * CS2));
    }
}

void lbo_init_equilibrium(int nx, int ny, int nz, const uint8_t* solid,
                          const double* rho_r, const double* rho_b, double* n)
{
    size_t N = (size_t)nx * ny * nz;
    const double* rho[2] = {rho_r, rho_b};
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < Q; ++k)
            for (size_t i = 0; i < N; ++i)
                n[((size_t)a * Q + k) * N + i] = solid[i] ? 0.0 : zeta_of(k) * rho[a][i];
}

/* Sec. 2: rho^a = sum_k n_k^a and rho^a u^a = sum_k n_k^a c_k */
void lbo_density(int nx, int ny, int nz, const uint8_t* solid, const double* n,
                 double* rho, double* j)
{
    size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long long ii = 0; ii < (long long)N; ++ii) {
        size_t i = (size_t)ii;
        for (int a = 0; a < 2; ++a) {
            double s = 0, sx = 0, sy = 0, sz = 0;
            if (!solid[i]) {
                for (int k = 0; k < Q; ++k) {
                    double v = n[((size_t)a * Q + k) * N + i];
                    s += v;
                    sx += v * CX[k];
                    sy += v * CY[k];
                    sz += v * CZ[k];
                }
            }
            rho[(size_t)a * N + i] = s;
            j[((size_t)a * 3 + 0) * N + i] = sx;
            j[((size_t)a * 3 + 1) * N + i] = sy;
            j[((size_t)a * 3 + 2) * N + i] = sz;
        }
    }
}

/* psi^a = 1 - exp(-rho^a) (Sec. 2, effective mass) on fluid nodes; a solid node
 * carries the wall pseudo-density in place of psi. */
static void pseudopotential(const lbo_params* p, size_t N, const uint8_t* solid,
                            const double* rho, double* psi)
{
    for (int a = 0; a < 2; ++a)
        for (size_t i = 0; i < N; ++i)
            psi[(size_t)a * N + i] = solid[i] ? p->eta_wall[a] : 1.0 - exp(-rho[(size_t)a * N + i]);
}

/* Eq. SCforce: F^a(x) = -psi^a(x) g sum_{x'} psi^{abar}(x') (x' - x), x' = x + c_k */
static void sc_force(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
                     const double* psi, double* F)
{
    size_t N = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = node(x, y, z, nx, ny);
                for (int a = 0; a < 2; ++a) {
                    int ab = 1 - a;
                    double s[3] = {0, 0, 0};
                    if (!solid[i]) {
                        for (int k = 1; k < Q; ++k) {
                            size_t ip = node(wrap(x + CX[k], nx), wrap(y + CY[k], ny),
                                             wrap(z + CZ[k], nz), nx, ny);
                            double G = weight_of(p->weights, k);
                            double ps = psi[(size_t)ab * N + ip];
                            s[0] += G * ps * CX[k];
                            s[1] += G * ps * CY[k];
                            s[2] += G * ps * CZ[k];
                        }
                    }
                    double pre = solid[i] ? 0.0 : -p->force_scale * p->g * psi[(size_t)a * N + i];
                    for (int d = 0; d < 3; ++d) F[((size_t)a * 3 + d) * N + i] = pre * s[d];
                }
            }
}

void lbo_force(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
               const double* n, double* F)
{
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 6 * N);
    double* psi = (double*)malloc(sizeof(double) * 2 * N);
    lbo_density(nx, ny, nz, solid, n, rho, j);
    pseudopotential(p, N, solid, rho, psi);
    sc_force(p, nx, ny, nz, solid, psi, F);
    free(rho);
    free(j);
    free(psi);
}

/* BGK collision with the force-shifted equilibrium velocity (Sec. 2):
 * n*_k = n_k - (n_k - n_k^eq(rho^a, u' + tau^a F^a / rho^a)) / tau^a */
static void collide(const lbo_params* p, size_t N, const uint8_t* solid, const double* n,
                    const double* rho, const double* j, const double* F, double* nstar)
{
#pragma omp parallel for schedule(static)
    for (long long ii = 0; ii < (long long)N; ++ii) {
        size_t i = (size_t)ii;
        if (solid[i]) {
            for (int a = 0; a < 2; ++a)
                for (int k = 0; k < Q; ++k) nstar[((size_t)a * Q + k) * N + i] = 0.0;
            continue;
        }
        double num[3] = {0, 0, 0}, den = 0;
        for (int a = 0; a < 2; ++a) {
            for (int d = 0; d < 3; ++d) num[d] += j[((size_t)a * 3 + d) * N + i] / p->tau[a];
            den += rho[(size_t)a * N + i] / p->tau[a];
        }
        double up[3];
        for (int d = 0; d < 3; ++d) up[d] = den > 0 ? num[d] / den : 0.0;
        for (int a = 0; a < 2; ++a) {
            double r = rho[(size_t)a * N + i];
            double ueq[3];
            for (int d = 0; d < 3; ++d)
                ueq[d] = r > 1e-12 ? up[d] + p->tau[a] * F[((size_t)a * 3 + d) * N + i] / r : up[d];
            double neq[Q];
            lbo_equilibrium(r, ueq, neq);
            for (int k = 0; k < Q; ++k) {
                double v = n[((size_t)a * Q + k) * N + i];
                nstar[((size_t)a * Q + k) * N + i] = v - (v - neq[k]) / p->tau[a];
            }
        }
    }
}

/* Eq. LBeqs streaming n_k(x + c_k, t+1) = n*_k(x, t), with mid-grid bounce-back
 * n_{kbar}(x, t+1) = n*_k(x, t) where x + c_k is solid. */
static void stream(int nx, int ny, int nz, const uint8_t* solid, const double* nstar, double* out)
{
    size_t N = (size_t)nx * ny * nz;
    memset(out, 0, sizeof(double) * 2 * Q * N);
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = node(x, y, z, nx, ny);
                if (solid[i]) continue;
                for (int k = 0; k < Q; ++k) {
                    size_t ip = node(wrap(x + CX[k], nx), wrap(y + CY[k], ny), wrap(z + CZ[k], nz), nx, ny);
                    for (int a = 0; a < 2; ++a) {
                        double v = nstar[((size_t)a * Q + k) * N + i];
                        if (solid[ip])
                            out[((size_t)a * Q + opposite_of(k)) * N + i] = v;
                        else
                            out[((size_t)a * Q + k) * N + ip] = v;
                    }
                }
            }
}

int lbo_run(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid, double* n, int steps)
{
    if (nx < 1 || ny < 1 || nz < 1 || steps < 0 || p->tau[0] <= 0.5 || p->tau[1] <= 0.5) return -1;
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 6 * N);
    double* psi = (double*)malloc(sizeof(double) * 2 * N);
    double* F = (double*)malloc(sizeof(double) * 6 * N);
    double* nstar = (double*)malloc(sizeof(double) * 2 * Q * N);
    if (!rho || !j || !psi || !F || !nstar) {
        free(rho); free(j); free(psi); free(F); free(nstar);
        return -1;
    }
    for (int t = 0; t < steps; ++t) {
        lbo_density(nx, ny, nz, solid, n, rho, j);        /* moments, Sec. 2 */
        pseudopotential(p, N, solid, rho, psi);           /* psi = 1 - exp(-rho) */
        sc_force(p, nx, ny, nz, solid, psi, F);           /* Eq. SCforce + wall */
        collide(p, N, solid, n, rho, j, F, nstar);        /* BGK, Eq. Equil */
        stream(nx, ny, nz, solid, nstar, n);              /* Eq. LBeqs + bounce-back */
    }
    free(rho); free(j); free(psi); free(F); free(nstar);
    return 0;
}

void lbo_moments(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
                 const double* n, double* rho_r, double* rho_b, double* u, double* cons)
{
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 6 * N);
    double* F = (double*)malloc(sizeof(double) * 6 * N);
    lbo_density(nx, ny, nz, solid, n, rho, j);
    lbo_force(p, nx, ny, nz, solid, n, F);
    double M[2] = {0, 0}, P[3] = {0, 0, 0}, bad = 0, fluid = 0;
    for (size_t i = 0; i < N; ++i) {
        if (rho_r) rho_r[i] = rho[i];
        if (rho_b) rho_b[i] = rho[N + i];
        double tot = rho[i] + rho[N + i];
        for (int d = 0; d < 3; ++d) {
            double m = j[(0 * 3 + d) * N + i] + j[(1 * 3 + d) * N + i];
            double f = F[(0 * 3 + d) * N + i] + F[(1 * 3 + d) * N + i];
            if (u) u[(size_t)d * N + i] = (!solid[i] && tot > 0) ? (m + 0.5 * f) / tot : 0.0;
            P[d] += m;
        }
        if (solid[i]) continue;
        fluid += 1;
        M[0] += rho[i];
        M[1] += rho[N + i];
        for (int a = 0; a < 2; ++a)
            for (int k = 0; k < Q; ++k)
                if (!isfinite(n[((size_t)a * Q + k) * N + i])) bad += 1;
    }
    if (cons) {
        cons[0] = M[0]; cons[1] = M[1];
        cons[2] = P[0]; cons[3] = P[1]; cons[4] = P[2];
        cons[5] = bad; cons[6] = fluid; cons[7] = 0;
    }
    free(rho); free(j); free(F);
}

/* length of the part of the unit segment [a, b] where the linear interpolant is > 0 */
static double positive_length(double a, double b)
{
    if (a > 0 && b > 0) return 1.0;
    if (a <= 0 && b <= 0) return 0.0;
    if (a > 0) return a / (a - b);
    return b / (b - a);
}

/* Solve the 4x4 system M s = v by Gaussian elimination with partial pivoting. */
static int solve4(double M[4][4], double v[4], double s[4])
{
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (fabs(M[piv][c]) < 1e-300) return -1;
        if (piv != c) {
            for (int k = 0; k < 4; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
            double t = v[c]; v[c] = v[piv]; v[piv] = t;
        }
        for (int r = c + 1; r < 4; ++r) {
            double f = M[r][c] / M[c][c];
            for (int k = c; k < 4; ++k) M[r][k] -= f * M[c][k];
            v[r] -= f * v[c];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double acc = v[r];
        for (int k = r + 1; k < 4; ++k) acc -= M[r][k] * s[k];
        s[r] = acc / M[r][r];
    }
    return 0;
}

/* Sec. 3: geometric contact angle of the r droplet on the wall plane z = 0.5.
 * The interface is phi = rho_r - rho_b = 0 (Sec. 2), located by linear
 * interpolation between nodes. h is the highest crossing above the wall; the
 * base b' is the diameter of the circle with the area of {phi > 0} at the
 * reference plane `offset` above the wall. From the cap above that plane the
 * sphere radius follows (r = (4h^2 + b^2)/(8h) written for the cap of height
 * h' = h - offset and base b'); the base at the wall follows from r and h, and
 * theta from Eq. geoCA read as theta = atan2(b/2, r - h). */
int lbo_contact_angle(int nx, int ny, int nz, const uint8_t* solid,
                      const double* rho_r, const double* rho_b, double offset,
                      lbo_droplet* out)
{
    return lbo_contact_angle_level(nx, ny, nz, solid, rho_r, rho_b, offset, 0.0, out);
}

/* As above with the interface taken at phi = level instead of phi = 0
 * (Fig. 4's error bars use half the maximum |phi|). */
int lbo_contact_angle_level(int nx, int ny, int nz, const uint8_t* solid,
                            const double* rho_r, const double* rho_b, double offset, double level,
                            lbo_droplet* out)
{
    memset(out, 0, sizeof(*out));
    const double zw = 0.5;
    size_t N = (size_t)nx * ny * nz;
    double* phi = (double*)malloc(sizeof(double) * N);
    for (size_t i = 0; i < N; ++i) phi[i] = solid[i] ? 0.0 : rho_r[i] - rho_b[i] - level;

    /* apex: highest phi = 0 crossing from phi > 0 below to phi <= 0 above */
    double top = -1e300;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int z = 0; z + 1 < nz; ++z) {
                size_t i0 = node(x, y, z, nx, ny), i1 = node(x, y, z + 1, nx, ny);
                if (solid[i0] || solid[i1]) continue;
                if (phi[i0] > 0 && phi[i1] <= 0) {
                    double zc = z + phi[i0] / (phi[i0] - phi[i1]);
                    if (zc > top) top = zc;
                }
            }
    double h = top - zw;

    /* base at the reference plane, area of the linear interpolant's positive part along x */
    double zref = zw + offset;
    int z0 = (int)floor(zref);
    double f = zref - z0;
    double area = 0.0;
    int plane_ok = (z0 >= 0 && z0 + 1 < nz);
    if (plane_ok) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int x1 = (x + 1) % nx;
                double a0 = (1 - f) * phi[node(x, y, z0, nx, ny)] + f * phi[node(x, y, z0 + 1, nx, ny)];
                double a1 = (1 - f) * phi[node(x1, y, z0, nx, ny)] + f * phi[node(x1, y, z0 + 1, nx, ny)];
                area += positive_length(a0, a1);
            }
    }
    double bref = 2.0 * sqrt(area / PI);
    double hp = h - offset;
    out->h = h;
    out->base_ref = bref;
    if (top > -1e299 && plane_ok && hp > 0 && bref > 0) {
        double r = (0.25 * bref * bref + hp * hp) / (2.0 * hp);
        double arg = r * r - (r - h) * (r - h);
        double b = 2.0 * sqrt(arg > 0 ? arg : 0.0);
        out->r = r;
        out->b = b;
        out->theta_deg = atan2(0.5 * b, r - h) * 180.0 / PI;
        out->ok = 1;
    }

    /* least-squares sphere x^2+y^2+z^2 = 2 a.x + d through interface points above the plane */
    double M[4][4] = {{0}}, v[4] = {0};
    int npts = 0;
    const int dirs[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i0 = node(x, y, z, nx, ny);
                if (solid[i0]) continue;
                for (int d = 0; d < 3; ++d) {
                    int x1 = x + dirs[d][0], y1 = y + dirs[d][1], z1 = z + dirs[d][2];
                    if (x1 >= nx || y1 >= ny || z1 >= nz) continue;
                    size_t i1 = node(x1, y1, z1, nx, ny);
                    if (solid[i1]) continue;
                    if ((phi[i0] > 0) == (phi[i1] > 0)) continue;
                    double t = phi[i0] / (phi[i0] - phi[i1]);
                    double px = x + t * dirs[d][0], py = y + t * dirs[d][1], pz = z + t * dirs[d][2];
                    if (pz < zref) continue;
                    double row[4] = {2 * px, 2 * py, 2 * pz, 1.0};
                    double rhs = px * px + py * py + pz * pz;
                    for (int r = 0; r < 4; ++r) {
                        for (int c = 0; c < 4; ++c) M[r][c] += row[r] * row[c];
                        v[r] += row[r] * rhs;
                    }
                    ++npts;
                }
            }
    out->n_points = npts;
    double s[4];
    if (npts >= 4 && solve4(M, v, s) == 0) {
        double R2 = s[3] + s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
        if (R2 > 0) {
            double R = sqrt(R2);
            double c = -(s[2] - zw) / R;
            if (c > 1) c = 1;
            if (c < -1) c = -1;
            out->xc = s[0];
            out->yc = s[1];
            out->zc = s[2];
            out->r_fit = R;
            out->theta_fit_deg = acos(c) * 180.0 / PI;
        }
    }
    free(phi);
    return out->ok ? 0 : -1;
}

/* Sec. 4.1 pressure tensor:
 * P_ij = sum_a sum_k (c_ki - u_i)(c_kj - u_j) n_k^a
 *      + 1/4 sum_{a, abar} g sum_{x'} [psi^a(x) psi^abar(x') + psi^abar(x) psi^a(x')] (x - x')_i (x - x')_j
 * with (x - x')^2 read as the outer product, the same neighbour weights and
 * force scale as the force, and u the velocity reported by lbo_moments. */
void lbo_pressure_tensor(const lbo_params* p, int nx, int ny, int nz, const uint8_t* solid,
                         const double* n, double* P)
{
    size_t N = (size_t)nx * ny * nz;
    double* rho = (double*)malloc(sizeof(double) * 2 * N);
    double* j = (double*)malloc(sizeof(double) * 6 * N);
    double* psi = (double*)malloc(sizeof(double) * 2 * N);
    double* u = (double*)malloc(sizeof(double) * 3 * N);
    lbo_density(nx, ny, nz, solid, n, rho, j);
    pseudopotential(p, N, solid, rho, psi);
    lbo_moments(p, nx, ny, nz, solid, n, NULL, NULL, u, NULL);
    const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t i = node(x, y, z, nx, ny);
                for (int c = 0; c < 6; ++c) {
                    double acc = 0;
                    if (!solid[i]) {
                        double ui[3] = {u[i], u[N + i], u[2 * N + i]};
                        for (int a = 0; a < 2; ++a)
                            for (int k = 0; k < Q; ++k) {
                                int cc[3] = {CX[k], CY[k], CZ[k]};
                                acc += (cc[I[c]] - ui[I[c]]) * (cc[J[c]] - ui[J[c]]) *
                                       n[((size_t)a * Q + k) * N + i];
                            }
                        for (int a = 0; a < 2; ++a) {
                            int ab = 1 - a;
                            for (int k = 1; k < Q; ++k) {
                                int cc[3] = {CX[k], CY[k], CZ[k]};
                                size_t ip = node(wrap(x + CX[k], nx), wrap(y + CY[k], ny),
                                                 wrap(z + CZ[k], nz), nx, ny);
                                double pair = psi[(size_t)a * N + i] * psi[(size_t)ab * N + ip] +
                                              psi[(size_t)ab * N + i] * psi[(size_t)a * N + ip];
                                acc += 0.25 * p->force_scale * p->g * weight_of(p->weights, k) * pair *
                                       cc[I[c]] * cc[J[c]];
                            }
                        }
                    }
                    P[(size_t)c * N + i] = acc;
                }
            }
    free(rho); free(j); free(psi); free(u);
}
