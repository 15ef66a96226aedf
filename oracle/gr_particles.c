/*
 * gr_particles.c - plain FP64 CPU oracle of the particle update around the
 * constraint solve (Sec. 4.4 Eqs. geodesic-acceleration, 3-velocity, force,
 * Lorentz-factor, coeff_j, coeff_4, coeff_5; Sec. 4.5 Eqs. src_s0..src_sij;
 * App. A Eqs. GR-K1, GR-D, GR-K2, F_exp, V_exp).
 *
 * TEST INFRASTRUCTURE ONLY, like gr_oracle.c: the tests, the smoke check and
 * the CPU-baseline leg of the bench load it; the product path never links,
 * imports or calls it and shares no code with it.
 *
 * Units and geometry as in gr_oracle.c: G = c = 1, box L = 1, scale factor
 * a = 1, periodic n^3 grid, h = 1/n, cell centres (i + 1/2) h, arrays
 * [n][n][n] C-order.  With a = 1 and c = 1 the paper's code-unit potentials
 * are Phi = alpha - 1 and Psi = 2 (1 - psi), the spatial metric is
 * psi^4 delta_ij and the shift is beta^i = B^i + d_i b (Sec. 4.3.1).
 *
 * What it computes, per particle, from the solved fields psi, alpha psi, B^i, b:
 *
 *   grid    alpha = (alpha psi) / psi, beta^j = B^j + D_j b, and the central
 *           differences D_i alpha, D_i psi, D_i beta^j (3-point stencil, the
 *           paper's gradient of Sec. 4.3.1);
 *   gather  alpha, psi, beta^j and the 3 + 3 + 9 derivatives at the particle
 *           by cloud-in-cell interpolation with the deposit's weights;
 *   kick    dt/2 of du_i/dt = F_i = sum_j c_j (f_j)_i in five substeps, each
 *           taking the velocity left by the previous one:
 *             j = 1, 2, 3:  c_j = -u_j,                  (f_j)_i = -D_i beta^j
 *             j = 4:        c_4 = (W^2 - 1)/W alpha/psi,  (f_4)_i = 2 D_i psi
 *                           (-d_i Psi with Psi = 2 (1 - psi))
 *             j = 5:        c_5 = W,                     (f_5)_i = -D_i alpha
 *           with W = sqrt(1 + psi^-4 |u|^2) at the current velocity; the
 *           synchronising kick (the second kick of the previous step) runs
 *           j = 1..5, the opening kick of the step j = 5..1;
 *   drift   x^i += dt (alpha psi^-4 u_i / W - beta^i), fields at the old
 *           position, W at the kicked velocity; x wrapped into [0, 1).
 *
 * The deposit with the metric (Sec. 4.5): as orc_deposit, but the Lorentz
 * factor W = sqrt(1 + psi^-4 |u|^2) takes psi at the particle (cloud-in-cell
 * interpolation of the given psi field), and sigma = sum_l m u_l^2 / W.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int64_t pix(int n, int i, int j, int k) { return ((int64_t)i * n + j) * n + k; }
static inline int pw(int i, int n) { return ((i % n) + n) % n; }

/* cloud-in-cell cell and weights of a position: the particle lies between
   the cell centres lo and lo + 1 (periodic) along each axis; fplus is the
   weight of lo, 1 - fplus that of lo + 1 (Eqs. s0/si/sij-code-unit-cic) */
static void cic_cell(int n, const double xp[3], int lo[3], double fplus[3])
{
    const double h = 1.0 / n;
    for (int d = 0; d < 3; d++) {
        double x = xp[d] - floor(xp[d]);
        double t = x / h - 0.5;
        double fl = floor(t);
        fplus[d] = 1.0 - (t - fl);
        lo[d] = pw((int)fl, n);
    }
}

/* cloud-in-cell interpolation of nf grid arrays at a position */
static void cic_gather(int n, const int lo[3], const double fplus[3], int nf, const double *const *g, double *out)
{
    for (int q = 0; q < nf; q++) out[q] = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) {
                double w = (a ? 1.0 - fplus[0] : fplus[0]) * (b ? 1.0 - fplus[1] : fplus[1]) *
                           (c ? 1.0 - fplus[2] : fplus[2]);
                int64_t id = pix(n, (lo[0] + a) % n, (lo[1] + b) % n, (lo[2] + c) % n);
                for (int q = 0; q < nf; q++) out[q] += w * g[q][id];
            }
}

/* 3-point central difference of f along axis a into out */
static void central_diff(int n, int a, const double *f, double *out)
{
    const double i2h = 0.5 * n;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                int ip[3] = {i, j, k}, im[3] = {i, j, k};
                ip[a] = pw(ip[a] + 1, n);
                im[a] = pw(im[a] - 1, n);
                out[pix(n, i, j, k)] = (f[pix(n, ip[0], ip[1], ip[2])] - f[pix(n, im[0], im[1], im[2])]) * i2h;
            }
}

/* The interpolated quantities of one particle:
   [0] alpha, [1] psi, [2..4] beta^j, [5..7] D_i alpha, [8..10] D_i psi,
   [11 + 3 j + i] D_i beta^j. */
enum { PG_ALPHA = 0, PG_PSI = 1, PG_BETA = 2, PG_DALPHA = 5, PG_DPSI = 8, PG_DBETA = 11, PG_N = 20 };

/* Grid arrays of the 20 quantities (each n^3) from psi, alpha psi, B^i, b. */
void orc_particle_fields(int n, const double *psi, const double *apsi, const double *Bx, const double *By,
                         const double *Bz, const double *b, double *out /* 20 n^3 */)
{
    const int64_t N = (int64_t)n * n * n;
    double *g[PG_N];
    for (int q = 0; q < PG_N; q++) g[q] = out + q * N;
    const double *B[3] = {Bx, By, Bz};
    for (int64_t c = 0; c < N; c++) {
        g[PG_ALPHA][c] = apsi[c] / psi[c];
        g[PG_PSI][c] = psi[c];
    }
    for (int j = 0; j < 3; j++) {
        central_diff(n, j, b, g[PG_BETA + j]); /* D_j b */
        for (int64_t c = 0; c < N; c++) g[PG_BETA + j][c] += B[j][c];
    }
    for (int i = 0; i < 3; i++) {
        central_diff(n, i, g[PG_ALPHA], g[PG_DALPHA + i]);
        central_diff(n, i, g[PG_PSI], g[PG_DPSI + i]);
        for (int j = 0; j < 3; j++) central_diff(n, i, g[PG_BETA + j], g[PG_DBETA + 3 * j + i]);
    }
}

static double lorentz(double psi, const double u[3])
{
    double p2 = psi * psi;
    return sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (p2 * p2));
}

/* one substep j (1..5) of a kick by half_dt with the gathered quantities q */
static void substep(int j, double half_dt, const double *q, double u[3])
{
    double c, f[3];
    if (j <= 3) {
        c = -u[j - 1];
        for (int i = 0; i < 3; i++) f[i] = -q[PG_DBETA + 3 * (j - 1) + i];
    } else if (j == 4) {
        double W = lorentz(q[PG_PSI], u);
        c = (W * W - 1.0) / W * q[PG_ALPHA] / q[PG_PSI];
        for (int i = 0; i < 3; i++) f[i] = 2.0 * q[PG_DPSI + i];
    } else {
        c = lorentz(q[PG_PSI], u);
        for (int i = 0; i < 3; i++) f[i] = -q[PG_DALPHA + i];
    }
    for (int i = 0; i < 3; i++) u[i] += half_dt * c * f[i];
}

/* Particle update of np particles (x, u: [3][np] SoA, in place): with
   do_sync the synchronising kick (substeps 1..5, dt/2), with do_open the
   opening kick (substeps 5..1, dt/2), with do_drift the drift by dt; all at
   the particle's position on entry, fields from orc_particle_fields. */
void orc_particle_update(int n, int64_t np, double *x, double *u, const double *fields, double dt, int do_sync,
                         int do_open, int do_drift)
{
    const int64_t N = (int64_t)n * n * n;
    const double *g[PG_N];
    for (int q = 0; q < PG_N; q++) g[q] = fields + q * N;
    for (int64_t p = 0; p < np; p++) {
        double xp[3] = {x[p], x[np + p], x[2 * np + p]};
        double up[3] = {u[p], u[np + p], u[2 * np + p]};
        int lo[3];
        double fplus[3], q[PG_N];
        cic_cell(n, xp, lo, fplus);
        cic_gather(n, lo, fplus, PG_N, g, q);
        if (do_sync)
            for (int j = 1; j <= 5; j++) substep(j, 0.5 * dt, q, up);
        if (do_open)
            for (int j = 5; j >= 1; j--) substep(j, 0.5 * dt, q, up);
        if (do_drift) {
            double W = lorentz(q[PG_PSI], up);
            double p2 = q[PG_PSI] * q[PG_PSI];
            double fac = q[PG_ALPHA] / (p2 * p2) / W;
            for (int d = 0; d < 3; d++) {
                double xn = xp[d] + dt * (fac * up[d] - q[PG_BETA + d]);
                xp[d] = xn - floor(xn);
            }
        }
        for (int d = 0; d < 3; d++) {
            x[d * np + p] = xp[d];
            u[d * np + p] = up[d];
        }
    }
}

/* Deposit with the Lorentz factor at the given conformal factor psi
   (NULL: psi = 1, which is orc_deposit). */
void orc_deposit_metric(int n, int64_t np, const double *x, const double *u, double mass, const double *psi,
                        double *s0, double *sx, double *sy, double *sz, double *sigma)
{
    const double h = 1.0 / n, vol = h * h * h;
    const int64_t N = (int64_t)n * n * n;
    double *out[5] = {s0, sx, sy, sz, sigma};
    for (int q = 0; q < 5; q++) memset(out[q], 0, N * sizeof(double));
    for (int64_t p = 0; p < np; p++) {
        double xp[3] = {x[p], x[np + p], x[2 * np + p]};
        double up[3] = {u[p], u[np + p], u[2 * np + p]};
        int lo[3];
        double fplus[3], ps = 1.0;
        cic_cell(n, xp, lo, fplus);
        if (psi) cic_gather(n, lo, fplus, 1, &psi, &ps);
        double W = lorentz(ps, up);
        double u2 = up[0] * up[0] + up[1] * up[1] + up[2] * up[2];
        double qv[5] = {mass * W / vol, mass * up[0] / vol, mass * up[1] / vol, mass * up[2] / vol,
                        mass * u2 / W / vol};
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int c = 0; c < 2; c++) {
                    double w = (a ? 1.0 - fplus[0] : fplus[0]) * (b ? 1.0 - fplus[1] : fplus[1]) *
                               (c ? 1.0 - fplus[2] : fplus[2]);
                    int64_t id = pix(n, (lo[0] + a) % n, (lo[1] + b) % n, (lo[2] + c) % n);
                    for (int q = 0; q < 5; q++) out[q][id] += qv[q] * w;
                }
    }
}
