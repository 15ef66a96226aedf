/*
 * gr_codeunits.c - plain FP64 CPU oracle of the constraint solve in the
 * paper's code units (Sec. 4.1) at any fiducial scale factor a.
 *
 * TEST INFRASTRUCTURE ONLY, like gr_oracle.c: the tests, the smoke check and
 * the CPU-baseline leg of the bench load it; the product path never links,
 * imports or calls it and shares no code with it.
 *
 * Code units (Sec. 4.1, box L = 1, c = 1, G = 1): H0 is the Hubble constant
 * today in units of c/L, the code-unit speed of light is ct = 1/H0, the
 * critical density rho_c = 3 H0^2 / (8 pi).  The code-unit sources are
 * st0 = s0 / (Omega_m rho_c), st_i = s_i / (Omega_m rho_c) and the trace
 * sigt = sigma / (Omega_m rho_c) of the deposit (c = 1), and the fields
 *   alpha = 1 + Phi / (a^2 ct^2),  psi = a^(1/2) (1 - Psi / (2 a^2 ct^2)),
 *   Vt_i = a ct^2 V_i,  Ut = a ct^2 U,  Bt^i = a^2 ct B^i,  bt = a^2 ct b,
 *   At_ij = ct A_ij / a.
 * orc_solve_code_units maps the code-unit guesses and sources to the
 * geometric form of Sec. 2.4 at scale factor a (homogeneous density
 * rho_hat = Omega_m rho_c a^-3), rescaled to its a = 1 form (below), solves
 * it with orc_solve_constraints and maps the solution back.  orc_code_units_residual evaluates the code-unit
 * equations as the paper prints them (Eqs. MG-linear-1a, MG-linear-1,
 * H-constraint-MG-1, CMC-MG-1 with Q-function, MG-linear-2a, MG-linear-2)
 * with the same discrete operators, so a test can hold the mapped solution
 * against the printed equations.  Readings (the paper is silent or
 * inconsistent): the trace s_m of Eqs. CMC-MG-1 and Q-function is
 * st = psi^-4 sigma / (Omega_m rho_c) = a^-2 chi^-4 sigt with
 * chi = 1 - Psi/(2 a^2 ct^2); At_ij is the Eq. Aij-discrete-2 combination of
 * Vt and Ut divided by a^2 ct, the factor the definitions above imply;
 * Omega_Lambda enters none of the printed code-unit equations (it sets a(t),
 * which the static solve takes as given).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI_CU 3.14159265358979323846

/* from gr_oracle.c */
int orc_solve_constraints(int n, const double *const *src, double *const *fld, double rho_hat, double S_hat, double tol,
                          int max_cycles, int nu1, int nu2, int *cycles, double *res0, double *res, int *status);
void orc_laplacian(int n, const double *f, double *out);
void orc_div3(int n, const double *Fx, const double *Fy, const double *Fz, double *out);
void orc_aij(int n, const double *Vx, const double *Vy, const double *Vz, const double *U, double *A);
double orc_mean(int n, const double *f);
double orc_rms(int n, const double *f);
void orc_grad(int n, int a, const double *f, double *out);

/* field order as everywhere: psi slot (Psi), alpha psi slot (Phi), V_x, V_y, V_z, U, B^x, B^y, B^z, b.
   The geometric problem at scale factor a is solved in its a = 1 form:
   with psi = a^(1/2) chi and alpha psi = a^(1/2) phi the equations of Sec.
   2.4 at a (rho_hat(a) = Omega_m rho_c a^-3, Kdot = 12 pi rho_hat(a)) are
   those at a = 1 for chi, phi, V' = V / a^2, U' = U / a^2, B' = a B,
   b' = a b with the sources s0 / a, s_i / a^2, sigma / a^3 (the trace
   s = psi^-4 sigma = a^-2 chi^-4 sigma enters as s / a) and
   rho_hat' = a^2 rho_hat(a), whose unknowns chi - 1 and phi - 1 stay small
   (a test holds this form against the direct solve at a). */
int orc_solve_code_units(int n, double a, double Om, double H0, const double *const *src_code,
                         double *const *fld_code, double tol, int max_cycles, int *cycles, double *res0, double *res,
                         int *status)
{
    const int64_t N = (int64_t)n * n * n;
    const double ct = 1.0 / H0, rho_c = 3.0 * H0 * H0 / (8.0 * PI_CU), q = Om * rho_c;
    const double a2c2 = a * a * ct * ct;
    double *buf = (double *)malloc(5 * N * sizeof(double));
    if (!buf) return 3;
    const double *src[5];
    const double sscale[5] = {q / a, q / (a * a), q / (a * a), q / (a * a), q / (a * a * a)};
    for (int k = 0; k < 5; k++) {
        double *s = buf + k * N;
        for (int64_t c = 0; c < N; c++) s[c] = sscale[k] * src_code[k][c];
        src[k] = s;
    }
    /* guesses to the a = 1 form, in place */
    for (int64_t c = 0; c < N; c++) {
        double chi = 1.0 - fld_code[0][c] / (2.0 * a2c2);
        fld_code[0][c] = chi;
        fld_code[1][c] = (1.0 + fld_code[1][c] / a2c2) * chi;
    }
    for (int f = 2; f < 10; f++) {
        double s = f < 6 ? 1.0 / (a * a * a * ct * ct) : 1.0 / (a * ct);
        for (int64_t c = 0; c < N; c++) fld_code[f][c] *= s;
    }
    int st = orc_solve_constraints(n, src, fld_code, q / a, 0.0, tol, max_cycles, 2, 2, cycles, res0, res, status);
    /* solution back to code units */
    for (int64_t c = 0; c < N; c++) {
        double chi = fld_code[0][c], phi = fld_code[1][c];
        fld_code[0][c] = 2.0 * a2c2 * (1.0 - chi);
        fld_code[1][c] = a2c2 * (phi - chi) / chi;
    }
    for (int f = 2; f < 10; f++) {
        double s = f < 6 ? a * a * a * ct * ct : a * ct;
        for (int64_t c = 0; c < N; c++) fld_code[f][c] *= s;
    }
    free(buf);
    return st;
}

/* Relative residuals RMS(eps) / RMS(right-hand side) of the ten code-unit
   equations, in solve order (V_x, V_y, V_z, U, Psi, Phi, B^x, B^y, B^z, b),
   on code-unit sources and fields. */
int orc_code_units_residual(int n, double a, double Om, double H0, const double *const *src_code,
                            const double *const *fld_code, double *rel)
{
    const int64_t N = (int64_t)n * n * n;
    const double ct = 1.0 / H0, a2c2 = a * a * ct * ct;
    double *w = (double *)malloc(14 * N * sizeof(double));
    if (!w) return 3;
    double *lap = w, *rhs = w + N, *t1 = w + 2 * N, *t2 = w + 3 * N, *A = w + 4 * N, *AA = w + 10 * N,
           *chi = w + 11 * N, *t3 = w + 12 * N, *t4 = w + 13 * N;
    const double *Psi = fld_code[0], *Phi = fld_code[1], *V[3] = {fld_code[2], fld_code[3], fld_code[4]},
                 *U = fld_code[5], *B[3] = {fld_code[6], fld_code[7], fld_code[8]}, *b = fld_code[9];
    const double *st0 = src_code[0], *sig = src_code[4];
    /* lap Vt_i = 3 Omega_m a (st_i - <st_i>) */
    for (int i = 0; i < 3; i++) {
        double m = orc_mean(n, src_code[1 + i]);
        orc_laplacian(n, V[i], lap);
        for (int64_t c = 0; c < N; c++) rhs[c] = 3.0 * Om * a * (src_code[1 + i][c] - m);
        for (int64_t c = 0; c < N; c++) t1[c] = lap[c] - rhs[c];
        rel[i] = orc_rms(n, t1) / orc_rms(n, rhs);
    }
    /* lap Ut = -1/4 div Vt ; lap bt = -1/4 div Bt */
    for (int e = 0; e < 2; e++) {
        const double *const *F = e ? B : V;
        orc_div3(n, F[0], F[1], F[2], rhs);
        for (int64_t c = 0; c < N; c++) rhs[c] *= -0.25;
        orc_laplacian(n, e ? b : U, lap);
        for (int64_t c = 0; c < N; c++) t1[c] = lap[c] - rhs[c];
        rel[e ? 9 : 3] = orc_rms(n, t1) / orc_rms(n, rhs);
    }
    /* At_ij, AtAt, chi */
    orc_aij(n, V[0], V[1], V[2], U, A);
    for (int64_t c = 0; c < 6 * N; c++) A[c] /= a * a * ct;
    for (int64_t c = 0; c < N; c++) {
        double s = 0.0;
        for (int k = 0; k < 3; k++) s += A[k * N + c] * A[k * N + c];
        for (int k = 3; k < 6; k++) s += 2.0 * A[k * N + c] * A[k * N + c];
        AA[c] = s;
        chi[c] = 1.0 - Psi[c] / (2.0 * a2c2);
    }
    /* Eq. H-constraint-MG-1: chi lap Psi = 3/2 a Om [st0 - chi^6] + AtAt/4 chi^-6 */
    orc_laplacian(n, Psi, lap);
    for (int64_t c = 0; c < N; c++) {
        double x6 = pow(chi[c], 6.0);
        rhs[c] = 1.5 * a * Om * (st0[c] - x6) + 0.25 * AA[c] / x6;
        t1[c] = chi[c] * lap[c] - rhs[c];
    }
    rel[4] = orc_rms(n, t1) / orc_rms(n, rhs);
    /* Eq. CMC-MG-1 with Eq. Q-function */
    for (int64_t c = 0; c < N; c++) t2[c] = Phi[c] * chi[c];
    orc_laplacian(n, t2, lap);
    for (int64_t c = 0; c < N; c++) {
        double x = chi[c], x6 = pow(x, 6.0), x7 = x6 * x;
        double sm = sig[c] / (a * a * x * x * x * x);
        double Q = 0.75 * a * Om / x * (st0[c] + 5.0 * x6 + 2.0 * sm) + 7.0 / 8.0 * AA[c] / x7;
        rhs[c] = Q / a2c2 * Phi[c] + 1.5 * a * Om / x * (st0[c] - x6 + sm) + AA[c] / x7;
        t1[c] = lap[c] - rhs[c];
    }
    rel[5] = orc_rms(n, t1) / orc_rms(n, rhs);
    /* Eq. MG-linear-2a: lap Bt^i = 2 d_j [(1 + Phi/a^2 ct^2) chi^-6 At^ij] */
    static const int comp[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}}; /* xx yy zz xy xz yz */
    for (int i = 0; i < 3; i++) {
        memset(rhs, 0, N * sizeof(double));
        for (int j = 0; j < 3; j++) {
            for (int64_t c = 0; c < N; c++)
                t3[c] = (1.0 + Phi[c] / a2c2) / pow(chi[c], 6.0) * A[comp[i][j] * N + c];
            orc_grad(n, j, t3, t4);
            for (int64_t c = 0; c < N; c++) rhs[c] += 2.0 * t4[c];
        }
        orc_laplacian(n, B[i], lap);
        for (int64_t c = 0; c < N; c++) t1[c] = lap[c] - rhs[c];
        rel[6 + i] = orc_rms(n, t1) / orc_rms(n, rhs);
    }
    free(w);
    return 0;
}
