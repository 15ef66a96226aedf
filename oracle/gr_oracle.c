/*
 * gr_oracle.c - plain FP64 CPU oracle of the constrained-GR elliptic solve.
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline
 * leg of the bench load this file's shared library; the product path (the
 * CUDA library and its Python binding) never links, imports or calls it, and
 * shares no code with it.
 *
 * What it computes (geometric units G = c = 1, box L = 1, periodic n^3 grid,
 * h = 1/n, cell centres x_i = (i + 1/2) h, arrays [n][n][n] C-order with
 * index (i*n + j)*n + k, i the x index):
 *
 *   deposit   cloud-in-cell sources s0, s_l, sigma = sum_l s_ll (Sec. 4.1.2,
 *             Eqs. s0/si/sij-code-unit-cic, with psi = 1 in the Lorentz factor)
 *   V_i       lap V_i = 8 pi (s_i - <s_i>)                (Eq. MG-linear-1a)
 *   U         lap U = -1/4 div V                          (Eq. MG-linear-1)
 *   A_ij, AA  A_ij = d_i V_j + d_j V_i - 1/2 d_ij div V + 2 d_i d_j U
 *                                             (Eqs. Aij-discrete-2, U-cross-deriv)
 *   psi       lap psi = -2 pi s0 / psi - AA / (8 psi^7) + 2 pi rho psi^5
 *                                             (Eq. sol-scheme-H-constraint)
 *   alpha psi lap(alpha psi) = m (alpha psi) - psi^5 Kdot   (Eq. sol-scheme-CMC)
 *             m = 2 pi psi^-2 (s0 + 2 psi^-4 sigma) + 7/8 psi^-8 AA + 5/12 psi^4 K^2
 *   B^i       lap B^i = 2 d_j (alpha psi^-6 A^ij)         (Eqs. MDC-CF, MG-linear-2a)
 *   b         lap b = -1/4 div B                          (Eq. MG-linear-2)
 *
 * Discretisation (Sec. 4.3.1): 7-point Laplacian, 3-point central
 * differences, 4-point cross derivative, 3-point second difference for the
 * diagonal d_i d_i U.  Solver (Sec. 4.3): red-black Gauss-Seidel V(nu1, nu2)
 * cycles over every level n, n/2, ..., 2 (Sec. 4.3.1, last paragraph).  The
 * linear equations use the coarse-grid correction form (Eq. GR-linear-coarse);
 * the psi equation uses the full approximation scheme (Sec. 4.3.2.1) with one
 * Newton step per cell visit.  Restriction R is the 8-child average and
 * prolongation P the cell-centred trilinear interpolation (weights 3/4, 1/4
 * per axis); the paper names R and P without giving them.
 *
 * Background scalars: K^2 = 24 pi rho_hat, Kdot = 12 pi rho_hat + 4 pi S_hat
 * (Eqs. 1-Friedmann, 2-Friedmann with rho_Lambda = 0).
 *
 * Static nested refinement patches (the last part of this file): the same
 * equations on a chain of cubic patches, each refining its parent by 2,
 * coupled to the base by composite-grid FAS with flux matching.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

enum { ORC_POISSON = 0, ORC_HELMHOLTZ = 1, ORC_PSI = 2 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NOMEM = 3, ORC_ERR_NOCONV = 4, ORC_ERR_NONFINITE = 5 };

/* sweeps on the 2^3 level: red-black GS on the 8-cell periodic Laplacian
   contracts by 1/9 per sweep, so 32 sweeps reach rounding */
#define COARSEST_SWEEPS 32

static inline int64_t ix(int n, int i, int j, int k) { return ((int64_t)i * n + j) * n + k; }
static inline int up(int i, int n) { return i + 1 == n ? 0 : i + 1; }
static inline int dn(int i, int n) { return i == 0 ? n - 1 : i - 1; }
static inline int64_t cells(int n) { return (int64_t)n * n * n; }

/* ------------------------------------------------------------------ */
/* Cloud-in-cell deposit (Sec. 4.1.2, Eqs. s0/si/sij-code-unit-cic)    */
/* ------------------------------------------------------------------ */

/* The particle at x_p lies between the cell centres x_i <= x_p < x_{i+1};
   f+ = (x_{i+1} - x_p)/h goes to cell i and f- = 1 - f+ to cell i+1.  Each
   particle adds m W w / h^3 to s0, m u_l w / h^3 to s_l and
   m |u|^2 / W w / h^3 to sigma, with W = sqrt(1 + |u|^2) (psi = 1). */
void orc_deposit(int n, int64_t np, const double *x, const double *u, double mass,
                 double *s0, double *sx, double *sy, double *sz, double *sigma)
{
    const double h = 1.0 / n, vol = h * h * h;
    const int64_t N = cells(n);
    memset(s0, 0, N * sizeof(double));
    memset(sx, 0, N * sizeof(double));
    memset(sy, 0, N * sizeof(double));
    memset(sz, 0, N * sizeof(double));
    memset(sigma, 0, N * sizeof(double));
    for (int64_t p = 0; p < np; p++) {
        int lo[3];
        double fplus[3];
        for (int d = 0; d < 3; d++) {
            double xp = x[d * np + p];
            xp -= floor(xp); /* periodic box [0, 1) */
            double t = xp / h - 0.5;     /* position in units of h from centre 0 */
            double fl = floor(t);
            fplus[d] = 1.0 - (t - fl);   /* (x_{i+1} - x_p) / h */
            int i = (int)fl;
            lo[d] = (i % n + n) % n;
        }
        double ux = u[p], uy = u[np + p], uz = u[2 * np + p];
        double u2 = ux * ux + uy * uy + uz * uz;
        double W = sqrt(1.0 + u2);
        double q0 = mass * W / vol, qx = mass * ux / vol, qy = mass * uy / vol, qz = mass * uz / vol;
        double qs = mass * u2 / W / vol;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int c = 0; c < 2; c++) {
                    double w = (a ? 1.0 - fplus[0] : fplus[0]) * (b ? 1.0 - fplus[1] : fplus[1]) *
                               (c ? 1.0 - fplus[2] : fplus[2]);
                    int64_t id = ix(n, (lo[0] + a) % n, (lo[1] + b) % n, (lo[2] + c) % n);
                    s0[id] += q0 * w;
                    sx[id] += qx * w;
                    sy[id] += qy * w;
                    sz[id] += qz * w;
                    sigma[id] += qs * w;
                }
    }
}

/* ------------------------------------------------------------------ */
/* Finite-difference operators (Sec. 4.3.1)                            */
/* ------------------------------------------------------------------ */

double orc_mean(int n, const double *f)
{
    double s = 0.0;
    for (int64_t c = 0; c < cells(n); c++) s += f[c];
    return s / (double)cells(n);
}

double orc_rms(int n, const double *f)
{
    double s = 0.0;
    for (int64_t c = 0; c < cells(n); c++) s += f[c] * f[c];
    return sqrt(s / (double)cells(n));
}

/* 7-point Laplacian */
void orc_laplacian(int n, const double *f, double *out)
{
    const double ih2 = (double)n * n;
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                double nb = f[ix(n, up(i, n), j, k)] + f[ix(n, dn(i, n), j, k)] + f[ix(n, i, up(j, n), k)] +
                            f[ix(n, i, dn(j, n), k)] + f[ix(n, i, j, up(k, n))] + f[ix(n, i, j, dn(k, n))];
                out[ix(n, i, j, k)] = (nb - 6.0 * f[ix(n, i, j, k)]) * ih2;
            }
}

/* value of f at (i, j, k) shifted by s cells along axis a */
static inline double at(const double *f, int n, int i, int j, int k, int a, int s)
{
    int c[3] = {i, j, k};
    c[a] = ((c[a] + s) % n + n) % n;
    return f[ix(n, c[0], c[1], c[2])];
}

/* central first derivative along axis a: (f_{+a} - f_{-a}) / 2h */
void orc_grad(int n, int a, const double *f, double *out)
{
    const double i2h = 0.5 * n;
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++)
                out[ix(n, i, j, k)] = (at(f, n, i, j, k, a, 1) - at(f, n, i, j, k, a, -1)) * i2h;
}

/* 3-point divergence  sum_l (F^l_{+l} - F^l_{-l}) / 2h */
void orc_div3(int n, const double *Fx, const double *Fy, const double *Fz, double *out)
{
    const double i2h = 0.5 * n;
    const double *F[3] = {Fx, Fy, Fz};
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                double s = 0.0;
                for (int a = 0; a < 3; a++) s += at(F[a], n, i, j, k, a, 1) - at(F[a], n, i, j, k, a, -1);
                out[ix(n, i, j, k)] = s * i2h;
            }
}

/* The six independent components of A_ij (Eq. Aij-discrete-2), stored as
   xx, yy, zz, xy, xz, yz (each n^3).  Diagonal: 2 D_i V_i - 1/2 div V
   + 2 D_ii U with the 3-point second difference; off-diagonal:
   D_i V_j + D_j V_i + 2 D_ij U with the 4-cell cross derivative
   (Eq. U-cross-deriv). */
void orc_aij(int n, const double *Vx, const double *Vy, const double *Vz, const double *U, double *A)
{
    const double i2h = 0.5 * n, ih2 = (double)n * n;
    const double *V[3] = {Vx, Vy, Vz};
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    const int64_t N = cells(n);
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                double D[3][3]; /* D[a][l] = D_a V_l */
                for (int a = 0; a < 3; a++)
                    for (int l = 0; l < 3; l++)
                        D[a][l] = (at(V[l], n, i, j, k, a, 1) - at(V[l], n, i, j, k, a, -1)) * i2h;
                double divV = D[0][0] + D[1][1] + D[2][2];
                double u0 = U[ix(n, i, j, k)];
                for (int a = 0; a < 3; a++) {
                    double Uaa = (at(U, n, i, j, k, a, 1) - 2.0 * u0 + at(U, n, i, j, k, a, -1)) * ih2;
                    A[a * N + ix(n, i, j, k)] = 2.0 * D[a][a] - 0.5 * divV + 2.0 * Uaa;
                }
                for (int p = 0; p < 3; p++) {
                    int a = pa[p], b = pb[p];
                    int c[3];
                    double s = 0.0;
                    for (int sa = -1; sa <= 1; sa += 2)
                        for (int sb = -1; sb <= 1; sb += 2) {
                            c[0] = i; c[1] = j; c[2] = k;
                            c[a] = (c[a] + sa + n) % n;
                            c[b] = (c[b] + sb + n) % n;
                            s += (double)(sa * sb) * U[ix(n, c[0], c[1], c[2])];
                        }
                    double Uab = s * 0.25 * ih2;
                    A[(3 + p) * N + ix(n, i, j, k)] = D[a][b] + D[b][a] + 2.0 * Uab;
                }
            }
}

/* AA = A_ij A^ij with indices moved by delta_ij (conformal flatness, Eq. FCF-approx) */
void orc_aa(int n, const double *A, double *aa)
{
    const int64_t N = cells(n);
    for (int64_t c = 0; c < N; c++) {
        double d = A[c] * A[c] + A[N + c] * A[N + c] + A[2 * N + c] * A[2 * N + c];
        double o = A[3 * N + c] * A[3 * N + c] + A[4 * N + c] * A[4 * N + c] + A[5 * N + c] * A[5 * N + c];
        aa[c] = d + 2.0 * o;
    }
}

/* Coefficient and right-hand side of the lapse equation for phi = alpha psi
   (Eq. sol-scheme-CMC with rho_Lambda = 0, s = gamma^ij s_ij = psi^-4 sigma):
     lap phi - m phi = -psi^5 Kdot  */
void orc_lapse_coef(int n, const double *psi, const double *s0, const double *sigma, const double *aa, double K2,
                    double Kdot, double *m, double *f)
{
    for (int64_t c = 0; c < cells(n); c++) {
        double p = psi[c], p2 = p * p, p4 = p2 * p2, p8 = p4 * p4;
        m[c] = 2.0 * PI / p2 * (s0[c] + 2.0 * sigma[c] / p4) + 0.875 * aa[c] / p8 + (5.0 / 12.0) * p4 * K2;
        f[c] = -p4 * p * Kdot;
    }
}

/* Source of the B^i equations (Eqs. MG-linear-2a, Aij-discrete):
   S^i = 2 sum_j (A'^{ij}_{+j} - A'^{ij}_{-j}) / 2h,  A' = alpha psi^-6 A = phi psi^-7 A */
void orc_shift_source(int n, const double *A, const double *psi, const double *apsi, double *SB)
{
    const int64_t N = cells(n);
    const double i2h = 0.5 * n;
    double *Ap = (double *)malloc(6 * N * sizeof(double));
    if (!Ap) return;
    for (int64_t c = 0; c < N; c++) {
        double p = psi[c], p2 = p * p, p4 = p2 * p2;
        double w = apsi[c] / (p4 * p2 * p);
        for (int q = 0; q < 6; q++) Ap[q * N + c] = w * A[q * N + c];
    }
    /* component index of A'^{ij} in the xx, yy, zz, xy, xz, yz storage */
    const int comp[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++)
                for (int a = 0; a < 3; a++) {
                    double s = 0.0;
                    for (int l = 0; l < 3; l++) {
                        const double *F = Ap + comp[a][l] * N;
                        s += at(F, n, i, j, k, l, 1) - at(F, n, i, j, k, l, -1);
                    }
                    SB[a * N + ix(n, i, j, k)] = 2.0 * s * i2h;
                }
    free(Ap);
}

/* ------------------------------------------------------------------ */
/* Multigrid (Sec. 4.3)                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    int n;
    double *u, *f, *c0, *c1, *ur, *tmp; /* ur = R u of the finer level (FAS) */
    int own_u, own_c;
} level_t;

typedef struct {
    int kind, nlev, nu1, nu2;
    double rho;     /* rho_hat in the psi operator */
    level_t *lev;   /* lev[nlev-1] is the finest */
} hier_t;

/* Pointwise operator L(u) at one cell given the neighbour sum nb.
   Poisson: lap u.  Helmholtz: lap u - c0 u.  psi: the unknown is the
   deviation u = psi - 1 from the homogeneous background (the paper's Psi
   variable, Sec. 4.1.1, measures the same deviation), so that the Laplacian
   acts on a small field:
     L(u) = lap u + 2 pi s0 / psi + AA / (8 psi^7) - 2 pi rho_hat psi^5,
   psi = 1 + u, c0 = s0, c1 = AA. */
static inline double op_point(int kind, double u, double nb, double ih2, double c0, double c1, double rho)
{
    double lap = (nb - 6.0 * u) * ih2;
    if (kind == ORC_POISSON) return lap;
    if (kind == ORC_HELMHOLTZ) return lap - c0 * u;
    double v = 1.0 + u, v2 = v * v, v4 = v2 * v2;
    return lap + 2.0 * PI * c0 / v + c1 / (8.0 * v4 * v2 * v) - 2.0 * PI * rho * v4 * v;
}

static inline double nbsum(const double *u, int n, int i, int j, int k)
{
    return u[ix(n, up(i, n), j, k)] + u[ix(n, dn(i, n), j, k)] + u[ix(n, i, up(j, n), k)] +
           u[ix(n, i, dn(j, n), k)] + u[ix(n, i, j, up(k, n))] + u[ix(n, i, j, dn(k, n))];
}

/* one Gauss-Seidel pass over the cells of one colour ((i+j+k) % 2 == color) */
static void gs_colour(const hier_t *H, level_t *L, int color)
{
    const int n = L->n;
    const double h2 = 1.0 / ((double)n * n), ih2 = (double)n * n;
    double *u = L->u;
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = (i + j + color) & 1; k < n; k += 2) {
                int64_t c = ix(n, i, j, k);
                double nb = nbsum(u, n, i, j, k);
                if (H->kind == ORC_POISSON) {
                    u[c] = (nb - h2 * L->f[c]) / 6.0;
                } else if (H->kind == ORC_HELMHOLTZ) {
                    u[c] = (nb - h2 * L->f[c]) / (6.0 + h2 * L->c0[c]);
                } else {
                    /* one Newton step on g(u) = L(u) - f, psi = 1 + u */
                    double v = 1.0 + u[c], v2 = v * v, v4 = v2 * v2;
                    double g = op_point(ORC_PSI, u[c], nb, ih2, L->c0[c], L->c1[c], H->rho) - L->f[c];
                    double dg = -6.0 * ih2 - 2.0 * PI * L->c0[c] / v2 - 7.0 * L->c1[c] / (8.0 * v4 * v4) -
                                10.0 * PI * H->rho * v4;
                    u[c] -= g / dg;
                }
            }
}

static void sweep(const hier_t *H, level_t *L)
{
    gs_colour(H, L, 0); /* red */
    gs_colour(H, L, 1); /* black */
}

/* eps = L(u) - f (Eqs. epsilon-error-lin, epsilon-error-nonlin-1) */
static void residual(const hier_t *H, const level_t *L, double *eps)
{
    const int n = L->n;
    const double ih2 = (double)n * n;
#pragma omp parallel for
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                int64_t c = ix(n, i, j, k);
                double c0 = L->c0 ? L->c0[c] : 0.0, c1 = L->c1 ? L->c1[c] : 0.0;
                eps[c] = op_point(H->kind, L->u[c], nbsum(L->u, n, i, j, k), ih2, c0, c1, H->rho) - L->f[c];
            }
}

/* R: average of the 8 children */
static void restrict8(int nf, const double *fine, double *coarse)
{
    const int nc = nf / 2;
#pragma omp parallel for
    for (int I = 0; I < nc; I++)
        for (int J = 0; J < nc; J++)
            for (int K = 0; K < nc; K++) {
                double s = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int c = 0; c < 2; c++) s += fine[ix(nf, 2 * I + a, 2 * J + b, 2 * K + c)];
                coarse[ix(nc, I, J, K)] = 0.125 * s;
            }
}

/* P: fine += trilinear interpolation of the coarse field e; the fine cell
   2I + a takes 3/4 of coarse cell I and 1/4 of cell I - 1 (a = 0) or I + 1
   (a = 1) along each axis */
static void prolong_add(int nf, const double *e, double *fine)
{
    const int nc = nf / 2;
#pragma omp parallel for
    for (int i = 0; i < nf; i++)
        for (int j = 0; j < nf; j++)
            for (int k = 0; k < nf; k++) {
                int I[2], J[2], K[2];
                I[0] = i / 2; I[1] = (i & 1) ? up(I[0], nc) : dn(I[0], nc);
                J[0] = j / 2; J[1] = (j & 1) ? up(J[0], nc) : dn(J[0], nc);
                K[0] = k / 2; K[1] = (k & 1) ? up(K[0], nc) : dn(K[0], nc);
                const double w[2] = {0.75, 0.25};
                double s = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int c = 0; c < 2; c++) s += w[a] * w[b] * w[c] * e[ix(nc, I[a], J[b], K[c])];
                fine[ix(nf, i, j, k)] += s;
            }
}

static void subtract_mean(int n, double *f)
{
    double m = orc_mean(n, f);
    for (int64_t c = 0; c < cells(n); c++) f[c] -= m;
}

/* The uniform part of the 2^3 level's error.  The Laplacian annihilates a
   constant, so a red-black sweep damps the constant error mode of the
   Helmholtz and psi equations only by 1/(1 + h^2 m / 6) per sweep, m the
   equation's non-Laplacian coefficient (m = c0; psi: 2 pi s0 / psi^2 +
   7 AA / (8 psi^8) + 10 pi rho psi^4): slow where m is small (a weak
   background, e.g. a small Hubble rate in code units).  After each sweep
   the level therefore takes the constant shift that zeroes the sum of its
   residuals to first order, u -= sum(f - L(u)) / sum(m). */
static void zero_mode(const hier_t *H, level_t *L)
{
    const int n = L->n;
    const double ih2 = (double)n * n;
    double sr = 0.0, sm = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                int64_t c = ix(n, i, j, k);
                double u = L->u[c];
                sr += L->f[c] - op_point(H->kind, u, nbsum(L->u, n, i, j, k), ih2, L->c0[c], L->c1 ? L->c1[c] : 0.0,
                                         H->rho);
                if (H->kind == ORC_HELMHOLTZ) {
                    sm += L->c0[c];
                } else {
                    double v = 1.0 + u, v2 = v * v, v4 = v2 * v2;
                    sm += 2.0 * PI * L->c0[c] / v2 + 7.0 * L->c1[c] / (8.0 * v4 * v4) + 10.0 * PI * H->rho * v4;
                }
            }
    if (!(sm > 0.0)) return;
    const double shift = -sr / sm; /* L(u + c) = L(u) - m c to first order */
    for (int64_t c = 0; c < cells(n); c++) L->u[c] += shift;
}

/* The 2^3 level (Sec. 4.3.1, last paragraph): COARSEST_SWEEPS red-black
   sweeps, each followed (Helmholtz, psi) by the zero-mode shift above;
   Poisson: source mean removed before and solution mean after. */
static void coarsest(const hier_t *H, level_t *L)
{
    if (H->kind == ORC_POISSON) subtract_mean(L->n, L->f);
    for (int s = 0; s < COARSEST_SWEEPS; s++) {
        sweep(H, L);
        if (H->kind != ORC_POISSON) zero_mode(H, L);
    }
    if (H->kind == ORC_POISSON) subtract_mean(L->n, L->u);
}

static void vcycle_level(const hier_t *H, int l)
{
    level_t *A = &H->lev[l];
    if (l == 0) {
        coarsest(H, A);
        return;
    }
    level_t *C = &H->lev[l - 1];
    const int nc = C->n;
    const int64_t Nc = cells(nc);
    for (int s = 0; s < H->nu1; s++) sweep(H, A);
    residual(H, A, A->tmp);
    restrict8(A->n, A->tmp, C->f); /* R eps */
    if (H->kind == ORC_PSI) {
        /* FAS: u^H = R u^h and f^H = L^H(R u^h) - R eps^h  (Sec. 4.3.2.1) */
        restrict8(A->n, A->u, C->u);
        memcpy(C->ur, C->u, Nc * sizeof(double));
        const double ih2 = (double)nc * nc;
        for (int i = 0; i < nc; i++)
            for (int j = 0; j < nc; j++)
                for (int k = 0; k < nc; k++) {
                    int64_t c = ix(nc, i, j, k);
                    C->f[c] = op_point(ORC_PSI, C->u[c], nbsum(C->u, nc, i, j, k), ih2, C->c0[c], C->c1[c], H->rho) -
                              C->f[c];
                }
    } else {
        /* correction form L^H(du^H) = -R eps^h, du^H = 0 initially (Eq. GR-linear-coarse) */
        for (int64_t c = 0; c < Nc; c++) {
            C->f[c] = -C->f[c];
            C->u[c] = 0.0;
        }
    }
    vcycle_level(H, l - 1);
    if (H->kind == ORC_PSI) {
        for (int64_t c = 0; c < Nc; c++) C->tmp[c] = C->u[c] - C->ur[c];
        prolong_add(A->n, C->tmp, A->u);
    } else {
        prolong_add(A->n, C->u, A->u);
    }
    for (int s = 0; s < H->nu2; s++) sweep(H, A);
}

static int log2i(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return l;
}

static int valid_n(int n) { return n >= 4 && n <= 4096 && (n & (n - 1)) == 0; }

static void hier_free(hier_t *H)
{
    if (!H->lev) return;
    for (int l = 0; l < H->nlev; l++) {
        level_t *L = &H->lev[l];
        if (L->own_u) free(L->u);
        free(L->f);
        if (L->own_c) {
            free(L->c0);
            free(L->c1);
        }
        free(L->ur);
        free(L->tmp);
    }
    free(H->lev);
    H->lev = NULL;
}

/* Build the level hierarchy n -> 2.  The finest level uses the caller's u
   and coefficient arrays and a private copy of f; coarse coefficients are the
   restriction of the fine ones, restricted once per hierarchy. */
static int hier_build(hier_t *H, int kind, int n, double *u, const double *f, const double *c0, const double *c1,
                      double rho, int nu1, int nu2)
{
    H->kind = kind;
    H->nu1 = nu1;
    H->nu2 = nu2;
    H->rho = rho;
    H->nlev = log2i(n); /* levels n, n/2, ..., 2 */
    H->lev = (level_t *)calloc(H->nlev, sizeof(level_t));
    if (!H->lev) return ORC_ERR_NOMEM;
    for (int l = H->nlev - 1; l >= 0; l--) {
        level_t *L = &H->lev[l];
        L->n = 2 << l;
        int64_t N = cells(L->n);
        int fine = (l == H->nlev - 1);
        L->f = (double *)malloc(N * sizeof(double));
        L->ur = (double *)malloc(N * sizeof(double));
        L->tmp = (double *)malloc(N * sizeof(double));
        if (!L->f || !L->ur || !L->tmp) return ORC_ERR_NOMEM;
        if (fine) {
            L->u = u;
            memcpy(L->f, f, N * sizeof(double));
            L->c0 = (double *)c0;
            L->c1 = (double *)c1;
        } else {
            L->own_u = 1;
            L->u = (double *)calloc(N, sizeof(double));
            if (!L->u) return ORC_ERR_NOMEM;
            if (kind != ORC_POISSON) {
                level_t *F = &H->lev[l + 1];
                L->own_c = 1;
                L->c0 = (double *)malloc(N * sizeof(double));
                if (!L->c0) return ORC_ERR_NOMEM;
                restrict8(F->n, F->c0, L->c0);
                if (kind == ORC_PSI) {
                    L->c1 = (double *)malloc(N * sizeof(double));
                    if (!L->c1) return ORC_ERR_NOMEM;
                    restrict8(F->n, F->c1, L->c1);
                }
            }
        }
    }
    return ORC_OK;
}

/* RMS of eps = L(u) - f on one grid; eps_out may be NULL */
double orc_residual(int kind, int n, const double *u, const double *f, const double *c0, const double *c1, double rho,
                    double *eps_out)
{
    hier_t H = {kind, 1, 0, 0, rho, NULL};
    level_t L = {n, (double *)u, (double *)f, (double *)c0, (double *)c1, NULL, NULL, 0, 0};
    double *eps = eps_out ? eps_out : (double *)malloc(cells(n) * sizeof(double));
    if (!eps) return NAN;
    residual(&H, &L, eps);
    double r = orc_rms(n, eps);
    if (!eps_out) free(eps);
    return r;
}

/* Single steps, exported for the tests: one Gauss-Seidel pass over one
   colour, the restriction R (nf -> nf/2) and fine += P(coarse). */
void orc_gs_colour(int kind, int n, double *u, const double *f, const double *c0, const double *c1, double rho,
                   int color)
{
    hier_t H = {kind, 1, 0, 0, rho, NULL};
    level_t L = {n, u, (double *)f, (double *)c0, (double *)c1, NULL, NULL, 0, 0};
    gs_colour(&H, &L, color);
}

void orc_restrict(int nf, const double *fine, double *coarse) { restrict8(nf, fine, coarse); }

void orc_prolong_add(int nf, const double *coarse, double *fine) { prolong_add(nf, coarse, fine); }

/* One V(nu1, nu2) cycle on u (in place).  For the Poisson kind f is used as
   given (callers subtract its mean) and the solution mean is not touched. */
int orc_vcycle(int kind, int n, double *u, const double *f, const double *c0, const double *c1, double rho, int nu1,
               int nu2)
{
    if (!valid_n(n)) return ORC_ERR_ARG;
    hier_t H;
    memset(&H, 0, sizeof(H));
    int st = hier_build(&H, kind, n, u, f, c0, c1, rho, nu1, nu2);
    if (st == ORC_OK) vcycle_level(&H, H.nlev - 1);
    hier_free(&H);
    return st;
}

/* Solve one equation: V-cycles until RMS(eps)/ref <= tol or max_cycles.
   Poisson: the source mean is removed first and the solution mean is set to
   zero after every cycle (periodic zero mode, Sec. 4.3.1).  ref <= 0 selects
   RMS(f); a reference below 1e-300 is replaced by 1.  Returns a status and
   fills cycles, the initial and the final relative residual. */
int orc_solve_eq(int kind, int n, double *u, const double *f, const double *c0, const double *c1, double rho,
                 double ref, double tol, int max_cycles, int nu1, int nu2, int *cycles, double *res0, double *res)
{
    if (!valid_n(n) || max_cycles < 0 || nu1 < 0 || nu2 < 0) return ORC_ERR_ARG;
    const int64_t N = cells(n);
    double *ff = (double *)malloc(N * sizeof(double));
    if (!ff) return ORC_ERR_NOMEM;
    memcpy(ff, f, N * sizeof(double));
    if (kind == ORC_POISSON) {
        subtract_mean(n, ff);
        subtract_mean(n, u);
    }
    if (ref <= 0.0) ref = orc_rms(n, ff);
    if (!(ref >= 1e-300)) ref = 1.0;
    hier_t H;
    memset(&H, 0, sizeof(H));
    int st = hier_build(&H, kind, n, u, ff, c0, c1, rho, nu1, nu2);
    int cyc = 0;
    double r = NAN, r0 = NAN;
    if (st == ORC_OK) {
        level_t *F = &H.lev[H.nlev - 1];
        r0 = r = orc_residual(kind, n, u, ff, c0, c1, rho, F->tmp) / ref;
        if (!isfinite(r)) st = ORC_ERR_NONFINITE;
        while (st == ORC_OK && r > tol && cyc < max_cycles) {
            vcycle_level(&H, H.nlev - 1);
            if (kind == ORC_POISSON) subtract_mean(n, u);
            r = orc_residual(kind, n, u, ff, c0, c1, rho, F->tmp) / ref;
            cyc++;
            if (!isfinite(r)) st = ORC_ERR_NONFINITE;
        }
        if (st == ORC_OK && r > tol) st = ORC_ERR_NOCONV;
    }
    hier_free(&H);
    free(ff);
    if (cycles) *cycles = cyc;
    if (res0) *res0 = r0;
    if (res) *res = r;
    return st;
}

/* ------------------------------------------------------------------ */
/* The ten-equation solve in the order of Sec. 2.4 / Sec. 4.3.1:       */
/* V_x, V_y, V_z, U, psi, alpha psi, B^x, B^y, B^z, b                   */
/* ------------------------------------------------------------------ */

/* Right-hand side, coefficients and reference norm of equation eq, derived
   from the sources and the current fields (the fields that eq depends on
   must already hold their solutions).  f, c0, c1 are n^3 outputs; returns
   the equation's kind.  The psi and alpha psi equations are posed for the
   deviations psi - 1 and alpha psi - 1 from the homogeneous background. */
int orc_eq_setup(int eq, int n, const double *const *src /*s0 sx sy sz sigma*/, const double *const *fld /*10*/,
                 double rho_hat, double S_hat, double *f, double *c0, double *c1, double *ref)
{
    const int64_t N = cells(n);
    const double K2 = 24.0 * PI * rho_hat, Kdot = 12.0 * PI * rho_hat + 4.0 * PI * S_hat;
    if (eq <= 2) {
        /* lap V_i = 8 pi (s_i - <s_i>)  (Eq. MG-linear-1a, mean removal of Sec. 4.3.1) */
        double m = orc_mean(n, src[1 + eq]);
        for (int64_t c = 0; c < N; c++) f[c] = 8.0 * PI * (src[1 + eq][c] - m);
        *ref = orc_rms(n, f);
        return ORC_POISSON;
    }
    if (eq == 3 || eq == 9) {
        /* lap U = -1/4 div V ; lap b = -1/4 div B */
        const double *const *F = eq == 3 ? fld + 0 : fld + 6;
        orc_div3(n, F[0], F[1], F[2], f);
        for (int64_t c = 0; c < N; c++) f[c] *= -0.25;
        double m = orc_mean(n, f);
        for (int64_t c = 0; c < N; c++) f[c] -= m;
        *ref = orc_rms(n, f);
        return ORC_POISSON;
    }
    double *A = (double *)malloc(6 * N * sizeof(double));
    if (!A) return -1;
    orc_aij(n, fld[0], fld[1], fld[2], fld[3], A);
    int kind;
    if (eq == 4) {
        /* psi = 1 + u: f = 0, c0 = s0, c1 = AA ; reference RMS(2 pi s0) */
        orc_aa(n, A, c1);
        memcpy(c0, src[0], N * sizeof(double));
        memset(f, 0, N * sizeof(double));
        *ref = 2.0 * PI * orc_rms(n, src[0]);
        kind = ORC_PSI;
    } else if (eq == 5) {
        /* alpha psi = 1 + u: lap u - m u = -psi^5 Kdot + m ; reference RMS(psi^5 Kdot) */
        double *aa = (double *)malloc(N * sizeof(double));
        if (!aa) {
            free(A);
            return -1;
        }
        orc_aa(n, A, aa);
        orc_lapse_coef(n, fld[4], src[0], src[4], aa, K2, Kdot, c0, f);
        free(aa);
        *ref = orc_rms(n, f);
        for (int64_t c = 0; c < N; c++) f[c] += c0[c];
        kind = ORC_HELMHOLTZ;
    } else {
        /* B^i: S_B^i = 2 div(A')^i, mean removed */
        double *SB = (double *)malloc(3 * N * sizeof(double));
        if (!SB) {
            free(A);
            return -1;
        }
        orc_shift_source(n, A, fld[4], fld[5], SB);
        memcpy(f, SB + (int64_t)(eq - 6) * N, N * sizeof(double));
        free(SB);
        double m = orc_mean(n, f);
        for (int64_t c = 0; c < N; c++) f[c] -= m;
        *ref = orc_rms(n, f);
        kind = ORC_POISSON;
    }
    free(A);
    return kind;
}

/* Full solve.  src: s0, s_x, s_y, s_z, sigma (n^3 each); fld: psi, alpha psi,
   V_x, V_y, V_z, U, B^x, B^y, B^z, b in the order of the enum below, guesses
   in, solutions out.  Equation order (field index): V_x(2) V_y(3) V_z(4) U(5)
   psi(0) alpha psi(1) B^x(6) B^y(7) B^z(8) b(9).  Per-equation cycles,
   residuals and statuses are reported in solve order.  Returns the first
   non-OK status, else OK. */
static const int solve_field[10] = {2, 3, 4, 5, 0, 1, 6, 7, 8, 9};

int orc_solve_constraints(int n, const double *const *src, double *const *fld, double rho_hat, double S_hat, double tol,
                          int max_cycles, int nu1, int nu2, int *cycles, double *res0, double *res, int *status)
{
    if (!valid_n(n)) return ORC_ERR_ARG;
    const int64_t N = cells(n);
    double *f = (double *)malloc(N * sizeof(double));
    double *c0 = (double *)malloc(N * sizeof(double));
    double *c1 = (double *)malloc(N * sizeof(double));
    if (!f || !c0 || !c1) {
        free(f); free(c0); free(c1);
        return ORC_ERR_NOMEM;
    }
    /* fields in the order used by orc_eq_setup: V_x V_y V_z U psi apsi B^x B^y B^z b */
    const double *setup_fld[10] = {fld[2], fld[3], fld[4], fld[5], fld[0], fld[1], fld[6], fld[7], fld[8], fld[9]};
    int worst = ORC_OK;
    for (int e = 0; e < 10; e++) {
        double ref = 1.0;
        int kind = orc_eq_setup(e, n, src, setup_fld, rho_hat, S_hat, f, c0, c1, &ref);
        int st;
        if (kind < 0) {
            st = ORC_ERR_NOMEM;
        } else {
            int cyc = 0;
            double r0 = NAN, r = NAN;
            double *u = fld[solve_field[e]];
            const int dev = (e == 4 || e == 5); /* psi, alpha psi: solve for the deviation from 1 */
            if (dev)
                for (int64_t c = 0; c < N; c++) u[c] -= 1.0;
            st = orc_solve_eq(kind, n, u, f, c0, c1, rho_hat, ref, tol, max_cycles, nu1, nu2, &cyc, &r0, &r);
            if (dev)
                for (int64_t c = 0; c < N; c++) u[c] += 1.0;
            if (cycles) cycles[e] = cyc;
            if (res0) res0[e] = r0;
            if (res) res[e] = r;
        }
        if (status) status[e] = st;
        if (st != ORC_OK && worst == ORC_OK) worst = st;
        if (st == ORC_ERR_NOMEM || st == ORC_ERR_NONFINITE) break;
    }
    free(f);
    free(c0);
    free(c1);
    return worst;
}


/* ------------------------------------------------------------------ */
/* Residuals at sampled cells, for grids too large for a full oracle   */
/* solve: each equation's right-hand side and coefficients evaluated   */
/* locally from the sources and fields (same formulas as orc_eq_setup) */
/* ------------------------------------------------------------------ */

/* A_ij (xx yy zz xy xz yz) at one cell from the V and U stencils */
static void aij_at(int n, const double *const *V, const double *U, int i, int j, int k, double A[6])
{
    const double i2h = 0.5 * n, ih2 = (double)n * n;
    double D[3][3];
    for (int a = 0; a < 3; a++)
        for (int l = 0; l < 3; l++) D[a][l] = (at(V[l], n, i, j, k, a, 1) - at(V[l], n, i, j, k, a, -1)) * i2h;
    const double divV = D[0][0] + D[1][1] + D[2][2];
    const double u0 = U[ix(n, i, j, k)];
    for (int a = 0; a < 3; a++) {
        const double Uaa = (at(U, n, i, j, k, a, 1) - 2.0 * u0 + at(U, n, i, j, k, a, -1)) * ih2;
        A[a] = 2.0 * D[a][a] - 0.5 * divV + 2.0 * Uaa;
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int p = 0; p < 3; p++) {
        const int a = pa[p], b = pb[p];
        double s = 0.0;
        for (int sa = -1; sa <= 1; sa += 2)
            for (int sb = -1; sb <= 1; sb += 2) {
                int c[3] = {i, j, k};
                c[a] = (c[a] + sa + n) % n;
                c[b] = (c[b] + sb + n) % n;
                s += (double)(sa * sb) * U[ix(n, c[0], c[1], c[2])];
            }
        A[3 + p] = D[a][b] + D[b][a] + 2.0 * s * 0.25 * ih2;
    }
}

static double aa_of(const double A[6])
{
    return A[0] * A[0] + A[1] * A[1] + A[2] * A[2] + 2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
}

static double div_at(int n, const double *const *F, int i, int j, int k)
{
    double s = 0.0;
    for (int a = 0; a < 3; a++) s += at(F[a], n, i, j, k, a, 1) - at(F[a], n, i, j, k, a, -1);
    return s * 0.5 * n;
}

/* S_B^comp at one cell: 2 sum_l D_l (phi psi^-7 A^{comp l}) */
static double shift_source_at(int n, const double *const *V, const double *U, const double *psi, const double *apsi,
                              int comp, int i, int j, int k)
{
    const int tab[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
    double s = 0.0;
    for (int l = 0; l < 3; l++)
        for (int sg = -1; sg <= 1; sg += 2) {
            int c[3] = {i, j, k};
            c[l] = (c[l] + sg + n) % n;
            double A[6];
            aij_at(n, V, U, c[0], c[1], c[2], A);
            const int64_t id = ix(n, c[0], c[1], c[2]);
            const double p = psi[id], p2 = p * p, p4 = p2 * p2;
            s += (double)sg * apsi[id] / (p4 * p2 * p) * A[tab[comp][l]];
        }
    return 2.0 * s * 0.5 * n;
}

/* eps = L(u) - f of equation eq (solve order) at the ncell cells idx[] of the
   natural layout, with the fields and sources given (fld in solve order:
   V_x V_y V_z U psi apsi B^x B^y B^z b).  The global source means of the
   Poisson-type equations are computed with one pass each.  eps[c] and the
   local right-hand side scale f[c] (the quantity whose RMS is the equation's
   reference: the Poisson source, 2 pi s0, psi^5 Kdot) are written out. */
void orc_residual_at(int eq, int n, const double *const *src, const double *const *fld, double rho_hat,
                     double S_hat, int64_t ncell, const int64_t *idx, double *eps, double *fscale)
{
    const double ih2 = (double)n * n;
    const double K2 = 24.0 * PI * rho_hat, Kdot = 12.0 * PI * rho_hat + 4.0 * PI * S_hat;
    const double *const *V = fld;     /* V_x V_y V_z */
    const double *U = fld[3];
    const double *B[3] = {fld[6], fld[7], fld[8]};
    double mean = 0.0;
    if (eq <= 2) mean = orc_mean(n, src[1 + eq]);
    for (int64_t c = 0; c < ncell; c++) {
        const int64_t id = idx[c];
        const int k = (int)(id % n), j = (int)((id / n) % n), i = (int)(id / ((int64_t)n * n));
        const double *u = fld[eq];
        const double sh = (eq == 4 || eq == 5) ? 1.0 : 0.0; /* Laplacian of the deviation from 1 */
        const double nb = (at(u, n, i, j, k, 0, 1) - sh) + (at(u, n, i, j, k, 0, -1) - sh) +
                          (at(u, n, i, j, k, 1, 1) - sh) + (at(u, n, i, j, k, 1, -1) - sh) +
                          (at(u, n, i, j, k, 2, 1) - sh) + (at(u, n, i, j, k, 2, -1) - sh);
        const double lap = (nb - 6.0 * (u[id] - sh)) * ih2;
        double e, f;
        if (eq <= 2) {
            f = 8.0 * PI * (src[1 + eq][id] - mean);
            e = lap - f;
        } else if (eq == 3 || eq == 9) {
            const double *F[3] = {eq == 3 ? V[0] : B[0], eq == 3 ? V[1] : B[1], eq == 3 ? V[2] : B[2]};
            f = -0.25 * div_at(n, F, i, j, k);
            e = lap - f;
        } else if (eq == 4) {
            double A[6];
            aij_at(n, V, U, i, j, k, A);
            const double p = u[id], p2 = p * p, p4 = p2 * p2;
            f = 2.0 * PI * src[0][id];
            e = lap + 2.0 * PI * src[0][id] / p + aa_of(A) / (8.0 * p4 * p2 * p) - 2.0 * PI * rho_hat * p4 * p;
        } else if (eq == 5) {
            double A[6];
            aij_at(n, V, U, i, j, k, A);
            const double p = fld[4][id], p2 = p * p, p4 = p2 * p2, p8 = p4 * p4;
            const double m = 2.0 * PI / p2 * (src[0][id] + 2.0 * src[4][id] / p4) + 0.875 * aa_of(A) / p8 +
                             (5.0 / 12.0) * p4 * K2;
            f = p4 * p * Kdot;
            e = lap - m * u[id] + f;
        } else {
            f = shift_source_at(n, V, U, fld[4], fld[5], eq - 6, i, j, k);
            e = lap - f;
        }
        eps[c] = e;
        fscale[c] = f;
    }
}

/* ------------------------------------------------------------------ */
/* Static nested refinement patches: composite-grid FAS                */
/* ------------------------------------------------------------------ */
/*
 * The paper solves its equations on the adaptive grid of its host code
 * (Sec. 3, Sec. 4.3) without stating how a refined region couples to its
 * parent.  This part takes the multilevel FAS reading (Brandt's multilevel
 * adaptive technique) for static cubic patches: patch p refines a block of
 * n_p/2 cells per side of its parent by 2 per axis; patch 1 lies in the
 * periodic base (its block may wrap), patch p + 1 inside patch p with at
 * least two parent cells to spare on every side.
 *
 *   - A patch solves its own equation on its interior cells.  Its two ghost
 *     layers hold the trilinear interpolation P of the parent (Dirichlet
 *     data; the same weights as the prolongation, 3/4 and 1/4 per axis).
 *   - After the patch's relaxation the parent takes, on the cells the patch
 *     covers, u = R u_patch and the right-hand side L_parent(u) - R eps_patch
 *     (eps = L(u) - f of the patch, R the 8-child average), so that the
 *     parent converges to the restricted patch solution there (FAS,
 *     Sec. 4.3.2.1, applied across levels of different extent).
 *   - After the parent's solve the patch interior takes P(u_new - u_old) of
 *     the parent's change and its ghosts are interpolated afresh.
 *   - Flux matching: on each uncovered parent cell that shares a face with
 *     the covered block, the coarse flux (u_in - u_out)/h_c through that face
 *     is replaced by the mean of the four fine fluxes (u_inner - u_ghost)/h_f
 *     through it, as the right-hand side change -(T_fine - T_coarse)/h_c
 *     taken at each injection.  The composite operator is then conservative
 *     (its volume-weighted sum telescopes), and with the trilinear ghosts the
 *     composite solution is second-order accurate; without it the flux
 *     mismatch acts as a spurious source.
 *
 * One composite cycle: base V-cycle, then for p = 1..P the correction and
 * nu2 sweeps of patch p, then for p = P..1 nu1 sweeps of patch p, its
 * residual and the injection into its parent.  The residual of level l is
 * RMS(eps_l) over all its cells after that injection (on covered cells it is
 * R eps of the finer level), relative to the level's own reference; a solve
 * converges when every level is at or below tol.
 *
 * Periodic Poisson-type equations: the coupled system is solvable only if
 * the volume-weighted sum of its right-hand sides vanishes, and a patch's
 * sources (deposited at its own resolution) need not sum to the base's over
 * the same region.  The system carries a scalar lambda added to the
 * source of every cell that no finer level covers, on every level (lambda
 * starts at 0).  After each injection into the base, m = mean of the base
 * right-hand side; every base cell loses m and lambda becomes lambda - m, so
 * the base stays mean-free and the patches see the same constant (on covered
 * cells it arrives through R eps).  The solution's mean is removed from every
 * level once, at the end.
 */
#define PG 2          /* ghost layers of a patch */
#define ORC_MAXP 4    /* patches in a chain */

static inline int64_t gx(int m, int i, int j, int k) { return ((int64_t)(i + PG) * m + (j + PG)) * m + (k + PG); }
static inline int wrapi(int i, int n) { return ((i % n) + n) % n; }
static inline int fdiv2(int i) { return i >= 0 ? i / 2 : -((-i + 1) / 2); }

/* One level seen as arrays with a common index map: the periodic base
   (natural n^3, indices wrap) or a patch (ghosted (n + 2 PG)^3). */
typedef struct {
    int n, ghosted;
    double *u, *f, *c0, *c1;
    double h2, ih2;
} view_t;

static inline int64_t vidx(const view_t *v, int i, int j, int k)
{
    if (v->ghosted) return gx(v->n + 2 * PG, i, j, k);
    return ix(v->n, wrapi(i, v->n), wrapi(j, v->n), wrapi(k, v->n));
}

static inline double vnb(const view_t *v, const double *a, int i, int j, int k)
{
    return a[vidx(v, i + 1, j, k)] + a[vidx(v, i - 1, j, k)] + a[vidx(v, i, j + 1, k)] + a[vidx(v, i, j - 1, k)] +
           a[vidx(v, i, j, k + 1)] + a[vidx(v, i, j, k - 1)];
}

/* L(u) of the level at one cell */
static inline double vop(int kind, const view_t *v, double rho, int i, int j, int k)
{
    const int64_t c = vidx(v, i, j, k);
    const double c0 = v->c0 ? v->c0[c] : 0.0, c1 = v->c1 ? v->c1[c] : 0.0;
    return op_point(kind, v->u[c], vnb(v, v->u, i, j, k), v->ih2, c0, c1, rho);
}

typedef struct {
    view_t v;              /* ghosted arrays of this patch */
    int o[3];              /* origin in parent cells */
    int nc, w;             /* covered parent cells per side (n / 2), window side (nc + 4) */
    double *eps, *win, *old, *Ru, *Re;
    double *flux;          /* the flux correction in force on each of the 6 nc^2 parent cells next to the block */
    double ref;
} patch_t;

/* parent cells o - 2 .. o + nc + 1 per axis into a w^3 window */
static void gather_window(const view_t *par, const patch_t *P, const double *a, double *win)
{
    const int w = P->w;
    for (int x = 0; x < w; x++)
        for (int y = 0; y < w; y++)
            for (int z = 0; z < w; z++)
                win[((int64_t)x * w + y) * w + z] = a[vidx(par, P->o[0] - 2 + x, P->o[1] - 2 + y, P->o[2] - 2 + z)];
}

/* trilinear interpolation of a window at patch cell (i, j, k), -PG <= i < n + PG:
   fine cell i sits in parent cell floor(i/2) and leans towards its neighbour
   on the side of i's half (weights 3/4, 1/4 per axis) */
static double interp_window(const double *win, int w, int i, int j, int k)
{
    int I[2], J[2], K[2];
    I[0] = fdiv2(i) + 2; I[1] = I[0] + ((i & 1) ? 1 : -1);
    J[0] = fdiv2(j) + 2; J[1] = J[0] + ((j & 1) ? 1 : -1);
    K[0] = fdiv2(k) + 2; K[1] = K[0] + ((k & 1) ? 1 : -1);
    const double wt[2] = {0.75, 0.25};
    double s = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++)
            for (int c = 0; c < 2; c++) s += wt[a] * wt[b] * wt[c] * win[((int64_t)I[a] * w + J[b]) * w + K[c]];
    return s;
}

static inline int is_interior(int n, int i, int j, int k)
{
    return i >= 0 && i < n && j >= 0 && j < n && k >= 0 && k < n;
}

/* ghost cells of a (ghosted m^3) patch array from the parent window */
static void fill_ghosts(const patch_t *P, const double *win, double *a)
{
    const int n = P->v.n, m = n + 2 * PG;
    for (int i = -PG; i < n + PG; i++)
        for (int j = -PG; j < n + PG; j++)
            for (int k = -PG; k < n + PG; k++)
                if (!is_interior(n, i, j, k)) a[gx(m, i, j, k)] = interp_window(win, P->w, i, j, k);
}

/* the block of a patch's cells that its child patch covers (co = NULL: no child) */
typedef struct {
    const int *co;
    int nc;
    double lam;
} cover_t;

/* right-hand side of a patch cell: f, plus lambda where no child covers it */
static inline double rhs_at(const view_t *v, const cover_t *cv, int i, int j, int k)
{
    const double f = v->f[vidx(v, i, j, k)];
    if (cv->co && i - cv->co[0] >= 0 && i - cv->co[0] < cv->nc && j - cv->co[1] >= 0 && j - cv->co[1] < cv->nc &&
        k - cv->co[2] >= 0 && k - cv->co[2] < cv->nc)
        return f;
    return f + cv->lam;
}

/* one red-black Gauss-Seidel colour over the patch interior (local colour
   (i + j + k) % 2), the same point update as gs_colour */
static void patch_gs(int kind, double rho, const view_t *v, const cover_t *cv, int color)
{
    const int n = v->n;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = (i + j + color) & 1; k < n; k += 2) {
                const int64_t c = vidx(v, i, j, k);
                const double nb = vnb(v, v->u, i, j, k);
                const double f = rhs_at(v, cv, i, j, k);
                double *u = v->u;
                if (kind == ORC_POISSON) {
                    u[c] = (nb - v->h2 * f) / 6.0;
                } else if (kind == ORC_HELMHOLTZ) {
                    u[c] = (nb - v->h2 * f) / (6.0 + v->h2 * v->c0[c]);
                } else {
                    double w = 1.0 + u[c], w2 = w * w, w4 = w2 * w2;
                    double g = op_point(ORC_PSI, u[c], nb, v->ih2, v->c0[c], v->c1[c], rho) - f;
                    double dg = -6.0 * v->ih2 - 2.0 * PI * v->c0[c] / w2 - 7.0 * v->c1[c] / (8.0 * w4 * w4) -
                                10.0 * PI * rho * w4;
                    u[c] -= g / dg;
                }
            }
}

/* eps = L(u) - f over the patch interior; returns RMS(eps) */
static double patch_residual(int kind, double rho, const patch_t *P, const cover_t *cv)
{
    const int n = P->v.n;
    double s = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                const int64_t c = vidx(&P->v, i, j, k);
                const double e = vop(kind, &P->v, rho, i, j, k) - rhs_at(&P->v, cv, i, j, k);
                P->eps[c] = e;
                s += e * e;
            }
    return sqrt(s / (double)cells(n));
}

/* Ru, Re: 8-child averages of the patch's u and eps (nc^3, natural) */
static void patch_restrict(const patch_t *P)
{
    const int nc = P->nc;
    for (int I = 0; I < nc; I++)
        for (int J = 0; J < nc; J++)
            for (int K = 0; K < nc; K++) {
                double su = 0.0, se = 0.0;
                for (int a = 0; a < 2; a++)
                    for (int b = 0; b < 2; b++)
                        for (int c = 0; c < 2; c++) {
                            const int64_t id = vidx(&P->v, 2 * I + a, 2 * J + b, 2 * K + c);
                            su += P->v.u[id];
                            se += P->eps[id];
                        }
                P->Ru[ix(nc, I, J, K)] = 0.125 * su;
                P->Re[ix(nc, I, J, K)] = 0.125 * se;
            }
}

typedef struct {
    int kind, np, nu1, nu2, n0;
    double rho;
    hier_t H;                    /* base hierarchy; its finest f is the working right-hand side */
    view_t base;                 /* finest base level */
    double *forig;               /* the base right-hand side as set up */
    patch_t P[ORC_MAXP + 1];     /* P[1..np] */
    double ref[ORC_MAXP + 1];
    double lambda;               /* the Poisson solvability constant */
} comp_t;

static view_t *parent_of(comp_t *C, int p) { return p == 1 ? &C->base : &C->P[p - 1].v; }

static cover_t cover_of(const comp_t *C, int p)
{
    cover_t cv = {NULL, 0, C->lambda};
    if (p < C->np) {
        cv.co = C->P[p + 1].o;
        cv.nc = C->P[p + 1].nc;
    }
    return cv;
}

/* u = R u_patch and f = L(u) - R eps on the parent cells patch p covers;
   the parent window after the injection becomes the patch's u_old */
static void inject(comp_t *C, int p)
{
    patch_t *P = &C->P[p];
    view_t *par = parent_of(C, p);
    const int nc = P->nc;
    patch_restrict(P);
    for (int I = 0; I < nc; I++)
        for (int J = 0; J < nc; J++)
            for (int K = 0; K < nc; K++)
                par->u[vidx(par, P->o[0] + I, P->o[1] + J, P->o[2] + K)] = P->Ru[ix(nc, I, J, K)];
    gather_window(par, P, par->u, P->old);
    for (int I = 0; I < nc; I++)
        for (int J = 0; J < nc; J++)
            for (int K = 0; K < nc; K++) {
                const int a = P->o[0] + I, b = P->o[1] + J, c = P->o[2] + K;
                par->f[vidx(par, a, b, c)] = vop(C->kind, par, C->rho, a, b, c) - P->Re[ix(nc, I, J, K)];
            }
    {
        /* parent cells next to the block: the coarse flux through the shared face
           replaced by the mean of the four fine fluxes (as a right-hand side change) */
        const int n = P->v.n, m = n + 2 * PG;
        const double hc = sqrt(par->h2), hf = 0.5 * hc;
        int q = 0;
        for (int ax = 0; ax < 3; ax++)
            for (int sd = -1; sd <= 1; sd += 2)
                for (int t1 = 0; t1 < nc; t1++)
                    for (int t2 = 0; t2 < nc; t2++, q++) {
                        const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
                        int in[3], out[3];
                        in[ax] = sd < 0 ? 0 : nc - 1;
                        in[b1] = t1;
                        in[b2] = t2;
                        for (int d = 0; d < 3; d++) out[d] = in[d] + (d == ax ? sd : 0);
                        const double uin = par->u[vidx(par, P->o[0] + in[0], P->o[1] + in[1], P->o[2] + in[2])];
                        const double uout = par->u[vidx(par, P->o[0] + out[0], P->o[1] + out[1], P->o[2] + out[2])];
                        const double Tc = (uin - uout) / hc;
                        double Tf = 0.0;
                        for (int e1 = 0; e1 < 2; e1++)
                            for (int e2 = 0; e2 < 2; e2++) {
                                int fi[3], fg[3];
                                fi[ax] = sd < 0 ? 0 : n - 1;
                                fg[ax] = sd < 0 ? -1 : n;
                                fi[b1] = fg[b1] = 2 * t1 + e1;
                                fi[b2] = fg[b2] = 2 * t2 + e2;
                                Tf += (P->v.u[gx(m, fi[0], fi[1], fi[2])] - P->v.u[gx(m, fg[0], fg[1], fg[2])]) / hf;
                            }
                        Tf *= 0.25;
                        const double corr = -(Tf - Tc) / hc;
                        par->f[vidx(par, P->o[0] + out[0], P->o[1] + out[1], P->o[2] + out[2])] += corr - P->flux[q];
                        P->flux[q] = corr;
                    }
    }
    if (p == 1 && C->kind == ORC_POISSON) {
        /* the base loses the mean of its right-hand side; lambda follows */
        const int64_t N = cells(C->n0);
        double *f = C->base.f;
        double m = 0.0;
        for (int64_t q = 0; q < N; q++) m += f[q];
        m /= (double)N;
        for (int64_t q = 0; q < N; q++) f[q] -= m;
        C->lambda -= m;
    }
}

/* patches P..1: nu sweeps, residual, injection; then the base residual.
   res[l] = relative residual of level l */
static void comp_down(comp_t *C, int nu, double *res)
{
    for (int p = C->np; p >= 1; p--) {
        patch_t *P = &C->P[p];
        const cover_t cv = cover_of(C, p);
        for (int s = 0; s < nu; s++) {
            patch_gs(C->kind, C->rho, &P->v, &cv, 0);
            patch_gs(C->kind, C->rho, &P->v, &cv, 1);
        }
        res[p] = patch_residual(C->kind, C->rho, P, &cv) / C->ref[p];
        inject(C, p);
    }
    res[0] = orc_residual(C->kind, C->n0, C->base.u, C->base.f, C->base.c0, C->base.c1, C->rho, NULL) / C->ref[0];
}

/* patches 1..P: the parent's correction P(u_new - u_old) on the interior,
   fresh ghosts, nu sweeps */
static void comp_up(comp_t *C, int nu)
{
    for (int p = 1; p <= C->np; p++) {
        patch_t *P = &C->P[p];
        view_t *par = parent_of(C, p);
        const int n = P->v.n, m = n + 2 * PG;
        gather_window(par, P, par->u, P->win);
        const int64_t W = (int64_t)P->w * P->w * P->w;
        for (int64_t q = 0; q < W; q++) P->old[q] = P->win[q] - P->old[q];  /* old := new - old */
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                for (int k = 0; k < n; k++) P->v.u[gx(m, i, j, k)] += interp_window(P->old, P->w, i, j, k);
        fill_ghosts(P, P->win, P->v.u);
        const cover_t cv = cover_of(C, p);
        for (int s = 0; s < nu; s++) {
            patch_gs(C->kind, C->rho, &P->v, &cv, 0);
            patch_gs(C->kind, C->rho, &P->v, &cv, 1);
        }
    }
}

static void comp_free(comp_t *C)
{
    for (int p = 1; p <= C->np; p++) {
        patch_t *P = &C->P[p];
        free(P->eps); free(P->win); free(P->old); free(P->Ru); free(P->Re); free(P->flux);
        P->eps = P->win = P->old = P->Ru = P->Re = P->flux = NULL;
    }
    free(C->forig);
    C->forig = NULL;
    hier_free(&C->H);
}

static int patch_chain_valid(int n0, int np, const int *pn, const int *po)
{
    if (!valid_n(n0) || np < 0 || np > ORC_MAXP) return 0;
    int npar = n0;
    for (int p = 0; p < np; p++) {
        const int n = pn[p];
        if (!valid_n(n) || n < 8) return 0;
        for (int d = 0; d < 3; d++) {
            const int o = po[3 * p + d];
            if (p == 0) {
                if (o < 0 || o >= n0 || n / 2 + 4 > n0) return 0;
            } else if (o < 2 || o + n / 2 + 2 > npar) {
                return 0;
            }
        }
        npar = n;
    }
    return 1;
}

/* largest of the levels' residuals, NaN if one is not finite */
static double worst_of(const double *r, int nl)
{
    double w = 0.0;
    for (int l = 0; l < nl; l++) {
        if (!isfinite(r[l])) return NAN;
        if (r[l] > w) w = r[l];
    }
    return w;
}

/* The composite solve of one equation on ghosted patch arrays already in
   C->P[p].v (u with interior guess, f, c0, c1) and the base arrays. */
static int comp_solve(comp_t *C, double tol, int max_cycles, int *cycles, double *res0, double *res)
{
    double r[ORC_MAXP + 1];
    /* ghosts of the guesses, coarse to fine */
    for (int p = 1; p <= C->np; p++) {
        gather_window(parent_of(C, p), &C->P[p], parent_of(C, p)->u, C->P[p].win);
        fill_ghosts(&C->P[p], C->P[p].win, C->P[p].v.u);
    }
    comp_down(C, 0, r);
    if (res0)
        for (int l = 0; l <= C->np; l++) res0[l] = r[l];
    int st = ORC_OK, cyc = 0;
    double worst = worst_of(r, C->np + 1);
    if (!isfinite(worst)) st = ORC_ERR_NONFINITE;
    while (st == ORC_OK && worst > tol && cyc < max_cycles) {
        vcycle_level(&C->H, C->H.nlev - 1);
        comp_up(C, C->nu2);
        comp_down(C, C->nu1, r);
        cyc++;
        worst = worst_of(r, C->np + 1);
        if (!isfinite(worst)) st = ORC_ERR_NONFINITE;
    }
    if (st == ORC_OK && worst > tol) st = ORC_ERR_NOCONV;
    if (C->kind == ORC_POISSON) {
        /* the solution's mean off every level */
        const double m = orc_mean(C->n0, C->base.u);
        for (int64_t q = 0; q < cells(C->n0); q++) C->base.u[q] -= m;
        for (int p = 1; p <= C->np; p++) {
            const int mm = C->P[p].v.n + 2 * PG;
            for (int64_t q = 0; q < (int64_t)mm * mm * mm; q++) C->P[p].v.u[q] -= m;
        }
    }
    if (cycles) *cycles = cyc;
    if (res)
        for (int l = 0; l <= C->np; l++) res[l] = r[l];
    return st;
}

/* set up the base hierarchy and the patch work arrays of C (patch u, f, c0,
   c1 must be set by the caller afterwards or before: they are not touched) */
static int comp_init(comp_t *C, int kind, int n0, int np, const int *pn, const int *po, double rho, double *u0,
                     const double *f0, const double *c00, const double *c10, int nu1, int nu2)
{
    C->kind = kind; C->np = np; C->nu1 = nu1; C->nu2 = nu2; C->n0 = n0; C->rho = rho;
    const int64_t N0 = cells(n0);
    C->forig = (double *)malloc(N0 * sizeof(double));
    if (!C->forig) return ORC_ERR_NOMEM;
    memcpy(C->forig, f0, N0 * sizeof(double));
    if (kind == ORC_POISSON) subtract_mean(n0, C->forig);
    int st = hier_build(&C->H, kind, n0, u0, C->forig, c00, c10, rho, nu1, nu2);
    if (st != ORC_OK) return st;
    level_t *F = &C->H.lev[C->H.nlev - 1];
    C->base.n = n0; C->base.ghosted = 0;
    C->base.u = u0; C->base.f = F->f; C->base.c0 = (double *)c00; C->base.c1 = (double *)c10;
    C->base.h2 = 1.0 / ((double)n0 * n0); C->base.ih2 = (double)n0 * n0;
    for (int p = 1; p <= np; p++) {
        patch_t *P = &C->P[p];
        const int n = pn[p - 1];
        const double nh = (double)n0 * (double)(1 << p); /* 1/h of this patch */
        P->v.n = n; P->v.ghosted = 1;
        P->v.h2 = 1.0 / (nh * nh); P->v.ih2 = nh * nh;
        for (int d = 0; d < 3; d++) P->o[d] = po[3 * (p - 1) + d];
        P->nc = n / 2; P->w = n / 2 + 4;
        const int64_t M = (int64_t)(n + 2 * PG) * (n + 2 * PG) * (n + 2 * PG);
        const int64_t W = (int64_t)P->w * P->w * P->w, Nc = cells(P->nc);
        P->eps = (double *)calloc(M, sizeof(double));
        P->win = (double *)calloc(W, sizeof(double));
        P->old = (double *)calloc(W, sizeof(double));
        P->Ru = (double *)calloc(Nc, sizeof(double));
        P->Re = (double *)calloc(Nc, sizeof(double));
        P->flux = (double *)calloc(6 * P->nc * P->nc, sizeof(double));
        if (!P->eps || !P->win || !P->old || !P->Ru || !P->Re || !P->flux) return ORC_ERR_NOMEM;
    }
    return ORC_OK;
}

static double rms_interior(int n, const double *a)
{
    const int m = n + 2 * PG;
    double s = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) s += a[gx(m, i, j, k)] * a[gx(m, i, j, k)];
    return sqrt(s / (double)cells(n));
}

/* interior n^3 (natural) <-> ghosted (n + 2 PG)^3 */
static void to_ghosted(int n, const double *in, double *out, double add)
{
    const int m = n + 2 * PG;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) out[gx(m, i, j, k)] = in[ix(n, i, j, k)] + add;
}

static void from_ghosted(int n, const double *in, double *out, double add)
{
    const int m = n + 2 * PG;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) out[ix(n, i, j, k)] = in[gx(m, i, j, k)] + add;
}

/* Composite solve of one equation (kind, rho as orc_solve_eq) on the base
   (u0, f0, c00, c10: n0^3 natural) and a chain of np patches: pn[p] cells
   per side, origins po[3p..3p+2] in parent cells; up/fp/c0p/c1p: interior
   pn^3 natural arrays (c0p, c1p entries may be NULL where the kind has no
   such coefficient).  refs[l] (np + 1 values) are the levels' reference
   norms, <= 0 for RMS(f) of the level (the base's after mean removal for
   Poisson).  res0/res receive the np + 1 relative residuals (base first). */
int orc_composite_eq(int kind, int n0, int np, const int *pn, const int *po, double rho, double *u0,
                     const double *f0, const double *c00, const double *c10, double *const *up,
                     const double *const *fp, const double *const *c0p, const double *const *c1p, const double *refs,
                     double tol, int max_cycles, int nu1, int nu2, int *cycles, double *res0, double *res)
{
    if (!patch_chain_valid(n0, np, pn, po) || max_cycles < 0 || nu1 < 0 || nu2 < 0) return ORC_ERR_ARG;
    comp_t C;
    memset(&C, 0, sizeof(C));
    int st = comp_init(&C, kind, n0, np, pn, po, rho, u0, f0, c00, c10, nu1, nu2);
    double *store[ORC_MAXP + 1][4];
    memset(store, 0, sizeof(store));
    for (int p = 1; p <= np && st == ORC_OK; p++) {
        const int n = pn[p - 1];
        const int64_t M = (int64_t)(n + 2 * PG) * (n + 2 * PG) * (n + 2 * PG);
        for (int q = 0; q < 4; q++) {
            store[p][q] = (double *)calloc(M, sizeof(double));
            if (!store[p][q]) st = ORC_ERR_NOMEM;
        }
        if (st != ORC_OK) break;
        view_t *v = &C.P[p].v;
        v->u = store[p][0]; v->f = store[p][1];
        v->c0 = c0p && c0p[p - 1] ? store[p][2] : NULL;
        v->c1 = c1p && c1p[p - 1] ? store[p][3] : NULL;
        to_ghosted(n, up[p - 1], v->u, 0.0);
        to_ghosted(n, fp[p - 1], v->f, 0.0);
        if (v->c0) to_ghosted(n, c0p[p - 1], v->c0, 0.0);
        if (v->c1) to_ghosted(n, c1p[p - 1], v->c1, 0.0);
    }
    if (st == ORC_OK) {
        C.ref[0] = (refs && refs[0] > 0) ? refs[0] : orc_rms(n0, C.forig);
        for (int p = 1; p <= np; p++)
            C.ref[p] = (refs && refs[p] > 0) ? refs[p] : rms_interior(pn[p - 1], C.P[p].v.f);
        for (int l = 0; l <= np; l++)
            if (!(C.ref[l] >= 1e-300)) C.ref[l] = 1.0;
        st = comp_solve(&C, tol, max_cycles, cycles, res0, res);
        for (int p = 1; p <= np; p++) from_ghosted(pn[p - 1], C.P[p].v.u, up[p - 1], 0.0);
    }
    for (int p = 1; p <= np; p++)
        for (int q = 0; q < 4; q++) free(store[p][q]);
    comp_free(&C);
    return st;
}

/* ------------------------------------------------------------------ */
/* Sources and the ten-equation solve on a patch chain                 */
/* ------------------------------------------------------------------ */

/* CIC at resolution N (spacing 1/N: the arithmetic of orc_deposit with
   n = N), kept on the nw^3 window of cells O + a (mod N), 0 <= a < nw.
   A patch at level p of a base n0 is the window N = n0 2^p, O = its origin
   in cells of that resolution. */
void orc_deposit_window(int N, const int *O, int nw, int64_t np, const double *x, const double *u, double mass,
                        double *s0, double *sx, double *sy, double *sz, double *sigma)
{
    const double h = 1.0 / N, vol = h * h * h;
    const int64_t M = cells(nw);
    memset(s0, 0, M * sizeof(double));
    memset(sx, 0, M * sizeof(double));
    memset(sy, 0, M * sizeof(double));
    memset(sz, 0, M * sizeof(double));
    memset(sigma, 0, M * sizeof(double));
    for (int64_t p = 0; p < np; p++) {
        int lo[3];
        double fplus[3];
        for (int d = 0; d < 3; d++) {
            double xp = x[d * np + p];
            xp -= floor(xp);
            double t = xp / h - 0.5;
            double fl = floor(t);
            fplus[d] = 1.0 - (t - fl);
            int i = (int)fl;
            lo[d] = (i % N + N) % N;
        }
        double ux = u[p], uy = u[np + p], uz = u[2 * np + p];
        double u2 = ux * ux + uy * uy + uz * uz;
        double W = sqrt(1.0 + u2);
        double q0 = mass * W / vol, qx = mass * ux / vol, qy = mass * uy / vol, qz = mass * uz / vol;
        double qs = mass * u2 / W / vol;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++)
                for (int c = 0; c < 2; c++) {
                    const int ra = wrapi((lo[0] + a) % N - O[0], N), rb = wrapi((lo[1] + b) % N - O[1], N),
                              rc = wrapi((lo[2] + c) % N - O[2], N);
                    if (ra >= nw || rb >= nw || rc >= nw) continue;
                    double w = (a ? 1.0 - fplus[0] : fplus[0]) * (b ? 1.0 - fplus[1] : fplus[1]) *
                               (c ? 1.0 - fplus[2] : fplus[2]);
                    int64_t id = ix(nw, ra, rb, rc);
                    s0[id] += q0 * w;
                    sx[id] += qx * w;
                    sy[id] += qy * w;
                    sz[id] += qz * w;
                    sigma[id] += qs * w;
                }
    }
}

static inline int64_t gxs(int m, int i, int j, int k, int a, int s)
{
    int c[3] = {i, j, k};
    c[a] += s;
    return gx(m, c[0], c[1], c[2]);
}

/* A_ij (xx yy zz xy xz yz) at a patch cell from ghosted V, U (the stencils
   of orc_aij; 1/h = nh) */
static void aij_ghosted(int m, const double *const *V, const double *U, double nh, int i, int j, int k, double A[6])
{
    const double i2h = 0.5 * nh, ih2 = nh * nh;
    double D[3][3];
    for (int a = 0; a < 3; a++)
        for (int l = 0; l < 3; l++) D[a][l] = (V[l][gxs(m, i, j, k, a, 1)] - V[l][gxs(m, i, j, k, a, -1)]) * i2h;
    const double divV = D[0][0] + D[1][1] + D[2][2];
    const double u0 = U[gx(m, i, j, k)];
    for (int a = 0; a < 3; a++) {
        const double Uaa = (U[gxs(m, i, j, k, a, 1)] - 2.0 * u0 + U[gxs(m, i, j, k, a, -1)]) * ih2;
        A[a] = 2.0 * D[a][a] - 0.5 * divV + 2.0 * Uaa;
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
    for (int p = 0; p < 3; p++) {
        const int a = pa[p], b = pb[p];
        double s = 0.0;
        for (int sa = -1; sa <= 1; sa += 2)
            for (int sb = -1; sb <= 1; sb += 2) {
                int c[3] = {i, j, k};
                c[a] += sa;
                c[b] += sb;
                s += (double)(sa * sb) * U[gx(m, c[0], c[1], c[2])];
            }
        A[3 + p] = D[a][b] + D[b][a] + 2.0 * s * 0.25 * ih2;
    }
}

/* Right-hand side, coefficients (ghosted arrays, interior written) and
   reference of equation e on a patch of n cells at 1/h = nh: the formulas of
   orc_eq_setup with derivatives taken on the ghosted fields G (setup order
   V_x V_y V_z U psi apsi B^x B^y B^z b; the entries the equation reads are
   filled).  The momentum sources lose the base mean smean of s_i (the
   homogeneous background); the divergence sources of U, b and B^i keep
   theirs (on the periodic base it vanishes up to rounding). */
static int patch_eq_setup(int e, int n, double nh, const double *const *src, const double *const *G, double smean,
                          double rho_hat, double S_hat, double *f, double *c0, double *c1, double *ref)
{
    const int m = n + 2 * PG;
    const double K2 = 24.0 * PI * rho_hat, Kdot = 12.0 * PI * rho_hat + 4.0 * PI * S_hat, i2h = 0.5 * nh;
    double s2 = 0.0;
    int kind = ORC_POISSON;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                const int64_t g = gx(m, i, j, k), id = ix(n, i, j, k);
                if (e <= 2) {
                    f[g] = 8.0 * PI * (src[1 + e][id] - smean);
                    s2 += f[g] * f[g];
                } else if (e == 3 || e == 9) {
                    const double *const *F = G + (e == 3 ? 0 : 6);
                    double s = 0.0;
                    for (int a = 0; a < 3; a++) s += F[a][gxs(m, i, j, k, a, 1)] - F[a][gxs(m, i, j, k, a, -1)];
                    f[g] = -0.25 * s * i2h;
                    s2 += f[g] * f[g];
                } else if (e == 4) {
                    double A[6];
                    aij_ghosted(m, G, G[3], nh, i, j, k, A);
                    c1[g] = aa_of(A);
                    c0[g] = src[0][id];
                    f[g] = 0.0;
                    s2 += src[0][id] * src[0][id];
                    kind = ORC_PSI;
                } else if (e == 5) {
                    double A[6];
                    aij_ghosted(m, G, G[3], nh, i, j, k, A);
                    const double aa = aa_of(A);
                    const double p = G[4][g], p2 = p * p, p4 = p2 * p2, p8 = p4 * p4;
                    c0[g] = 2.0 * PI / p2 * (src[0][id] + 2.0 * src[4][id] / p4) + 0.875 * aa / p8 +
                            (5.0 / 12.0) * p4 * K2;
                    const double fk = -p4 * p * Kdot;
                    s2 += fk * fk;
                    f[g] = fk + c0[g];
                    kind = ORC_HELMHOLTZ;
                } else {
                    const int tab[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
                    double s = 0.0;
                    for (int l = 0; l < 3; l++)
                        for (int sg = -1; sg <= 1; sg += 2) {
                            int c[3] = {i, j, k};
                            c[l] += sg;
                            double A[6];
                            aij_ghosted(m, G, G[3], nh, c[0], c[1], c[2], A);
                            const int64_t q = gx(m, c[0], c[1], c[2]);
                            const double p = G[4][q], p2 = p * p, p4 = p2 * p2;
                            s += (double)sg * G[5][q] / (p4 * p2 * p) * A[tab[e - 6][l]];
                        }
                    f[g] = 2.0 * s * i2h;
                    s2 += f[g] * f[g];
                }
            }
    *ref = sqrt(s2 / (double)cells(n));
    if (e == 4) *ref *= 2.0 * PI;
    if (!(*ref >= 1e-300)) *ref = 1.0;
    return kind;
}

/* Ten-equation composite solve (the order of orc_solve_constraints) on the
   base (src0: 5 arrays, fld0: 10 fields in field order, n0^3) and a patch
   chain (pn, po as orc_composite_eq; srcp[5p + q], fldp[10p + q]: pn^3
   natural arrays, q in the base's order).  cycles[e], status[e] per
   equation in solve order; res[e (np + 1) + l] the final relative residual
   of level l (0 = base). */
int orc_solve_composite(int n0, int np, const int *pn, const int *po, const double *const *src0,
                        const double *const *srcp, double *const *fld0, double *const *fldp, double rho_hat,
                        double S_hat, double tol, int max_cycles, int nu1, int nu2, int *cycles, double *res,
                        int *status)
{
    if (!patch_chain_valid(n0, np, pn, po) || max_cycles < 0 || nu1 < 0 || nu2 < 0) return ORC_ERR_ARG;
    const int64_t N0 = cells(n0);
    /* setup order V_x V_y V_z U psi apsi B^x B^y B^z b -> field index */
    static const int fidx[10] = {2, 3, 4, 5, 0, 1, 6, 7, 8, 9};
    double *f = (double *)malloc(N0 * sizeof(double));
    double *c0 = (double *)malloc(N0 * sizeof(double));
    double *c1 = (double *)malloc(N0 * sizeof(double));
    double *G[ORC_MAXP + 1][10];
    double *wk[ORC_MAXP + 1][4];
    double *win[ORC_MAXP + 1];
    memset(G, 0, sizeof(G));
    memset(wk, 0, sizeof(wk));
    memset(win, 0, sizeof(win));
    int worst = (f && c0 && c1) ? ORC_OK : ORC_ERR_NOMEM;
    for (int p = 1; p <= np && worst == ORC_OK; p++) {
        const int n = pn[p - 1], w = n / 2 + 4;
        const int64_t M = (int64_t)(n + 2 * PG) * (n + 2 * PG) * (n + 2 * PG);
        for (int q = 0; q < 10; q++)
            if (!(G[p][q] = (double *)calloc(M, sizeof(double)))) worst = ORC_ERR_NOMEM;
        for (int q = 0; q < 4; q++)
            if (!(wk[p][q] = (double *)calloc(M, sizeof(double)))) worst = ORC_ERR_NOMEM;
        if (!(win[p] = (double *)calloc((int64_t)w * w * w, sizeof(double)))) worst = ORC_ERR_NOMEM;
    }
    const double *setup0[10];
    for (int q = 0; q < 10; q++) setup0[q] = fld0[fidx[q]];
    for (int e = 0; e < 10 && worst == ORC_OK; e++) {
        /* ghosted copies of the solved fields the equation reads, coarse to fine */
        int need[10] = {0};
        if (e == 3) need[0] = need[1] = need[2] = 1;
        if (e == 4 || e == 5) need[0] = need[1] = need[2] = need[3] = 1;
        if (e == 5) need[4] = 1;
        if (e >= 6 && e <= 8) need[0] = need[1] = need[2] = need[3] = need[4] = need[5] = 1;
        if (e == 9) need[6] = need[7] = need[8] = 1;
        for (int p = 1; p <= np; p++) {
            const int n = pn[p - 1];
            patch_t P;
            memset(&P, 0, sizeof(P));
            P.v.n = n; P.nc = n / 2; P.w = n / 2 + 4;
            for (int d = 0; d < 3; d++) P.o[d] = po[3 * (p - 1) + d];
            view_t par;
            memset(&par, 0, sizeof(par));
            if (p == 1) { par.n = n0; par.ghosted = 0; }
            else { par.n = pn[p - 2]; par.ghosted = 1; }
            for (int q = 0; q < 10; q++) {
                if (!need[q]) continue;
                to_ghosted(n, fldp[10 * (p - 1) + fidx[q]], G[p][q], 0.0);
                gather_window(&par, &P, p == 1 ? setup0[q] : G[p - 1][q], win[p]);
                fill_ghosts(&P, win[p], G[p][q]);
            }
        }
        double ref0 = 1.0;
        const int kind = orc_eq_setup(e, n0, src0, setup0, rho_hat, S_hat, f, c0, c1, &ref0);
        if (kind < 0) {
            worst = ORC_ERR_NOMEM;
            break;
        }
        const int dev = (e == 4 || e == 5);
        double refs[ORC_MAXP + 1];
        refs[0] = ref0 >= 1e-300 ? ref0 : 1.0;
        comp_t C;
        memset(&C, 0, sizeof(C));
        double *u0 = fld0[fidx[e]];
        if (dev)
            for (int64_t q = 0; q < N0; q++) u0[q] -= 1.0;
        int st = comp_init(&C, kind, n0, np, pn, po, rho_hat, u0, f, kind == ORC_POISSON ? NULL : c0,
                           kind == ORC_PSI ? c1 : NULL, nu1, nu2);
        for (int p = 1; p <= np && st == ORC_OK; p++) {
            const int n = pn[p - 1];
            const double smean = e <= 2 ? orc_mean(n0, src0[1 + e]) : 0.0;
            view_t *v = &C.P[p].v;
            v->u = wk[p][0]; v->f = wk[p][1];
            v->c0 = kind == ORC_POISSON ? NULL : wk[p][2];
            v->c1 = kind == ORC_PSI ? wk[p][3] : NULL;
            patch_eq_setup(e, n, (double)n0 * (double)(1 << p), srcp + 5 * (p - 1), (const double *const *)G[p],
                           smean, rho_hat, S_hat, v->f, wk[p][2], wk[p][3], &refs[p]);
            to_ghosted(n, fldp[10 * (p - 1) + fidx[e]], v->u, dev ? -1.0 : 0.0);
        }
        if (st == ORC_OK) {
            for (int l = 0; l <= np; l++) C.ref[l] = refs[l];
            double r[ORC_MAXP + 1];
            int cyc = 0;
            st = comp_solve(&C, tol, max_cycles, &cyc, NULL, r);
            if (cycles) cycles[e] = cyc;
            if (res)
                for (int l = 0; l <= np; l++) res[e * (np + 1) + l] = r[l];
            for (int p = 1; p <= np; p++)
                from_ghosted(pn[p - 1], C.P[p].v.u, fldp[10 * (p - 1) + fidx[e]], dev ? 1.0 : 0.0);
        }
        if (dev)
            for (int64_t q = 0; q < N0; q++) u0[q] += 1.0;
        comp_free(&C);
        if (status) status[e] = st;
        if (st != ORC_OK && worst == ORC_OK) worst = st;
        if (st == ORC_ERR_NOMEM || st == ORC_ERR_NONFINITE) break;
    }
    for (int p = 1; p <= np; p++) {
        for (int q = 0; q < 10; q++) free(G[p][q]);
        for (int q = 0; q < 4; q++) free(wk[p][q]);
        free(win[p]);
    }
    free(f);
    free(c0);
    free(c1);
    return worst;
}

/* ------------------------------------------------------------------ */
/* Pointwise checks on a patch, for grids too large for a full oracle   */
/* composite solve                                                      */
/* ------------------------------------------------------------------ */

/* Ghosted (n + 2 PG)^3 array from a patch's interior (natural n^3) and its
   parent (natural npar^3, periodic if the parent is the base): ghosts are
   the trilinear interpolation of the parent window at origin o. */
void orc_patch_ghosted(int n, const int *o, int npar, int parent_periodic, const double *parent,
                       const double *interior, double *out)
{
    view_t par;
    memset(&par, 0, sizeof(par));
    par.n = npar;
    par.ghosted = 0;
    patch_t P;
    memset(&P, 0, sizeof(P));
    P.v.n = n;
    P.nc = n / 2;
    P.w = n / 2 + 4;
    for (int d = 0; d < 3; d++) P.o[d] = o[d];
    double *win = (double *)malloc((size_t)P.w * P.w * P.w * sizeof(double));
    if (!win) return;
    if (parent_periodic) {
        gather_window(&par, &P, parent, win);
    } else {
        /* a patch parent: its interior cells o - 2 .. o + nc + 1 (the chain keeps them inside) */
        const int w = P.w;
        for (int x = 0; x < w; x++)
            for (int y = 0; y < w; y++)
                for (int z = 0; z < w; z++)
                    win[((int64_t)x * w + y) * w + z] = parent[ix(npar, o[0] - 2 + x, o[1] - 2 + y, o[2] - 2 + z)];
    }
    to_ghosted(n, interior, out, 0.0);
    fill_ghosts(&P, win, out);
    free(win);
}

/* eps = L(u) - f of equation e (solve order) on a patch without a child, at
   the interior cells idx[] (natural n^3 indices): the set-up of
   patch_eq_setup from the patch's sources src (5 interior arrays) and its
   ghosted fields G (setup order), then the operator at each cell.  fscale[c]
   receives the local reference quantity (the right-hand side; 2 pi s0 for
   psi; psi^5 Kdot for alpha psi).  No solvability constant is added: for the
   Poisson-type equations eps carries the solve's uniform lambda. */
void orc_patch_residual_at(int e, int n, double nh, const double *const *src, const double *const *G, double smean,
                           double rho_hat, double S_hat, int64_t ncell, const int64_t *idx, double *eps,
                           double *fscale)
{
    const int m = n + 2 * PG;
    const int64_t M = (int64_t)m * m * m;
    double *f = (double *)calloc(M, sizeof(double));
    double *c0 = (double *)calloc(M, sizeof(double));
    double *c1 = (double *)calloc(M, sizeof(double));
    if (!f || !c0 || !c1) {
        free(f); free(c0); free(c1);
        return;
    }
    double ref;
    const int kind = patch_eq_setup(e, n, nh, src, G, smean, rho_hat, S_hat, f, c0, c1, &ref);
    const double Kdot = 12.0 * PI * rho_hat + 4.0 * PI * S_hat;
    const int fi[10] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9};
    const double *u = G[fi[e]];
    view_t v;
    memset(&v, 0, sizeof(v));
    v.n = n;
    v.ghosted = 1;
    v.ih2 = nh * nh;
    v.h2 = 1.0 / v.ih2;
    double *ud = (double *)malloc(M * sizeof(double)); /* the equation's unknown: psi - 1, alpha psi - 1 */
    if (!ud) {
        free(f); free(c0); free(c1);
        return;
    }
    const double sh = (e == 4 || e == 5) ? 1.0 : 0.0;
    for (int64_t q = 0; q < M; q++) ud[q] = u[q] - sh;
    v.u = ud;
    v.f = f;
    v.c0 = kind == ORC_POISSON ? NULL : c0;
    v.c1 = kind == ORC_PSI ? c1 : NULL;
    for (int64_t c = 0; c < ncell; c++) {
        const int64_t id = idx[c];
        const int k = (int)(id % n), j = (int)((id / n) % n), i = (int)(id / ((int64_t)n * n));
        const int64_t g = gx(m, i, j, k);
        eps[c] = vop(kind, &v, rho_hat, i, j, k) - f[g];
        if (e == 4) fscale[c] = 2.0 * PI * src[0][id];
        else if (e == 5) fscale[c] = pow(G[4][g], 5) * Kdot;
        else fscale[c] = f[g];
    }
    free(ud);
    free(f);
    free(c0);
    free(c1);
}

/* The set-up of one equation on a patch (patch_eq_setup), exported for the
   test that holds it against orc_eq_setup on a full periodic grid: src are
   the patch's 5 interior arrays, G its ten ghosted fields in setup order;
   f, c0, c1 receive ghosted (n + 2 PG)^3 arrays (interior written).
   Returns the kind. */
int orc_patch_eq_setup(int e, int n, double nh, const double *const *src, const double *const *G, double smean,
                       double rho_hat, double S_hat, double *f, double *c0, double *c1, double *ref)
{
    return patch_eq_setup(e, n, nh, src, G, smean, rho_hat, S_hat, f, c0, c1, ref);
}
