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

static void coarsest(const hier_t *H, level_t *L)
{
    if (H->kind == ORC_POISSON) subtract_mean(L->n, L->f);
    for (int s = 0; s < COARSEST_SWEEPS; s++) sweep(H, L);
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
