/*
 * gr.h - C ABI of the GB300 constrained-GR elliptic solver.
 *
 * The library solves, on a uniform periodic n^3 grid (box side L, cell size
 * h = L/n, cell centres x_i = (i + 1/2) h, G = c = 1), the ten elliptic
 * equations of the fully constrained ADM formulation with CMC slicing,
 * minimal-distortion shift and conformal flatness (arXiv:1905.08890,
 * Sec. 2.4 solution sequence, Sec. 4.3 multigrid):
 *
 *   V_i        lap V_i = 8 pi (s_i - <s_i>)             Eq. MG-linear-1a (geometric units)
 *   U          lap U   = -1/4 div V                     Eq. MG-linear-1
 *   psi        lap psi = -2 pi s0/psi - AA/(8 psi^7) + 2 pi rho_hat psi^5
 *                                                        Eq. sol-scheme-H-constraint
 *   alpha psi  lap(alpha psi) = m alpha psi - psi^5 Kdot Eq. sol-scheme-CMC
 *              m = 2 pi psi^-2 (s0 + 2 psi^-4 sigma) + 7/8 psi^-8 AA + 5/12 psi^4 K^2
 *   B^i        lap B^i = 2 d_j (alpha psi^-6 A^ij)      Eqs. MDC-CF, MG-linear-2a
 *   b          lap b   = -1/4 div B                     Eq. MG-linear-2
 *
 * with A_ij = d_i V_j + d_j V_i - 1/2 delta_ij div V + 2 d_i d_j U
 * (Eq. Aij-discrete-2), AA = A_ij A^ij, K^2 = 24 pi rho_hat and
 * Kdot = 12 pi rho_hat + 4 pi S_hat (Eqs. 1-Friedmann, 2-Friedmann with
 * rho_Lambda = 0).  Sources come from a cloud-in-cell deposit of particles
 * (Sec. 4.1.2).  Discretisation: 7-point Laplacian, 3-point central
 * differences, 4-cell cross derivative (Sec. 4.3.1).  Solver: red-black
 * Gauss-Seidel V(nu1, nu2) cycles down to the 2^3 level.
 *
 * Conventions for every call:
 *  - Arrays are double [n][n][n], C order, index (i*n + j)*n + k, i the x
 *    index.  All array pointers are DEVICE pointers owned by the caller
 *    (for example torch CUDA tensors), contiguous, 8-byte aligned, and must
 *    not alias one another unless a call says so.  The context owns its own
 *    multigrid scratch.
 *  - All work is queued on the context's stream.  Calls that return host
 *    scalars (norms, reports) synchronise that stream before returning.
 *    Kernels are launched with programmatic dependent launch (a kernel may
 *    be scheduled while its predecessor on the stream drains, and waits for
 *    it before touching memory), so the stream's order of effects is that of
 *    plain launches; a stream that refuses the attribute gets plain launches.
 *  - Static nested refinement patches (gr_patch, gr_deposit_patches,
 *    gr_opts.patch) extend the periodic base with a chain of finer cubic
 *    regions solved as one composite problem.
 *  - No call aborts or throws.  Errors are returned as gr_status; the
 *    thread-local gr_last_error() describes the last one.  Arguments are
 *    validated before any GPU work is queued.
 *  - Not thread safe per context: one host thread drives a context at a time.
 */
#ifndef GR_H
#define GR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GR_OK = 0,
    GR_ERR_ARG = 1,       /* invalid argument (bad n, null pointer, bad option) */
    GR_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    GR_ERR_NOMEM = 3,     /* device or host allocation failed */
    GR_ERR_NOCONV = 4,    /* max_cycles reached above tol; fields hold the last iterate */
    GR_ERR_NONFINITE = 5, /* a residual norm became NaN or Inf */
    GR_ERR_STATE = 6      /* call not valid in the context's state */
} gr_status;

/* Equations in solve order (Sec. 2.4: momentum constraint, Hamiltonian
   constraint, lapse, shift; Sec. 4.3.1 for the V/U and B/b split). */
typedef enum {
    GR_VX = 0, GR_VY, GR_VZ, GR_U, GR_PSI, GR_APSI, GR_BX, GR_BY, GR_BZ, GR_B_SCALAR,
    GR_NEQ
} gr_eq;

typedef enum {
    GR_PREC_FP64 = 0,     /* every sweep, transfer and residual in FP64 */
    GR_PREC_MIXED = 1,    /* FP64 fine residual and update; FP32 correction V-cycle
                             (psi: on the Newton linearisation); FP64 2^3 level */
    GR_PREC_MIXED_DF = 2  /* as GR_PREC_MIXED, but the finest level's set-up, residual,
                             update and write-back in double-float (pairs of FP32,
                             48-bit significand); results agree with GR_PREC_FP64 to
                             the tolerance */
} gr_prec;

typedef struct gr_ctx gr_ctx; /* opaque */

/* CIC sources, device arrays of n^3 doubles each, natural layout, each
   starting on a 16-byte boundary (the kernels move them in 16-byte vectors;
   an entry point given a NULL or misaligned array returns GR_ERR_ARG):
   s0 = sqrt(gamma) rho, s[l] = sqrt(gamma) S_l, sigma = sum_l s_ll (Sec. 3). */
typedef struct {
    double *s0;
    double *s[3];
    double *sigma;
} gr_sources;

/* The ten potentials, device arrays of n^3 doubles each, natural layout,
   16-byte aligned like the sources.  psi is the
   conformal factor, apsi = alpha psi; beta^i = B^i + d^i b and
   W_i = V_i + d_i U (Sec. 4.3.1). */
typedef struct {
    double *psi;
    double *apsi;
    double *V[3];
    double *U;
    double *B[3];
    double *b;
} gr_fields;

/* Static nested refinement patches (the paper's solver runs on an adaptive
   grid, Sec. 3 and Sec. 4.3; this library offers a chain of static cubic
   patches).  patch[0] refines the periodic base; patch[p] refines
   patch[p - 1].  Patch p has n cells per side at spacing h / 2^(p + 1) and
   covers the parent cells origin .. origin + n/2 - 1 per axis (parent cell
   units; patch[0]'s block may wrap around the periodic base).  Constraints:
   n a power of two, 8 <= n <= 512; patch[0]: 0 <= origin < base n and
   n/2 + 4 <= base n; patch[p > 0]: origin >= 2 and origin + n/2 + 2 <= the
   parent's n.  src and fld are caller-owned device arrays of n^3 doubles,
   natural layout (index (i n + j) n + k within the patch): src as
   gr_deposit_patches writes it, fld the guesses in and the solutions out. */
#define GR_MAX_PATCHES 4
typedef struct {
    int n;
    int origin[3];
    gr_sources src;
    gr_fields fld;
} gr_patch;

typedef struct {
    double tol;       /* stop an equation when RMS(eps)/ref <= tol (see gr_solve_constraints) */
    int max_cycles;   /* per equation; >= 0 */
    int nu1, nu2;     /* pre- and post-smoothing red-black sweeps per level, 0..8 */
    gr_prec prec;
    double rho_hat;   /* fiducial density; <= 0 or NaN selects mass*np/L^3 of the last gr_deposit */
    double S_hat;     /* fiducial trace of the stress (dust: 0); NaN selects 0 */
    int verbose;      /* 0 silent; 1 one line per equation on stderr */
    int profile;      /* nonzero: time the finest-level kernels with CUDA events (gr_report.prof_*) */
    int check_guess;  /* nonzero: per equation, drop the given guess for the plain one (psi = alpha psi = 1,
                         vectors 0) when its residual is not finite or, after the first cycle, still above
                         the plain guess's initial residual (gr_report.guess_rejected) */
    int fmg;          /* nonzero (mixed modes, n >= 32): the first correction of every equation is a full
                         multigrid cycle (nested iteration) instead of a V-cycle: the fine residual is
                         averaged down to 16^3, solved there by two V-cycles, and each finer level starts
                         from the trilinear prolongation of the coarser solution and takes one V-cycle.
                         A classical non-learned warm start; the paper's solver uses V-cycles only
                         (Sec. 4.3.1), so the default is 0.  Ignored by GR_PREC_FP64. */
    const gr_fields *host_out; /* gr_solve_constraints only, may be NULL: ten arrays of n^3 doubles (host memory,
                         pinned for overlap, or any memory cudaMemcpyAsync accepts), caller-owned.  Each field
                         is copied there as soon as its equation is solved, on a copy stream of the context,
                         so the copies overlap the remaining equations; the call's stream waits for the last
                         copy before the call returns, so a synchronisation of that stream covers them.  The
                         base fields only: patch fields stay in the patches' device arrays. */
    int npatch;       /* gr_solve_constraints only: 0 (default) solves the periodic base alone; 1..GR_MAX_PATCHES
                         solves the composite problem on the base and the chain patch[0..npatch-1] (composite-grid
                         FAS: a patch's ghost layers take the trilinear interpolation of its parent, the parent
                         takes the restricted patch solution and residual on the cells the patch covers, and the
                         coarse flux through each face of a covered block is replaced by the mean of the four
                         fine fluxes).  Every equation then stops when the base and every patch are at or below
                         tol, each relative to its own reference.  Patches relax in FP64 with GR_PREC_FP64 and
                         in double-float (pairs of FP32) in the mixed modes; check_guess is ignored. */
    const gr_patch *patch;
} gr_opts;

/* Finest-level kernel classes timed when gr_opts.profile is set. */
typedef enum {
    GR_PROF_SWEEP64 = 0,   /* FP64 red-black colour pass */
    GR_PROF_SWEEP32,       /* FP32 red-black colour pass (mixed) */
    GR_PROF_RESTRICT,      /* residual fused with restriction (FP64 or FP32) */
    GR_PROF_PROLONG,       /* trilinear prolongation + correction (FP64 or FP32) */
    GR_PROF_MIXED_RESID,   /* fine residual feeding the FP32 correction (mixed: FP64; mixed_df: double-float,
                              with the correction's first red pass) */
    GR_PROF_MIXED_UPDATE,  /* u += FP32 correction (mixed_df: fused with the last black pass) */
    GR_PROF_NORM64,        /* FP64 residual norm (FP64 path) */
    GR_PROF_SETUP,         /* sources, coefficients and layout changes of the finest level */
    GR_PROF_COARSE,        /* every multigrid kernel below the finest level (and full multigrid's coarser cycles) */
    GR_PROF_PATCH,         /* nested patches: set-up, relaxation, residual, transfers and injection */
    GR_PROF_SMOOTH3,       /* three FP32 colour passes fused into one pass over memory (finest level, nu = 2) */
    GR_NPROF
} gr_prof_class;

typedef struct {
    int cycles[GR_NEQ];           /* V-cycles (mixed: outer iterations) per equation */
    double res0[GR_NEQ];          /* relative residual of the initial guess */
    double res[GR_NEQ];           /* relative residual at exit */
    gr_status eq_status[GR_NEQ];
    double seconds;               /* wall time of the whole call (host clock around the stream) */
    double eq_seconds[GR_NEQ];    /* per equation, CUDA events */
    long long cell_updates;       /* cells relaxed: every sweep on every level, all equations (the exact
                                     solve of a linear 2^3 level counts its 8 cells once) */
    long long kernel_launches;    /* kernels this call launched */
    int prof_launches[GR_NPROF];  /* with gr_opts.profile: launches per gr_prof_class */
    double prof_ms[GR_NPROF];     /* with gr_opts.profile: summed CUDA-event time per class */
    int guess_rejected[GR_NEQ];   /* with gr_opts.check_guess: 1 where the plain guess replaced the given one */
    double res_level[GR_NEQ][GR_MAX_PATCHES + 1]; /* with patches: relative residual at exit of the base (0) and of
                                                     patch p (p + 1); res is their maximum */
} gr_report;

/* Fill *o with the defaults: tol 1e-10, max_cycles 50, V(2,2), FP64,
   rho_hat and S_hat from the deposit / dust, verbose 0, profile 0, check_guess 0, fmg 0, no host_out,
   no patches. */
void gr_default_opts(gr_opts *o);

/* Create a context for an n^3 grid of box side L.  n must be a power of two,
   4 <= n <= 1024; L > 0.  cuda_stream is a cudaStream_t (NULL = the legacy
   default stream); the device is the current device of the calling thread.
   Allocates the multigrid scratch (about 12 n^3 doubles) and 16 doubles of
   mapped pinned host memory, which kernels write the residual norms into for
   the host to read.  On success *out owns both; release with gr_destroy. */
gr_status gr_create(int n, double L, void *cuda_stream, gr_ctx **out);

/* Release a context and its device memory (synchronises its stream).  NULL is ignored. */
void gr_destroy(gr_ctx *ctx);

/* Cloud-in-cell deposit (Sec. 4.1.2, Eqs. s0/si/sij-code-unit-cic) of np
   identical particles of rest mass `mass`.  x and u are arrays in
   structure-of-arrays layout [3][np]: positions (wrapped periodically into
   [0, L)) and lower-index 4-velocities u_l.  Both device memory, or both host
   memory: host arrays (pinned for full speed) are copied in chunks of
   GR_HOST_CHUNK particles (environment, read at gr_create; default 4M)
   through two device staging buffers that the context allocates at first
   use, each chunk's copy overlapping the previous chunk's deposit on a copy
   stream of the context; the call returns once the copies are queued, and the
   host arrays must stay valid until the context's stream has passed them.
   A mix of host and device pointers is GR_ERR_ARG.  Each particle adds, with CIC
   weight w over the 8 surrounding cell centres, m W w/h^3 to s0,
   m u_l w/h^3 to s_l and m |u|^2/W w/h^3 to sigma, W = sqrt(1 + |u|^2)
   (the conformal factor is taken as 1 in the Lorentz factor).  The five
   output arrays are overwritten.  np = 0 gives zero sources.  Also records
   mass*np/L^3 as the default rho_hat of the context. */
gr_status gr_deposit(gr_ctx *ctx, int64_t np, const double *x, const double *u, double mass, gr_sources *out);

/* Solve the ten equations in solve order (gr_eq), each until its relative
   residual RMS(eps)/ref <= opts->tol, eps = L(u) - f (Eqs. epsilon-error-lin,
   epsilon-error-nonlin-1), with ref: V_i RMS(8 pi (s_i - <s_i>)); U
   RMS(1/4 div V); psi RMS(2 pi s0); alpha psi RMS(psi^5 Kdot); B^i RMS of
   its source; b RMS(1/4 div B); a ref below 1e-300 is replaced by 1.
   Poisson-type sources have their mean removed and their solutions are
   returned with zero mean (periodic zero mode).  inout holds the initial
   guesses on entry (for example the previous solution, or psi = apsi = 1
   and zero vectors) and the solutions on return; the sources are not
   modified.  Each equation uses the fields solved before it.  Returns GR_OK,
   or the first failing equation's status (NOCONV: fields keep the last
   iterate and the remaining equations are still solved; NONFINITE: stops).
   rep (host, may be NULL) receives per-equation cycles and residuals. */
/* Cloud-in-cell sources of every patch of a chain (gr_opts.patch): each
   patch's five src arrays are overwritten with the deposit of the np
   particles at the patch's resolution (the formulas of gr_deposit with
   spacing h / 2^(p + 1)), restricted to the patch's cells; particles whose
   cloud misses the patch add nothing.  x, u: device arrays as in gr_deposit
   (host memory returns GR_ERR_ARG).  Queued on the context's stream.
   GR_ERR_ARG for an invalid chain or a NULL array. */
gr_status gr_deposit_patches(gr_ctx *ctx, int npatch, const gr_patch *patch, int64_t np, const double *x,
                             const double *u, double mass);

gr_status gr_solve_constraints(gr_ctx *ctx, const gr_sources *src, gr_fields *inout, const gr_opts *opts,
                               gr_report *rep);

/* One V(nu1, nu2) cycle (mixed precision: one defect-correction iteration)
   of equation eq, with its right-hand side and coefficients derived from the
   sources and the current fields exactly as in gr_solve_constraints.  For
   Poisson-type equations the solution mean is set to zero afterwards.
   *res_after (host, may be NULL) receives the relative residual after the
   cycle. */
gr_status gr_vcycle(gr_ctx *ctx, gr_eq eq, const gr_sources *src, gr_fields *inout, const gr_opts *opts,
                    double *res_after);

/* Residual eps = L(u) - f of equation eq at the current fields (right-hand
   side and coefficients derived as in gr_solve_constraints; for Poisson-type
   equations the source mean is removed first).  res_field (device, n^3
   doubles, may be NULL) receives eps; *rel_norm (host, may be NULL)
   receives RMS(eps)/ref.  Always evaluated in FP64. */
gr_status gr_residual(gr_ctx *ctx, gr_eq eq, const gr_sources *src, const gr_fields *fields, const gr_opts *opts,
                      double *res_field, double *rel_norm);

/* Message of the last error on the calling thread ("" if none). */
const char *gr_last_error(void);

/* Kernels launched by this library in this process so far (all contexts). */
long long gr_kernel_launches(void);

/* ------------------------------------------------------------------------
   Learned initial guess.  The paper has no counterpart: this is a small 3D
   U-Net that maps the sources to an initial guess of the ten fields, to
   shorten the V-cycle iterations of gr_solve_constraints.  Architecture:
   four levels of 16, 32, 64, 128 channels, two circular 3^3 convolutions with
   ReLU per level and side, 2^3 average pooling, cell-centred trilinear x2
   upsampling, concatenated skips, 1x1 head to 10 channels (psi - 1,
   alpha psi - 1, V_x, V_y, V_z, U, B^x, B^y, B^z, b), standardised per
   channel.  Inputs: log(0.01 + s0/rho_hat) and s_i/(rho_hat v_rms),
   standardised.  BF16 activations and weights, FP32 accumulation on the
   tensor cores, FP32 master weights and Adam.  The network owns its device
   memory (about 1.4 GB at 128^3); calls queue on its stream and synchronise it
   where they return host values.
   ------------------------------------------------------------------------ */
typedef struct gr_net gr_net;

/* Create a network for n^3 grids (power of two, 32 <= n <= 512) with
   He-normal weights drawn from seed and identity normalisation. */
gr_status gr_net_create(int n, void *cuda_stream, uint64_t seed, gr_net **out);
void gr_net_destroy(gr_net *net);
/* Number of FP32 parameters (conv weights [27][cout][cin] and biases per
   layer in order, then the head [10][16] and its bias). */
size_t gr_net_num_params(const gr_net *net);
/* Copy the FP32 parameters to / from host memory (set also resets Adam). */
gr_status gr_net_get_params(gr_net *net, float *host);
gr_status gr_net_set_params(gr_net *net, const float *host);
/* Input (4 channels) and output (10 channels) standardisation: value =
   (x - mean) / std going in, std * y + mean coming out. */
gr_status gr_net_set_norm(gr_net *net, const float *in_mean, const float *in_std, const float *out_mean,
                          const float *out_std);
/* Write the network's guess of all ten fields into guess (device arrays). */
gr_status gr_net_infer(gr_net *net, const gr_sources *src, double rho_hat, double v_rms, gr_fields *guess);
/* The network's guess for a finer periodic grid of the same box: n_fine =
   the network's n times 2^k (k >= 0, n_fine <= 1024).  The sources (device,
   n_fine^3 each; sigma unused) are averaged over the 2^k cubed cells each
   network cell covers, the network runs on the averages, and its ten
   outputs are interpolated trilinearly between the network's (periodic)
   cell centres to every fine cell of guess (device, n_fine^3 each).  k = 0
   is gr_net_infer.  Scratch: four network-grid arrays of doubles, allocated
   by the network on first use.  Queued on the network's stream. */
gr_status gr_net_guess(gr_net *net, int n_fine, const gr_sources *src, double rho_hat, double v_rms,
                       gr_fields *guess);
/* Mean squared error of the standardised output against target (device
   fields, e.g. a converged solve) and its gradient; host_grads (may be NULL)
   receives gr_net_num_params floats.  Parameters are not changed. */
gr_status gr_net_loss_grad(gr_net *net, const gr_sources *src, const gr_fields *target, double rho_hat,
                           double v_rms, float *loss_out, float *host_grads);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) on that loss with learning rate lr. */
gr_status gr_net_train_step(gr_net *net, const gr_sources *src, const gr_fields *target, double rho_hat,
                            double v_rms, float lr, float *loss_out);
/* Copy activation tensor `tensor` (forward order: 0 input, 1..20 the layer
   outputs, pools and concatenations) of the last forward pass to host FP32;
   count must equal its size. */
gr_status gr_net_activation(gr_net *net, int tensor, float *host, size_t count);

/* ---- code units (Sec. 4.1) ----------------------------------------------
   The paper's code units at a fiducial scale factor a: box L = 1, c = G = 1,
   H0 the Hubble constant today in units of c/L, so the code-unit speed of
   light is ct = 1/H0 and the critical density rho_c = 3 H0^2 / (8 pi). */
typedef struct {
    double a;       /* fiducial scale factor, > 0 */
    double Omega_m; /* matter density parameter today, > 0 */
    double Omega_L; /* Lambda density parameter today, >= 0: it sets a(t) (Eqs. 1-Friedmann-code,
                       2-Friedmann-code) but enters none of the code-unit elliptic equations */
    double H0;      /* Hubble constant today in units of c / L, > 0 */
} gr_cosmology;
/* The ten-equation solve in code units (Eqs. Wi-code-units, H-constraint-MG-1,
   CMC-MG-1 with Q-function, MDC-code-units; Sec. 4.3.1 Eqs. MG-linear-1a,
   MG-linear-1, MG-linear-2a, MG-linear-2).  src: the code-unit sources
   st0 = s0 / (Omega_m rho_c), st_i = s_i / (Omega_m rho_c) and the trace
   sigt = sum_l st_ll (device, n^3 each, not modified; a deposit with mass
   m / (Omega_m rho_c) gives them).  fld: the code-unit fields, guesses in and
   solutions out: the psi slot holds Psi and the apsi slot Phi, defined by
   alpha = 1 + Phi / (a^2 ct^2), psi = a^(1/2) (1 - Psi / (2 a^2 ct^2)); V,
   U, B, b hold Vt = a ct^2 V, Ut = a ct^2 U, Bt = a^2 ct B, bt = a^2 ct b
   (all zero with Psi = Phi = 0 is the plain guess).  The problem is solved
   as the equivalent a = 1 geometric problem (sources s0 / a, s_i / a^2,
   sigma / a^3 of the geometric sources, rho_hat = Omega_m rho_c / a; the
   fields psi / a^(1/2), alpha psi / a^(1/2), V / a^2, U / a^2, a B, a b),
   with gr_solve_constraints and opts (its rho_hat and S_hat are replaced;
   npatch and host_out must be 0 / NULL); rep and the return status are
   that solve's, its residuals those of the a = 1 problem.  The context's box
   side must be 1.  Scratch: the context's first-use allocation of 5 n^3
   doubles.  GR_ERR_ARG: NULL pointers, parameters out of range, L != 1,
   patches or host_out requested. */
gr_status gr_solve_code_units(gr_ctx *ctx, const gr_cosmology *cosmo, const gr_sources *src, gr_fields *fld,
                              const gr_opts *opts, gr_report *rep);

/* ---- the particle update around the solve (Sec. 4.2 steps 3 and 6-8;
   Sec. 4.4; Sec. 4.5; App. A) ------------------------------------------
   Geometric units with a = 1, c = 1: the spatial metric is psi^4 delta_ij,
   alpha = (alpha psi) / psi, beta^i = B^i + d_i b, and the paper's code-unit
   potentials are Phi = alpha - 1, Psi = 2 (1 - psi).  Particles: x, u are
   device arrays [3][np] (SoA, x then y then z), positions in the periodic box
   [0, L), u the lower-index spatial 4-velocity u_i per unit rest mass. */
enum {
    GR_KICK_SYNC = 1, /* the synchronising kick u^(n-1/2) -> u^n: substeps j = 1..5 (Eq. GR-K2) */
    GR_KICK_OPEN = 2, /* the opening kick u^n -> u^(n+1/2): substeps j = 5..1 (Eq. GR-K1) */
    GR_DRIFT = 4      /* the drift x^n -> x^(n+1) (Eq. GR-D) */
};
/* Kicks and drift of np particles in the solved fields fld (psi, alpha psi,
   B^i, b are read; the other fields are not).  Each kick adds dt/2 F to u in
   the five substeps of Sec. 4.4 (Eqs. coeff_j, coeff_4, coeff_5):
   c_j = -u_j with (f_j)_i = -d_i beta^j (j = 1, 2, 3), c_4 = (W^2 - 1)/W
   alpha/psi with (f_4)_i = -d_i Psi, c_5 = W with (f_5)_i = -d_i Phi, each
   substep at the velocity the previous one left, W = sqrt(1 + psi^-4 |u|^2)
   (Eq. Lorentz-factor).  The drift adds dt (alpha psi^-4 u_i / W - beta^i)
   (Eq. V_exp) and wraps x into [0, L).  Everything is evaluated at the
   particle's position on entry: the fields and their 3-point central
   differences are formed on the grid and interpolated to the particle with
   the cloud-in-cell weights of gr_deposit.  flags: any of GR_KICK_SYNC,
   GR_KICK_OPEN (applied in that order), GR_DRIFT (after the kicks, with
   the kicked velocity); a time loop calls it once per step with all three
   after the solve (the first step without GR_KICK_SYNC).  Arithmetic: the
   interpolated quantities and the substeps in FP32, positions and
   velocities accumulated in FP64.  Scratch: the context's first-use
   allocation of 20 n^3 floats.  Queued on the context's stream; x and u are
   updated in place.  GR_ERR_ARG: NULL arrays, np < 0, host memory, dt not
   finite or flags outside the three bits. */
gr_status gr_particle_update(gr_ctx *ctx, int64_t np, double *x, double *u, const gr_fields *fld, double dt,
                             int flags);
/* gr_particle_update with flags GR_KICK_SYNC and/or GR_KICK_OPEN (x unchanged). */
gr_status gr_kick(gr_ctx *ctx, int64_t np, const double *x, double *u, const gr_fields *fld, double dt, int flags);
/* gr_particle_update with GR_DRIFT alone (u unchanged). */
gr_status gr_drift(gr_ctx *ctx, int64_t np, double *x, const double *u, const gr_fields *fld, double dt);
/* gr_deposit with the Lorentz factor of the current metric (Sec. 4.5 Eqs.
   src_s0, src_si, src_sij): W = sqrt(1 + psi^-4 |u|^2) with psi (device,
   n^3, natural layout: the previous solution's conformal factor) interpolated
   to the particle by cloud-in-cell; s0 += m W w / h^3, s_l += m u_l w / h^3,
   sigma += m |u|^2 / W w / h^3.  psi = NULL is gr_deposit (psi = 1).  Device
   particle arrays only (GR_ERR_ARG otherwise).  Sets the default rho_hat
   like gr_deposit. */
gr_status gr_deposit_metric(gr_ctx *ctx, int64_t np, const double *x, const double *u, double mass, const double *psi,
                            gr_sources *out);

/* Allocation-free residual of one momentum-constraint equation,
   lap V_i = 8 pi (s_i - <s_i>): the same residual and relative norm as
   gr_residual for GR_VX..GR_VZ, for callers that cannot allocate device
   memory.  The paper has no counterpart; this entry point exists for
   callers whose device memory is owned entirely by another allocator (a
   framework's caching pool or a fixed pre-reserved arena) and for loops that
   must not pay the device-wide synchronisation of cudaMalloc/cudaFree, so
   they cannot create a gr_ctx.
   n: power of two, 4 <= n <= 256 (larger n returns GR_ERR_ARG: the fixed
   scratch covers at most 256^3 cells).  L > 0: box side.  V, s: device
   arrays of n^3 doubles, natural layout (V_i and s_i), on the current
   device.  The C entry point cannot see buffer sizes: the caller owns that
   every array holds n^3 doubles (the Python binding checks it).  res_field (device,
   n^3 doubles, may be NULL) receives eps = lap_h V - 8 pi (s - <s>);
   *rel_norm (host, may be NULL) receives RMS(eps) / RMS(8 pi (s - <s>))
   (reference 1 below 1e-300).  cuda_stream: cudaStream_t (NULL = legacy
   default stream); the call synchronises it.
   No device memory is allocated or freed: the scratch is a 256 KB array
   compiled into the library, present on every device that loads it until
   the process exits.  The first call on a device looks up that array's
   device address (cudaGetSymbolAddress), so make a first call on each device
   before capturing any stream.  The address is kept for the life of the
   process: after cudaDeviceReset on a device this entry point must not be
   called on that device again.  All calls share the array: every slot a
   call reads is written earlier in the same call, so stale contents are
   harmless, but calls that overlap on the GPU (different streams or host
   threads at the same time) race on it and must be serialised by the caller. */
gr_status gr_momentum_residual_noalloc(int n, double L, const double *V, const double *s, double *res_field,
                                       double *rel_norm, void *cuda_stream);

/* Diagnostic, not part of the method: the FMA issue rate of the current
   device, in FLOP/s (2 per fused multiply-add), FP64 (fp64 != 0) or FP32.
   Eight blocks of 256 threads per SM each run 8 independent chains of `iters`
   FMAs (1 <= iters <= 2^32) after a short warm-up launch; the time is taken
   with CUDA events on cuda_stream (NULL = legacy default stream), which the
   call synchronises.  Allocates and frees a small device array.
   *flops_per_s (host) receives the rate (0 on error).  Errors: GR_ERR_ARG,
   GR_ERR_NOMEM, GR_ERR_CUDA. */
gr_status gr_fma_rate(int fp64, long long iters, void *cuda_stream, double *flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* GR_H */
