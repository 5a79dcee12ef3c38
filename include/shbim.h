/*
 * shbim.h -- C ABI of the GB300 boundary-integral operator library.
 *
 * Operators of Sorgentone, Tornberg & Vlahovska, "A 3D boundary integral method for the
 * electrohydrodynamics of surfactant-covered drops": the Laplace layer operators of the
 * leaky-dielectric problem (Eqs. BIE01, E_n, dl_op_laplace), the Stokes single and double
 * layer (Eqs. main_eq, GandT, op_stokes) and their Galerkin projections (Eqs. BIM_galerkin,
 * galerkin_En), discretised with spherical harmonics on Gaussian grids (Section 2), the
 * regular rule (Eq. reg_quadrature) and the rotated-pole singular rule (Eq. mod_weights).
 *
 * Conventions shared by every call
 * --------------------------------
 * Coefficients: real orthonormal spherical harmonics, Condon-Shortley phase,
 *   S_n0 = Pbar_n^0(cos t), S_nm = sqrt2 Pbar_n^m cos(m f), S_n,-m = sqrt2 Pbar_n^m sin(m f),
 *   Pbar_n^m = sqrt((2n+1)/(4 pi) (n-m)!/(n+m)!) P_n^m   (Eqs. normalized_spharm, pneg).
 *   A degree-p scalar field is (p+1)^2 doubles, entry n*n + n + m.
 * Grids: a degree-q grid has q+1 Gauss-Legendre latitudes theta_j = acos(t_j) ordered by
 *   increasing theta, and 2q+2 longitudes phi_k = pi k/(q+1) (Eq. spharm_ex); values are
 *   stored [j][k] row-major, (q+1)(2q+2) doubles per field.
 * Drops: drop i has degree p_i. Its targets are the nodes of its degree-p_i grid; its
 *   quadrature sources are the nodes of its degree q_i = 2 p_i + 1 grid.
 * Multi-drop vectors are concatenated drop-major. A scalar density has (p_i+1)^2 entries
 *   for drop i; a vector density (Stokes) stores its three components component-major
 *   inside each drop: [drop0: x-coefs, y-coefs, z-coefs][drop1: ...].
 *   Target-grid outputs are concatenated the same way, (p_i+1)(2p_i+2) per component.
 * Ownership: every pointer argument named *_dev is device memory owned by the caller and
 *   must stay valid until the work queued on `stream` has finished. *_host arguments are
 *   read before the call returns. The library owns the context, its tables, geometry and
 *   workspaces (allocated with cudaMalloc in shbim_set_drops and freed in shbim_destroy).
 * Streams: every call queues its work on `stream` (a cudaStream_t passed as void*; NULL
 *   means the legacy default stream) and returns without synchronising, except where a
 *   call says it reads results back to the host.
 * Errors: every call returns 0 on success or a negative SHBIM_ERR_* code; the message of
 *   the last failure is returned by shbim_last_error(ctx). No call aborts the process.
 */
#ifndef SHBIM_H
#define SHBIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SHBIM_OK 0
#define SHBIM_ERR_ARG (-1)          /* invalid argument (sizes, null pointers, state) */
#define SHBIM_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define SHBIM_ERR_NOMEM (-3)        /* device allocation failed */
#define SHBIM_ERR_NOT_CONVERGED (-4)/* GMRES hit its iteration limit */
#define SHBIM_ERR_TIMEOUT (-5)      /* a bounded wait inside a kernel ran out (see shbim_set_wait_limit) */
#define SHBIM_ERR_NONFINITE (-6)    /* a NaN or Inf was detected in a reduction */

#define SHBIM_CONTINUE 0            /* shbim_gmres_step: not converged yet */
#define SHBIM_CONVERGED 1           /* shbim_gmres_step: relative residual <= tol */

/* Arithmetic of the all-pairs sums (the singular self rows, the transforms and GMRES are
 * always FP64). */
#define SHBIM_PREC_FP64 0           /* FP64 sums */
#define SHBIM_PREC_FP32_COMP 1      /* FP32 pair arithmetic, positions relative to the drop
                                       centres, compensated (two-sum) accumulation */
#define SHBIM_PREC_DF64 2           /* FP64-class sums in double-float arithmetic on the FP32 pipe:
                                       every quantity is an FP32 pair (value, low part), ~2^-44
                                       relative per operation (Dekker; Knuth two-sum) */

/* Kernels of the Laplace operator (shbim_eval_electric `which`). Both carry 1/(4 pi). */
#define SHBIM_LAPLACE_DL 0          /* L[s](x0) = 1/(4pi) int s(x) (x0-x).n(x0) / r^3 dS  (Eq. E_n) */
#define SHBIM_LAPLACE_SL 1          /* S_L[s](x0) = 1/(4pi) int s(x) / r dS */

/* Output kinds. */
#define SHBIM_OUT_GRID 0            /* values at every target (degree-p grid of each drop) */
#define SHBIM_OUT_COEF 1            /* Galerkin coefficients: forward transform of the values */

/* Transform directions and grids for shbim_sht. */
#define SHBIM_SHT_INVERSE 0         /* coefficients -> grid values (Eq. spharm_ex) */
#define SHBIM_SHT_FORWARD 1         /* grid values -> Galerkin inner products (., Y_nm) */
#define SHBIM_GRID_BASE 0           /* degree-p grid (the targets) */
#define SHBIM_GRID_UP 1             /* degree 2p+1 grid (the quadrature sources) */

/* Linear systems for GMRES. */
#define SHBIM_SYS_ELECTRIC 0        /* 1/2 s - (R-1)/(R+1) sum_j L_j[s] = b       (Eq. galerkin_En) */
#define SHBIM_SYS_STOKES 1          /* (lam_i+1) u - sum_j (lam_j-1) D_j[u] = b   (Eq. main_eq)    */
#define SHBIM_SYS_DIFFUSION 2       /* (I - c Delta_S) G = b on every drop (implicit surfactant
                                       diffusion, Algorithm 1), c set by shbim_set_diffusion;
                                       right-preconditioned by the sphere eigenvalues
                                       1 + c n(n+1)/a_i^2, a_i^2 = area_i / (4 pi) */

typedef struct shbim_ctx shbim_ctx;

typedef struct shbim_opts {
  int precision;        /* SHBIM_PREC_* for the all-pairs sums */
  int gmres_restart;    /* Krylov dimension m before a restart (1..200); 0 -> 50 */
  double gmres_tol;     /* relative residual ||b - A x|| / ||b|| to stop at; 0 -> 1e-8 */
  int gmres_maxiter;    /* total Arnoldi steps allowed; 0 -> 1000 */
  double R;             /* conductivity ratio of the electric system (Eq. EneEni) */
} shbim_opts;

/* Create a context. `opts` may be NULL (defaults: FP64, m = 50, tol 1e-8, R = 1).
 * Returns SHBIM_ERR_ARG for out-of-range options. */
int shbim_create(const shbim_opts* opts, shbim_ctx** out);

/* Destroy a context and free its device memory (synchronises the device first). */
int shbim_destroy(shbim_ctx* ctx);

/* Message of the last failure on this context ("" if none). Valid until the next call. */
const char* shbim_last_error(shbim_ctx* ctx);

/* Change the arithmetic of the all-pairs sums or the electric ratio R after creation. */
int shbim_set_precision(shbim_ctx* ctx, int precision);
int shbim_set_R(shbim_ctx* ctx, double R);

/* Define the drops and build everything that depends only on their shapes:
 * transform tables per distinct degree, target and source geometry (x, outward normal n,
 * area element; Section 1 and Eq. reg_quadrature) and the singular self rows of every
 * kernel (rotated-pole rule, Section 2.1).
 *   n_drops      number of drops (>= 1)
 *   p_host       degree of each drop, 1 <= p <= 64
 *   lambda_host  viscosity ratio of each drop (Eq. main_eq); may be NULL (all 1)
 *   xcoef_dev    position coefficients, per drop 3 (p+1)^2 doubles (x, y, z component-major)
 * Allocates device memory (SHBIM_ERR_NOMEM on failure). Synchronises `stream` on entry,
 * reads the degree-0 position coefficients back to the host (the drop centres) and
 * synchronises again while building; the last kernels it queues on `stream` may still be
 * running when it returns. Replaces any previous drop set of the context. */
int shbim_set_drops(shbim_ctx* ctx, int n_drops, const int32_t* p_host, const double* lambda_host,
                    const double* xcoef_dev, void* stream);

/* Nearly-singular correction (Section 2.1; on by default). When on, shbim_set_drops also finds
 * every target closer than 6 h_j to another drop j's source nodes (h_j = sqrt(area_j / N_s),
 * the spacing of drop j's degree 2p+1 grid) and, for each such pair, builds correction rows
 * so that drop j's contribution there comes from the regular rule on drop j's grid upsampled
 * four times per direction (degree 8p+7) instead of its degree 2p+1 grid. Turning it off or on
 * takes effect at the next shbim_set_drops. shbim_near_pairs returns the number of pairs. */
int shbim_set_near(shbim_ctx* ctx, int on);
int shbim_near_pairs(shbim_ctx* ctx);

/* Closest approach of the current drop set, measured by shbim_set_drops over the near pairs: the
 * smallest distance from a target to another drop's surface, sampled at the nodes of that drop's
 * four-times upsampled grid (at most ~0.2 h_j above the true distance), absolute (*dist_host) and
 * in units of that drop's spacing h_j (*ratio_host); +infinity when there are no near pairs or the
 * correction is off. The upsampled rule is validated down to 1.15 h_j (error ~1e-11 against a
 * sixteen-times upsampled reference); a smaller ratio means targets closer than that. Either pointer
 * may be NULL. */
int shbim_near_min_distance(shbim_ctx* ctx, double* dist_host, double* ratio_host);

/* Sizes of the current drop set: total scalar coefficients sum (p_i+1)^2, total targets
 * sum (p_i+1)(2p_i+2) and total sources sum (q_i+1)(2q_i+2). */
int shbim_sizes(shbim_ctx* ctx, int64_t* ncoef, int64_t* ntarget, int64_t* nsource);

/* Geometry of the targets as built by shbim_set_drops: per target x, y, z, nx, ny, nz and
 * the area element J relative to the unit sphere, each an array of ntarget doubles laid
 * out [x..][y..][z..][nx..][ny..][nz..][J..] (7 * ntarget doubles in out_dev). */
int shbim_target_geometry(shbim_ctx* ctx, double* out_dev, void* stream);

/* Shape of the linear part of the far field (Section 1, Eq. potential): E_inf(x) = E_u + E_q G x with
 * G a symmetric, traceless 3 x 3 matrix (row-major, 9 doubles read from the host), so that E_inf is
 * the gradient of a harmonic potential. The paper's quadrupole field, phi_inf = -E_q r^2 P_2(cos theta),
 * is G = diag(-1, -1, 2), i.e. E_inf = E_q (-x, -y, 2z) (Section 3); the default is diag(1, -1, 0),
 * the planar field E_q (x, -y, 0). SHBIM_ERR_ARG for a non-finite, non-symmetric or non-traceless G
 * (relative tolerance 1e-12). Applies to shbim_electric_rhs, shbim_rates and shbim_step. */
int shbim_set_field_shape(shbim_ctx* ctx, const double* G_host);

/* Form of the FP64-class (SHBIM_PREC_DF64) all-pairs sums. On (default): for pairs of drops whose
 * surfaces are at least 2^(19-Q) apart, positions relative to each drop's centre are split on a
 * power-of-two quantum 2^-Q chosen per geometry (the largest offsets of the layout stay below 2^(23-Q))
 * so that coordinate differences are exact in FP32, and the rest of each kernel term is double-float
 * arithmetic (about 2^-42 relative per term, fewer instructions per pair); closer pairs, and every
 * pair when off, use the general double-float form (about 2^-45 per term). */
int shbim_set_quantized_pairs(shbim_ctx* ctx, int on);

/* Equation of state of the surfactant (Section 1) used by shbim_rates, shbim_stokes_rhs and
 * shbim_step: SHBIM_EOS_LANGMUIR (default), the Langmuir law of Eq. langmuir normalised so that
 * gamma(1) = 1, with shbim_phys.beta and x_s; or SHBIM_EOS_LINEAR, the linear law
 * gamma = 1 + beta_t (1 - Gamma) (Eq. lin_eq_state, tension normalised on its equilibrium value), with
 * shbim_phys.beta read as the elasticity beta_t (x_s unused). SHBIM_ERR_ARG for any other value. */
#define SHBIM_EOS_LANGMUIR 0
#define SHBIM_EOS_LINEAR 1
int shbim_set_equation_of_state(shbim_ctx* ctx, int law);

/* Right-hand side of the electric system (Eq. galerkin_En): Galerkin coefficients of
 * R/(R+1) E_inf . n on every drop, for the far field E_inf(x) = E_u + E_q G x
 * (a uniform part E_u, a 3-vector read from the host, plus a linear field of strength E_q whose
 * shape G is the context's, shbim_set_field_shape).
 *   out_dev   ncoef coefficients */
int shbim_electric_rhs(shbim_ctx* ctx, const double* E_u_host, double E_q, double* out_dev,
                       void* stream);

/* Spherical-harmonic transforms of n_fields scalar fields, each on the drop that field_drop names
 * (Section 2: the expansion of Eq. spharm_ex and the Galerkin inner products (., Y_nm) by the regular
 * rule of Eq. reg_quadrature on that drop's grid). FP64.
 *   dir            SHBIM_SHT_INVERSE: coefficients -> grid values; SHBIM_SHT_FORWARD: grid values ->
 *                  Galerkin inner products
 *   grid           SHBIM_GRID_BASE (degree p of the field's drop) or SHBIM_GRID_UP (degree 2p+1)
 *   field_drop_host n_fields drop indices; field f has (p_d+1)^2 coefficients and (q+1)(2q+2) grid
 *                  values of its drop d = field_drop_host[f] and grid degree q
 *   in_dev, out_dev the fields concatenated in order: coefficients (inverse input, forward output)
 *                  or grid values (inverse output, forward input), each field's block after the
 *                  previous one's; must not alias
 * SHBIM_ERR_ARG for a drop index out of range, a bad direction or grid, or null pointers with
 * n_fields > 0. Consecutive fields of one drop are transformed by one launch. */
int shbim_sht(shbim_ctx* ctx, int dir, int grid, int n_fields, const int32_t* field_drop_host,
              const double* in_dev, double* out_dev, void* stream);

/* Laplace layer operator of the electric problem applied to a scalar density on all drops:
 * for every target x0 on drop i, sum over drops j of the kernel `which` integrated over
 * S_j -- the regular rule (Eq. reg_quadrature) on the degree-q source grid for j != i and
 * the rotated-pole singular rule (Eq. mod_weights) for j == i.
 *   dens_dev   sum_i (p_i+1)^2 coefficients
 *   out_dev    SHBIM_OUT_GRID: ntarget values; SHBIM_OUT_COEF: ncoef Galerkin coefficients */
int shbim_eval_electric(shbim_ctx* ctx, int which, const double* dens_dev, double* out_dev,
                        int out_kind, void* stream);

/* Stokes layer operators (Eqs. op_stokes, GandT) on all drops:
 *   out = sum_j S_j[f_j] + sum_j (lam_j - 1) D_j[u_j]
 * with the same regular / singular split as shbim_eval_electric.
 *   f_dev, u_dev  vector densities, 3 sum_i (p_i+1)^2 coefficients each; either may be
 *                 NULL (that term is omitted), not both
 *   out_dev       SHBIM_OUT_GRID: 3 ntarget values; SHBIM_OUT_COEF: 3 ncoef coefficients */
int shbim_eval_stokes(shbim_ctx* ctx, const double* f_dev, const double* u_dev, double* out_dev,
                      int out_kind, void* stream);

/* GMRES on one of the Galerkin systems (the paper does not name its solver; this is
 * restarted GMRES with classical Gram-Schmidt applied twice, in FP64).
 * shbim_gmres_begin: set up the system `sys` with right-hand side rhs_dev (length n = ncoef
 *   for SHBIM_SYS_ELECTRIC and SHBIM_SYS_DIFFUSION, 3 ncoef for SHBIM_SYS_STOKES) and initial
 *   guess x0_dev (NULL means zero); computes the initial residual (reads one norm back to the
 *   host). The diffusion system iterates on y = M x internally; x0_dev and x_dev are x.
 * shbim_gmres_step: one Arnoldi step (one operator application), restarting when the
 *   Krylov space is full; reads the new column's norms back to the host and returns
 *   SHBIM_CONTINUE, SHBIM_CONVERGED, or SHBIM_ERR_NOT_CONVERGED after gmres_maxiter steps.
 *   *resid_host (may be NULL) receives the current relative residual estimate.
 * shbim_gmres_finish: write the solution to x_dev (length n) and return the number of
 *   Arnoldi steps taken in *iters_host (may be NULL).
 * shbim_gmres_solve: begin + step until converged + finish; also reports the final true
 *   relative residual ||b - A x|| / ||b|| in *resid_host. */
int shbim_gmres_begin(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev,
                      void* stream);
/* Convergence control of shbim_gmres_solve (and of the solves inside shbim_gmres_solve_refined,
 * shbim_rates and shbim_step) on the device (on by default, with CUDA graphs on): after the first
 * Arnoldi step, each GMRES cycle is one CUDA graph whose conditional 'while' node repeats the Arnoldi
 * step -- operator application, classical Gram-Schmidt twice, normalisation, Givens rotation and the
 * residual test, all in kernels -- until the residual estimate reaches the tolerance, the Krylov space is
 * full or gmres_maxiter steps were taken; the least-squares update of x follows in the same graph. The
 * host synchronises once per cycle instead of once per step. Off, or where the graph cannot be built:
 * every step on the host as shbim_gmres_step. Both give the same iterates up to rounding. */
int shbim_set_device_gmres(shbim_ctx* ctx, int on);
/* Right preconditioner of the Stokes system (SHBIM_SYS_STOKES), on by default. Per drop i, with
 * Q_i an orthonormal basis (coefficient inner product) of its six rigid-body motions (translations,
 * and rotations e_k x x of its current shape) and r_i the radial field of the parameter sphere
 * orthogonalised against them:
 *   P_i^{-1} v = v/(lam_i+1) + (1/2 - 1/(lam_i+1)) Q_i Q_i^T v + (1/(2 lam_i) - 1/(lam_i+1)) r_i r_i^T v.
 * On a closed surface the double layer reproduces rigid motions (Eq. main_eq's self part maps them to
 * 2 u) and on a sphere maps the normal field to -1 times itself (self part 2 lam_i u); all other modes
 * of the self part lie near lam_i + 1, so P^{-1} clusters the spectrum at 1 and GMRES needs fewer steps
 * for drops of large or small viscosity ratio. GMRES iterates y = P x on A P^{-1}; solutions, residual
 * checks and the refinement's residuals are those of the system itself. Rebuilt with every geometry
 * (FP64, on the host: 7 vectors of 3 (p+1)^2 per drop). Off: plain GMRES. */
int shbim_set_stokes_preconditioner(shbim_ctx* ctx, int on);
int shbim_gmres_step(shbim_ctx* ctx, double* resid_host, void* stream);
int shbim_gmres_finish(shbim_ctx* ctx, double* x_dev, int* iters_host, void* stream);
int shbim_gmres_solve(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev,
                      double* x_dev, int* iters_host, double* resid_host, void* stream);

/* Physical parameters of the drop problem (Section 1).
 * E_n is solved with R; the traction uses Q and R (Eq. el_force, eps = 1); the capillary
 * force is scaled by 1/Ca_E (Eq. main_eq); the tension follows the Langmuir law normalised so
 * that gamma(1) = 1, gamma = (1 + beta ln(1 - x_s Gamma)) / (1 + beta ln(1 - x_s))
 * (Eq. langmuir; beta = 0 is a clean drop), or the linear law with beta as its elasticity
 * (shbim_set_equation_of_state). The far field is E_u + E_q G x, G the context's field
 * shape (shbim_set_field_shape).
 * inner_tol is the FP32 inner tolerance of the refined solves used when the context's
 * precision is SHBIM_PREC_FP32_COMP (otherwise plain FP64 GMRES). */
typedef struct shbim_phys {
  double R, Q, Ca_E;
  double beta, x_s;
  double E_u[3];
  double E_q;
  double inner_tol;
  double Pe;            /* surfactant Peclet number; 0 or infinity: no diffusion */
} shbim_phys;

/* Velocity and surfactant rate for the current drop shapes (steps i-vi of Section 1):
 * solves for E_n, forms E_t = -grad_S(phi_inf + S_L[(1-1/R) E_n]), the electric and
 * interfacial forces on each drop's degree 2p+1 grid (products de-aliased by projection to
 * degree p), solves the Stokes system with right-hand side -sum_j S_j[f/Ca_E - f^E] and forms
 * the surfactant rate -Gamma div_S u of nodes that move with u (Eq. surfactant0, material
 * form, no diffusion; Pe is not used here).
 *   gamma_dev  ncoef coefficients of Gamma
 *   u_dev      3 ncoef velocity coefficients (out);  gE_dev  ncoef rate coefficients (out)
 *   iters_host GMRES iterations of the electric and Stokes solves (2 ints, may be NULL)
 * Synchronises `stream` (GMRES reads residuals back). */
int shbim_rates(shbim_ctx* ctx, const shbim_phys* phys, const double* gamma_dev, double* u_dev,
                double* gE_dev, int* iters_host, void* stream);

/* Right-hand side of the Stokes system for given E_n coefficients (steps ii-v of Section 1):
 * the charge potential phi_q = S_L[(1 - 1/R) E_n], E_t = -grad_S(phi_inf + phi_q), the electric and
 * interfacial tractions (Eqs. el_force, interfacial_force, langmuir) on each drop's degree 2p+1 grid
 * (projected to degree p) and rhs = -sum_j S_j[f/Ca_E - f^E] (Eq. main_eq) -- what shbim_rates solves
 * the Stokes system with. The one-shot applications use the context's precision (in FP32_COMP mode its
 * one-shot precision). gamma_dev, En_dev: ncoef coefficients; rhs_dev: 3 ncoef (out). */
int shbim_stokes_rhs(shbim_ctx* ctx, const shbim_phys* phys, const double* gamma_dev, const double* En_dev,
                     double* rhs_dev, void* stream);

/* Surface Laplacian Delta_S (Laplace-Beltrami operator, the diffusion term of Eq. surfactant0)
 * of a scalar on every drop of the current shapes, in Galerkin form:
 * Delta_S f = g^{ab} (f_ab - Gamma^c_ab f_c) in the (theta, phi) chart, formed on each drop's
 * degree 2p+1 grid and projected to degree p by the regular rule.
 *   coef_dev, out_dev  ncoef coefficients each (device, caller-owned, must not alias) */
int shbim_laplace_beltrami(shbim_ctx* ctx, const double* coef_dev, double* out_dev, void* stream);
/* Coefficient c >= 0 of the diffusion system SHBIM_SYS_DIFFUSION, (I - c Delta_S) G = b
 * (SHBIM_ERR_ARG for negative or non-finite c). shbim_step sets it to dt / (2 Pe). */
int shbim_set_diffusion(shbim_ctx* ctx, double c);

/* One time step of Algorithm 1 (midpoint rule for x, IMEX stages for Gamma):
 * rates at (x, Gamma), half step, rates at the half step, full step
 *   x_out = x + dt u(t+dt/2),  Gamma_out = Gamma + dt g_E(t+dt/2),
 * and the error estimate err = dt max(|u(t+dt/2) - u(t)|, |g_E(t+dt/2) - g_E(t)|) (grid max
 * norms on the degree-p grids), i.e. the distance to the explicit Euler step. The drop layout
 * must have been set with shbim_set_drops; x_dev (3 ncoef) replaces the shapes. Outputs must
 * not alias the inputs, so the caller can reject the step (adaptive dt: accept if err < tol,
 * then dt <- dt (0.9 tol / err)^(1/2)). iters_host: 4 GMRES counts (may be NULL).
 * With 0 < Pe < infinity the surfactant follows the IMEX scheme of Algorithm 1: the half step
 * solves (I - dt/(2 Pe) Delta_S) Gamma_half = Gamma + dt/2 g_E(t) on the half-step surface and
 * the full step uses g_E(t+dt/2) + Delta_S Gamma_half / Pe.
 * The Stokes solve of the second stage starts from the first stage's velocity (the two differ by
 * O(dt)); every other solve starts from zero.
 * After the call the context holds the geometry of the half step. */
int shbim_step(shbim_ctx* ctx, const shbim_phys* phys, const double* x_dev, const double* gamma_dev,
               double dt, double* x_out_dev, double* gamma_out_dev, double* err_host, int* iters_host,
               void* stream);

/* Reparametrisation of the drop surfaces (Section 2.2: applied after every accepted step of
 * Algorithm 1 to keep the spherical-harmonic representation resolved). The paper builds it on an
 * optimisation of the node distribution and does not restate it; this library takes `steps` explicit
 * steps of the tangential gradient flow of the spectral energy E = sum_{n>=1,m} n^a |x_nm|^2 (three
 * components), each on every drop's degree 2p+1 grid:
 *   h = sum n^a x_nm S_nm,  t = h - (h . n) n,  x <- x - tau t,  tau = c / p^a,
 * projected back to degree p by the regular rule; the nodes move along the surface, which stays in
 * place to first order in tau per step. The surfactant concentration moves with the nodes:
 *   Gamma <- Gamma - tau grad_S Gamma . t   (then projected to degree p).
 *   steps       number of flow steps, 0..100000 (0: only the energy is computed)
 *   a           energy exponent, 0 <= a <= 8 (4 is usual);  c  step factor, 0 < c <= 1 (stable range)
 *   x_dev       3 ncoef position coefficients in the context's layout (device, in/out)
 *   gamma_dev   ncoef concentration coefficients (device, in/out) or NULL; must not overlap x_dev
 *   energy_host steps+1 doubles (host, out) or NULL: E before the first and after every step
 * Works in FP64 on the drop layout of shbim_set_drops and leaves the context's geometry as it was
 * (the next shbim_set_drops or shbim_step takes the new positions). SHBIM_ERR_ARG for arguments
 * outside these ranges or no drops set. Synchronises `stream`. */
int shbim_reparametrize(shbim_ctx* ctx, int steps, double a, double c, double* x_dev, double* gamma_dev,
                        double* energy_host, void* stream);

/* FP64-class arithmetic used where mixed precision needs it: the residuals of
 * shbim_gmres_solve_refined in SHBIM_PREC_FP32_COMP mode. SHBIM_PREC_DF64 (default: double-float on
 * the FP32 pipe) or SHBIM_PREC_FP64 (native); SHBIM_ERR_ARG otherwise. */
int shbim_set_outer_precision(shbim_ctx* ctx, int precision);

/* Arithmetic of the one-shot layer-operator applications of shbim_rates / shbim_step in
 * SHBIM_PREC_FP32_COMP mode (the charge potential S_L[q] and the Stokes right-hand side
 * S[f/Ca_E - f^E], applied once each and not iterated by GMRES): SHBIM_PREC_DF64 (default) or
 * SHBIM_PREC_FP64 give FP64-class results; SHBIM_PREC_FP32_COMP is faster but its ~1e-7 relative error
 * of S[f/Ca_E - f^E] is amplified in u and its surface divergence, because the single layer of the
 * capillary traction nearly cancels over each drop (a sphere under uniform tension does not move):
 * measured ~1e-5 relative in the surfactant rate of two p = 6 drops. SHBIM_ERR_ARG otherwise. */
int shbim_set_oneshot_precision(shbim_ctx* ctx, int precision);

/* Mixed-precision solve by iterative refinement: every outer step forms the residual
 * r = b - A x with FP64-class all-pairs sums, solves A d = r by GMRES with FP32 compensated sums,
 * and updates x += d, until the FP64-class relative residual reaches gmres_tol or max_outer steps
 * were taken (SHBIM_ERR_NOT_CONVERGED). The inner relative tolerance is inner_tol (e.g. 1e-5),
 * except where the step can finish the solve: then it is 0.5 gmres_tol / (current relative
 * residual), looser than inner_tol on the last step. The first inner solve aims at 0.5 gmres_tol at
 * once (one FP64-class residual per solve) for as long as that has succeeded for the system on this
 * context; after the first miss the system's later solves use the two-step form. With an initial guess
 * x0 the first residual b - A x0 is formed with the FP32 operator (the first inner solve cannot get
 * below the FP32 operator's accuracy anyway), so a guess adds no FP64-class residual: the solve takes
 * as many of them as from a zero start, and fewer inner steps when the guess is good. The outer residuals use the
 * context's outer precision (shbim_set_outer_precision).
 * Only the electric and Stokes systems (the diffusion system has no all-pairs sums;
 * SHBIM_ERR_ARG). The context's precision setting is restored on return. Reports the total inner Arnoldi
 * steps, the outer steps and the final FP64 relative residual (each pointer may be NULL). */
int shbim_gmres_solve_refined(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev,
                              double* x_dev, double inner_tol, int max_outer, int* inner_iters_host,
                              int* outer_iters_host, double* resid_host, void* stream);

/* Allocation-free Laplace pair sum, for callers that cannot allocate device memory when they call
 * it -- for example a host application that reserves all of its device memory up front and hands
 * out only fixed buffers, or code running where a cudaMalloc would block or fail. The paper has no
 * counterpart: this is a service variant of the FP64 all-pairs kernel.
 * Computes, for every target t, out[t] = 1/(4 pi) sum_s K(x_t, x_s) s_s over ALL sources (no
 * pair is excluded), with K = (x_t - x_s).n_t / r^3 for SHBIM_LAPLACE_DL and 1/r for
 * SHBIM_LAPLACE_SL, in FP64. Keeping targets and sources apart is the caller's task: a source
 * that coincides with a target (r = 0) makes that target's sum infinite (SL) or NaN (DL).
 *   tgt_dev   6 * n_tgt doubles: [x..][y..][z..][nx..][ny..][nz..] (normals unused for SL)
 *   src_dev   4 * n_src doubles: [x..][y..][z..][s..] with s the source strength
 *             (density times quadrature weight)
 *   out_dev   n_tgt doubles
 * The C ABI cannot see the sizes of the arrays behind the pointers: they must hold the counts
 * above (the Python binding checks its tensors).
 * Needs no context and calls no allocator: its partial sums live in one fixed array of
 * 2^21 doubles (16 MiB) in device memory, which every GPU that loads the library holds
 * until the process exits. Hence n_tgt must not exceed 2^21 (2097152); larger sizes return
 * SHBIM_ERR_ARG, as do a bad `which` or null pointers. The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it per device. All calls share
 * the array: calls whose work overlaps on the GPU (different streams, or different host
 * threads) race on it and must be serialised by the caller. Nothing in the array needs to start
 * at zero (every slot read is written by the same call). An error already pending on the device
 * when the call starts is reported as SHBIM_ERR_CUDA without launching anything. Returns 0,
 * SHBIM_ERR_ARG or SHBIM_ERR_CUDA. */
int shbim_pairs_laplace_noalloc(int which, const double* tgt_dev, int64_t n_tgt, const double* src_dev,
                                int64_t n_src, double* out_dev, void* stream);

/* ---- Learned warm start (an addition to the paper's method: the network only proposes an
 * initial guess; GMRES solves to its tolerance from there, so the residual test decides the error).
 * A multilayer perceptron h_l = tanh(bf16(h_{l-1}) bf16(W_l)^T + b_l) with a linear last
 * layer, bfloat16 weights (FP32 master copy) and FP32 accumulation on the tensor cores.
 *   widths      n_layers + 1 sizes (input, hidden..., output); max_batch rows per call
 *   W_host      [w_{l+1}][w_l] row-major FP32, b_host [w_{l+1}] (set: also resets Adam)
 *   x_dev/y_dev/t_dev  FP32 row-major [batch][width] device arrays
 * shbim_mlp_train_step: forward, loss sum (y - t)^2 / (2 batch) (read back into *loss_host
 *   when not NULL, which synchronises `stream`), backward, and, if update != 0, one Adam step
 *   (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr. Gradients stay readable through
 *   shbim_mlp_get_layer.
 * shbim_electric_warm_start: initial guess for the electric system from the drop shapes,
 *   x0 = 3(R+1)/(R+2) rhs + net(xcoef as FP32), i.e. the sphere solution E_n = 3R/(R+2) E.n
 *   (written through the right-hand side) plus the learned correction. The network must map
 *   3 ncoef inputs to ncoef outputs. */
typedef struct shbim_mlp shbim_mlp;
int shbim_mlp_create(int n_layers, const int32_t* widths, int max_batch, shbim_mlp** out);
int shbim_mlp_destroy(shbim_mlp* net);
int shbim_mlp_set_layer(shbim_mlp* net, int layer, const float* W_host, const float* b_host);
/* Optional input standardisation x_n = (x - shift) * scale, per input feature, applied in FP32
 * before the first bfloat16 rounding (NULL pointers remove it). */
int shbim_mlp_set_input_affine(shbim_mlp* net, const float* shift_host, const float* scale_host);
int shbim_mlp_get_layer(shbim_mlp* net, int layer, float* W_host, float* b_host, float* gW_host,
                        float* gb_host);
int shbim_mlp_forward(shbim_mlp* net, int batch, const float* x_dev, float* y_dev, void* stream);
int shbim_mlp_train_step(shbim_mlp* net, int batch, const float* x_dev, const float* t_dev, float lr,
                         int update, double* loss_host, void* stream);
int shbim_electric_warm_start(shbim_ctx* ctx, shbim_mlp* net, const double* xcoef_dev,
                              const double* rhs_dev, double* x0_dev, void* stream);

/* Learned initial guesses for both solves of shbim_rates (an extension of the method: the network only
 * proposes, GMRES solves to its tolerance from there).
 * shbim_warm_start_features: the network's input for the current drop set, FP32, laid out
 *   [position coefficients, 3 ncoef][Gamma coefficients, ncoef][E_u (3), E_q][lambda per drop][R, Q, Ca_E],
 *   shbim_warm_start_feature_count(ctx) = 4 ncoef + 7 + n_drops values (-1 without drops).
 * shbim_learned_guess: y = net(features) with 4 ncoef outputs; writes the electric guess
 *   E_n0 = 3(R+1)/(R+2) rhs_e + y[0, ncoef) (the sphere solution 3R/(R+2) E.n through the right-hand side
 *   plus the learned correction) to En0_dev and the velocity guess u0 = y[ncoef, 4 ncoef) to u0_dev;
 *   either output may be NULL (rhs_e_dev is needed only for E_n0). SHBIM_ERR_ARG if the network's widths
 *   do not match.
 * shbim_set_warm_start: a network that shbim_rates and shbim_step use for these guesses (NULL: none;
 *   the context does not own it). In the mixed-precision solves a guess costs no extra FP64-class
 *   residual while the system's FP32 operator allows finishing in one step (shbim_gmres_solve_refined). */
int64_t shbim_warm_start_feature_count(shbim_ctx* ctx);
int shbim_warm_start_features(shbim_ctx* ctx, const double* xcoef_dev, const double* gamma_dev,
                              const shbim_phys* phys, float* feat_dev, void* stream);
int shbim_learned_guess(shbim_ctx* ctx, shbim_mlp* net, const float* feat_dev, const double* rhs_e_dev,
                        double* En0_dev, double* u0_dev, void* stream);
int shbim_set_warm_start(shbim_ctx* ctx, shbim_mlp* net);

/* Number of kernel launches the library has queued since the context was created. */
int64_t shbim_launch_count(shbim_ctx* ctx);

/* CUDA graphs for the operator applications inside GMRES (on by default): for each geometry,
 * system and precision the second application is captured on a stream owned by the library
 * and later ones replay it on the caller's stream, with the Krylov vector copied through fixed
 * staging buffers. Kernel timing (shbim_set_timing) does not see inside a replay. If a capture
 * fails, the context falls back to direct launches. */
int shbim_set_graphs(shbim_ctx* ctx, int on);

/* Concurrency on a second stream owned by the library (on by default):
 * - inside one operator application (two or more drops): the singular self rows and the
 *   near-field correction run on the side stream while the caller's stream synthesises the source
 *   strengths and runs the all-pairs sums, which are added into the output after the two branches
 *   join; the order in which the three contributions are added differs from the serial order,
 *   which changes results only by rounding;
 * - in the double-float singular-row build (two or more chunks of targets): every other chunk runs
 *   on the side stream with its own work buffers (the same rows, bit for bit).
 * The side stream waits for everything queued earlier on the caller's stream and the caller's
 * stream waits for the side stream before the call's last kernels, so each call behaves as if it
 * ran on the caller's stream alone. Off: everything on the caller's stream. */
int shbim_set_concurrency(shbim_ctx* ctx, int on);

/* Launch-shape autotuning of the FP32 all-pairs kernels (on by default): on the first launch of
 * each kernel kind for a drop layout, every register blocking (1, 2 or 4 targets per thread)
 * with source-split counts around the layout's default is timed and the fastest kept. The shape
 * changes the FP32 summation order, so two contexts may differ at rounding level; with the
 * autotuner off every layout uses 1 target per thread and the default split count, which makes
 * FP32 results reproducible across contexts. Takes effect immediately. */
int shbim_set_autotune(shbim_ctx* ctx, int on);

/* Arithmetic of the singular-row build (Section 2.1; once per geometry, at the next
 * shbim_set_drops): SHBIM_PREC_DF64 (default: double-float on the FP32 pipe, FP64-class rows) or
 * SHBIM_PREC_FP64 (native). SHBIM_ERR_ARG otherwise. */
int shbim_set_rows_precision(shbim_ctx* ctx, int precision);

/* Arithmetic of the singular self-row application (a GEMV with the stored rows) when the context's
 * precision is SHBIM_PREC_FP32_COMP: SHBIM_PREC_DF64 (default) reads both FP32 planes of the rows and
 * of the density and accumulates in double-float, so the self term, which is of the size of the whole
 * operator value, carries FP64-class accuracy (the rows are HBM-bound: twice the bytes of the
 * alternative); SHBIM_PREC_FP32_COMP reads the high planes only and accumulates in FP32 (~1e-7
 * relative). The other precisions always use the double-float form. SHBIM_ERR_ARG otherwise. */
int shbim_set_self_precision(shbim_ctx* ctx, int precision);

/* Tensor-core stages of the double-float row build (at the next shbim_set_drops), a bit mask:
 * SHBIM_TC_FOURIER, the GEMM of the rows' weights with the DFT table; SHBIM_TC_LEGENDRE, the
 * Legendre stage that follows it (used only together with SHBIM_TC_FOURIER); SHBIM_TC_ROTATION,
 * the pole rotations, one GEMM per latitude and degree. The Fourier and Legendre stages apply for
 * drops of degree p <= 39; the rotations for degrees n <= 39 of drops up to p = 52 (the higher degrees
 * of such a drop, and every degree beyond, run on the FP32 pipe). They split their operands into
 * bfloat16 digits whose products accumulate exactly (error ~2^-40 of the sum of magnitudes per
 * output). A stage that is off, or does not fit, runs as the double-float FP32-pipe kernel. Default
 * SHBIM_TC_ALL (the tensor-core Legendre stage measures as fast as the FP32-pipe one); any other bit is
 * SHBIM_ERR_ARG. */
#define SHBIM_TC_FOURIER 1
#define SHBIM_TC_ROTATION 2
#define SHBIM_TC_LEGENDRE 4
#define SHBIM_TC_ALL 7
int shbim_set_tensor_cores(shbim_ctx* ctx, int mask);

/* Limit of every bounded wait inside the library's kernels, in seconds (1e-3 .. 60; default 1).
 * The tensor-core kernels of the singular-row build and the network wait on shared-memory
 * barriers for their bulk copies and tensor-core products; a kernel whose wait runs out stops
 * issuing work, lets the copies and products it has in flight land (each such wait bounded by 2 s),
 * frees its tensor memory and returns, and the call that launched it returns SHBIM_ERR_TIMEOUT with
 * the context still usable. (The network's GEMM has a fixed 1 s limit and marks a timed-out tile
 * with NaN.) Takes effect at the next launch. */
int shbim_set_wait_limit(shbim_ctx* ctx, double seconds);

/* Check of the bounded-wait path (a diagnostic; the paper has no counterpart): one thread waits on
 * a fresh shared-memory barrier with the context's wait limit. arrive != 0: the barrier's one
 * expected arrival is made first and the call returns 0. arrive == 0: nothing arrives, the wait
 * runs out after the limit and the call returns SHBIM_ERR_TIMEOUT. No copy or product is in flight
 * during the wait. Allocates a 4-byte flag; synchronises `stream`. */
int shbim_check_wait(shbim_ctx* ctx, int arrive, void* stream);

/* Pipe throughput probes (a measurement utility for roofline denominators; the paper has no
 * counterpart). Launches 4 CTAs of 256 threads per SM on the current device, each thread running
 * 8 independent dependency chains of one instruction for `iters` outer iterations, once to warm
 * up and once timed with CUDA events on `stream`; synchronises the stream. Writes the achieved
 * rate to *ops_per_s_host (flop/s for the FMA and MMA kinds, reciprocal square roots per second
 * for SHBIM_PROBE_RSQRT) and the timed duration to *ms_host (may be NULL). Allocates and frees a
 * small device buffer. SHBIM_ERR_ARG for a bad kind or iters < 1. */
#define SHBIM_PROBE_FFMA 0       /* FP32 fma */
#define SHBIM_PROBE_DFMA 1       /* FP64 fma */
#define SHBIM_PROBE_RSQRT 2      /* MUFU reciprocal square root, FP32 */
#define SHBIM_PROBE_HMMA_BF16 3  /* mma.sync m16n8k16 bf16 x bf16 -> f32 */
#define SHBIM_PROBE_DMMA_F64 4   /* mma.sync m8n8k4 f64 */
int shbim_probe_peak(int kind, int64_t iters, double* ops_per_s_host, double* ms_host, void* stream);

/* Launch shape of the FP32 all-pairs kernel of one kind (0 Laplace DL, 1 Laplace SL, 2 Stokes S[f] and
 * D[u] together, 3 Stokes S[f] alone, 4 Stokes D[u] alone; shbim_eval_stokes picks 2, 3 or 4 from the
 * densities it is given, and the single-term kinds skip the other term's arithmetic)
 * for the current layout. shbim_pair_shape writes targets per thread and the split count (either
 * pointer may be NULL) and returns 1 once the shape is fixed (tuned or set), 0 before, or an
 * error code. shbim_set_pair_shape fixes it (tpt in {1, 2, 4}, 1 <= splits <= the layout's
 * capacity, SHBIM_ERR_ARG otherwise) until the next shbim_set_drops with a new layout; it lets
 * a caller reuse a shape tuned earlier. */
int shbim_pair_shape(shbim_ctx* ctx, int kind, int* tpt_host, int* splits_host);
int shbim_set_pair_shape(shbim_ctx* ctx, int kind, int tpt, int splits);

/* Launch form of the FP32 all-pairs kernel of one kind: one CTA per work unit (a sub-tile of up to
 * 512 targets of one drop x one source split; 0) or persistent CTAs, as many as are resident,
 * taking units from an atomic counter in the order of the tile list, largest work first (1).
 * Autotuning tries both. shbim_pair_queue returns the form (or an error code);
 * shbim_set_pair_queue fixes it, like shbim_set_pair_shape. The counter lives in the context and
 * is back at zero after every launch, so launches of one context must not overlap on the GPU
 * (the library queues them on one stream). */
int shbim_pair_queue(shbim_ctx* ctx, int kind);
int shbim_set_pair_queue(shbim_ctx* ctx, int kind, int on);

/* Number of layer-operator applications (calls of the electric or Stokes operator, including
 * those made inside GMRES and the time step) since the context was created. */
int64_t shbim_operator_applications(shbim_ctx* ctx);

/* Kernel timing (measurement support, off by default). When on, the library brackets every
 * launch of the timed kernel classes below with CUDA events on the launching stream; launches
 * inside a replayed CUDA graph (the GMRES operator applications, see shbim_set_graphs) are not
 * bracketed. shbim_kernel_stats synchronises the device and returns the summed milliseconds and
 * the number of bracketed launches of one class since timing was (re)enabled. */
#define SHBIM_K_SELF_WEIGHTS 0      /* rotated-grid synthesis + kernel weights (singular rows) */
#define SHBIM_K_SELF_ANALYSIS 1     /* analysis of the weights (singular rows) */
#define SHBIM_K_PAIRS 2             /* all-pairs sums in FP32 (compensated) */
#define SHBIM_K_SELF_GEMV 3         /* application of the singular rows */
#define SHBIM_K_SHT 4               /* transforms of densities and outputs */
#define SHBIM_K_SELF_ROTATION 5     /* pole rotations of the singular-row build */
#define SHBIM_K_PAIRS_FP64CLASS 6   /* all-pairs sums in double-float or FP64 */
#define SHBIM_K_NEAR 7              /* nearly-singular corrections (upsampled sums at near targets) */
#define SHBIM_K_COUNT 8
int shbim_set_timing(shbim_ctx* ctx, int on);
int shbim_kernel_stats(shbim_ctx* ctx, int kernel_class, double* ms_host, int64_t* launches_host);
/* Algorithmic work of the bracketed launches of one class since timing was (re)enabled, in
 * floating-point operations of the method's formulas (an add or a multiply is 1, a fused
 * multiply-add 2, a reciprocal square root 1), whatever arithmetic the kernel uses to carry them out:
 * for the all-pairs classes, target-source pairs of other drops times the operations of one kernel
 * term (Laplace single layer 11, target-normal double layer 19, Stokeslet 29, stresslet 30, both
 * Stokes terms 42); 0 for the other classes. Synchronises the device like shbim_kernel_stats. */
int shbim_kernel_work(shbim_ctx* ctx, int kernel_class, double* flops_host);

#ifdef __cplusplus
}
#endif
#endif /* SHBIM_H */
