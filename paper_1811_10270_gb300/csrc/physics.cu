// Forces, surfactant rate and the midpoint time step (Section 1 steps i-viii, Algorithm 1).
//
// rates(): for the current drop shapes and a surfactant distribution Gamma,
//   (i)   solve the electric system for E_n (Eq. galerkin_En);
//   (ii)  phi_q = S_L[q] with the charge q = (1 - 1/R) E_n (jump of E_n, Eq. EneEni);
//   (iii) on each drop's upsampled grid: E_t = -grad_S(phi_inf + phi_q) (Eq. E_t),
//   (iv)  electric traction f^E (Eq. el_force, eps = 1),
//   (v)   Langmuir tension normalised to gamma(1) = 1 (Eq. langmuir) and the interfacial force
//         f = 2 gamma H n - grad_S gamma (Eq. interfacial_force), H = 1/2 div_S n;
//   then projects f/Ca_E - f^E to degree p (de-aliasing: products formed on the 2p+1 grid),
//   (vi)  solves the Stokes system with right-hand side -sum_j S_j[f/Ca_E - f^E] (Eq. main_eq),
//   and forms the surfactant rate -Gamma div_S u for nodes moving with u (Eq. surfactant0 in
//   material form, no diffusion), projected to degree p.
// step(): midpoint rule for x with the IMEX stages for Gamma (Algorithm 1):
//   half step with the rates at t, full step with the rates at t + dt/2; the error estimate is
//   dt times the grid max-norm of the difference between the two rates (the distance between
//   the midpoint and the explicit Euler step). With a finite Peclet number the half step is
//   implicit in the surfactant diffusion on the half-step surface,
//   (I - dt/(2 Pe) Delta_S) Gamma_half = Gamma + dt/2 g_E(t), and the full-step rate adds
//   Delta_S Gamma_half / Pe.
// laplace_beltrami(): Delta_S f = g^{ab} (f_ab - Gamma^c_ab f_c) in the (theta, phi) chart with
//   Gamma^c_ab = g^{cd} x_d . x_ab, formed on the degree 2p+1 grid and projected to degree p.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace shbim {

int sht_synth_scaled(shbim_ctx* ctx, const GridTables& g, int n_items, const double* coef,
                     int64_t coef_stride, double* out, int64_t item_stride, const double* scale,
                     double alpha, float* out32, cudaStream_t s);

namespace {

struct PhysDev {
  double R, Q, Ca_E, beta, x_s, eu0, eu1, eu2, eq, lnorm;
  double g[6];   // field shape (xx, xy, xz, yy, yz, zz): E_inf = E_u + eq G x
  int eos;       // SHBIM_EOS_LANGMUIR or SHBIM_EOS_LINEAR (beta read as the elasticity beta_t)
};

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// position derivatives of node i on the upsampled grid (xup layout [c][kind][ns])
struct Frame {
  double x[3], xt[3], xp[3], n[3];
  double E, F, G, det, H;
};

__device__ __forceinline__ Frame frame_at(const double* __restrict__ xup, int64_t ns, int64_t i) {
  Frame f;
  double xtt[3], xtp[3], xpp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* b = xup + (int64_t)c * kNumTab * ns;
    f.x[c] = b[i];
    f.xt[c] = b[ns + i];
    xtt[c] = b[3 * ns + i];
    xtp[c] = b[4 * ns + i];
    xpp[c] = b[5 * ns + i];
    f.xp[c] = b[6 * ns + i];
  }
  const double c0 = f.xt[1] * f.xp[2] - f.xt[2] * f.xp[1];
  const double c1 = f.xt[2] * f.xp[0] - f.xt[0] * f.xp[2];
  const double c2 = f.xt[0] * f.xp[1] - f.xt[1] * f.xp[0];
  const double W = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  f.n[0] = c0 / W;
  f.n[1] = c1 / W;
  f.n[2] = c2 / W;
  f.E = f.xt[0] * f.xt[0] + f.xt[1] * f.xt[1] + f.xt[2] * f.xt[2];
  f.F = f.xt[0] * f.xp[0] + f.xt[1] * f.xp[1] + f.xt[2] * f.xp[2];
  f.G = f.xp[0] * f.xp[0] + f.xp[1] * f.xp[1] + f.xp[2] * f.xp[2];
  f.det = f.E * f.G - f.F * f.F;
  const double L = xtt[0] * f.n[0] + xtt[1] * f.n[1] + xtt[2] * f.n[2];
  const double M = xtp[0] * f.n[0] + xtp[1] * f.n[1] + xtp[2] * f.n[2];
  const double N = xpp[0] * f.n[0] + xpp[1] * f.n[1] + xpp[2] * f.n[2];
  f.H = -(f.E * N - 2.0 * f.F * M + f.G * L) / (2.0 * f.det);
  return f;
}

// surface gradient of a scalar from its theta / phi derivatives
__device__ __forceinline__ void surf_grad(const Frame& f, double dt_, double dp, double* g) {
  const double a = (f.G * dt_ - f.F * dp) / f.det;
  const double b = (f.E * dp - f.F * dt_) / f.det;
#pragma unroll
  for (int c = 0; c < 3; ++c) g[c] = a * f.xt[c] + b * f.xp[c];
}

// fields [6][ns]: E_n, phi_theta, phi_phi, Gamma, Gamma_theta, Gamma_phi -> out [3][ns]
__global__ void k_traction(const double* __restrict__ xup, int64_t ns, const double* __restrict__ fl,
                           int64_t fstride, PhysDev P, double* __restrict__ out, int64_t ostride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  const Frame f = frame_at(xup, ns, i);
  const double En = fl[i], pt = fl[fstride + i], pp = fl[2 * fstride + i];
  const double Gm = fl[3 * fstride + i], Gt = fl[4 * fstride + i], Gp = fl[5 * fstride + i];
  double gphi[3], gG[3];
  surf_grad(f, pt, pp, gphi);
  surf_grad(f, Gt, Gp, gG);
  const double Ei[3] = {P.eu0 + P.eq * (P.g[0] * f.x[0] + P.g[1] * f.x[1] + P.g[2] * f.x[2]),
                        P.eu1 + P.eq * (P.g[1] * f.x[0] + P.g[3] * f.x[1] + P.g[4] * f.x[2]),
                        P.eu2 + P.eq * (P.g[2] * f.x[0] + P.g[4] * f.x[1] + P.g[5] * f.x[2])};
  const double Ein = Ei[0] * f.n[0] + Ei[1] * f.n[1] + Ei[2] * f.n[2];
  double Et[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) Et[c] = Ei[c] - Ein * f.n[c] - gphi[c];
  const double Et2 = Et[0] * Et[0] + Et[1] * Et[1] + Et[2] * Et[2];
  const double fn = 0.5 * ((1.0 - P.Q / (P.R * P.R)) * En * En - (1.0 - P.Q) * Et2);
  const double ft = (1.0 - P.Q / P.R) * En;
  // tension and its derivative in Gamma: the normalised Langmuir law (Eq. langmuir) or the linear law of
  // Section 1, gamma = 1 + beta_t (1 - Gamma)
  const bool lin = P.eos == SHBIM_EOS_LINEAR;
  const double gam = lin ? 1.0 + P.beta * (1.0 - Gm) : (1.0 + P.beta * log(1.0 - P.x_s * Gm)) / P.lnorm;
  const double dgam = lin ? -P.beta : (-P.beta * P.x_s / (1.0 - P.x_s * Gm)) / P.lnorm;
  const double inv_ca = 1.0 / P.Ca_E;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double fI = 2.0 * gam * f.H * f.n[c] - dgam * gG[c];
    const double fE = fn * f.n[c] + ft * Et[c];
    out[c * ostride + i] = fI * inv_ca - fE;
  }
}

// uf [3 comps][2 kinds: theta, phi][ustride], Gamma value -> -Gamma div_S u
__global__ void k_surf_rate(const double* __restrict__ xup, int64_t ns, const double* __restrict__ uf,
                            int64_t ustride, const double* __restrict__ Gm, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  const Frame f = frame_at(xup, ns, i);
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double ut = uf[(2 * k) * ustride + i], up = uf[(2 * k + 1) * ustride + i];
    a += ut * f.xt[k];
    b += ut * f.xp[k];
    c += up * f.xt[k];
    d += up * f.xp[k];
  }
  const double div = (f.G * a - f.F * (b + c) + f.E * d) / f.det;
  out[i] = -Gm[i] * div;
}

// fd [5][fstride]: f_theta, f_theta_theta, f_theta_phi, f_phi_phi, f_phi -> Delta_S f.
// g^{ab} Gamma^c_ab f_c is formed through X = g^{ab} x_ab: g^{ab} Gamma^c_ab = g^{cd} x_d . X.
__global__ void k_laplace_beltrami(const double* __restrict__ xup, int64_t ns, const double* __restrict__ fd,
                                   int64_t fstride, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  double xt[3], xp[3], xtt[3], xtp[3], xpp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* b = xup + (int64_t)c * kNumTab * ns;
    xt[c] = b[ns + i];
    xtt[c] = b[3 * ns + i];
    xtp[c] = b[4 * ns + i];
    xpp[c] = b[5 * ns + i];
    xp[c] = b[6 * ns + i];
  }
  const double E = xt[0] * xt[0] + xt[1] * xt[1] + xt[2] * xt[2];
  const double F = xt[0] * xp[0] + xt[1] * xp[1] + xt[2] * xp[2];
  const double G = xp[0] * xp[0] + xp[1] * xp[1] + xp[2] * xp[2];
  const double det = E * G - F * F;
  const double gtt = G / det, gtp = -F / det, gpp = E / det;
  double X[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) X[c] = gtt * xtt[c] + 2.0 * gtp * xtp[c] + gpp * xpp[c];
  const double a = xt[0] * X[0] + xt[1] * X[1] + xt[2] * X[2];
  const double b = xp[0] * X[0] + xp[1] * X[1] + xp[2] * X[2];
  const double ct = gtt * a + gtp * b, cp = gtp * a + gpp * b;
  const double ft = fd[i], ftt = fd[fstride + i], ftp = fd[2 * fstride + i], fpp = fd[3 * fstride + i],
               fp = fd[4 * fstride + i];
  out[i] = gtt * ftt + 2.0 * gtp * ftp + gpp * fpp - ct * ft - cp * fp;
}

__global__ void k_lincomb(double* __restrict__ y, const double* __restrict__ a, double alpha,
                          const double* __restrict__ b, double beta, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = alpha * a[e] + beta * b[e];
}

// max over nodes of the Euclidean norm of ncomp fields [ncomp][stride] -> atomic max (bits)
__global__ void k_maxnorm(const double* __restrict__ v, int64_t n, int ncomp, int64_t stride,
                          unsigned long long* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n) {
    for (int c = 0; c < ncomp; ++c) s += v[c * stride + i] * v[c * stride + i];
    s = sqrt(s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0 && s > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

int ensure_buf(shbim_ctx* ctx, double** p, size_t* cap, size_t need) {
  if (need <= *cap) return SHBIM_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need * sizeof(double)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc physics workspace");
  *cap = need;
  return SHBIM_OK;
}

int solve(shbim_ctx* ctx, int sys, const double* rhs, const double* x0, double* x, double inner_tol, int* iters,
          cudaStream_t s) {
  if (ctx->opts.precision == SHBIM_PREC_FP32_COMP) {
    int inner = 0, outer = 0;
    int rc = shbim_gmres_solve_refined(ctx, sys, rhs, x0, x, inner_tol, 20, &inner, &outer, nullptr, s);
    if (iters) *iters = inner;
    return rc;
  }
  return shbim_gmres_solve(ctx, sys, rhs, x0, x, iters, nullptr, s);
}

}  // namespace

// Workspace of the rates (W.buf): coefficient vectors, then grid fields on the degree 2p+1 grids.
struct RatesWork {
  double *rhs_e, *En, *q, *phi, *tco, *rhs_s, *fl, *tv, *uf, *gv;
};

int rates_work(shbim_ctx* ctx, RatesWork* w) {
  const int64_t n = ctx->ncoef, NS = ctx->nsource;
  auto& W = ctx->phys;
  const size_t need = (size_t)(4 * n + 6 * n) + (size_t)(6 + 3 + 6 + 1) * NS;
  if (int rc = ensure_buf(ctx, &W.buf, &W.cap, need)) return rc;
  w->rhs_e = W.buf;
  w->En = w->rhs_e + n;
  w->q = w->En + n;
  w->phi = w->q + n;
  w->tco = w->phi + n;        // 3n
  w->rhs_s = w->tco + 3 * n;  // 3n
  w->fl = w->rhs_s + 3 * n;   // 6 NS: E_n, phi_theta, phi_phi, Gamma, Gamma_theta, Gamma_phi
  w->tv = w->fl + 6 * NS;     // 3 NS
  w->uf = w->tv + 3 * NS;     // 6 NS
  w->gv = w->uf + 6 * NS;     // NS
  return SHBIM_OK;
}

// Right-hand side of the Stokes system for a given E_n (steps ii-v of Section 1): the charge potential
// phi_q = S_L[(1 - 1/R) E_n], E_t = -grad_S(phi_inf + phi_q), the electric and interfacial tractions on
// every drop's degree 2p+1 grid (products de-aliased by projection to degree p) and
// rhs = -sum_j S_j[f/Ca_E - f^E]. Leaves Gamma and its derivatives on the grids in the workspace.
int stokes_rhs(shbim_ctx* ctx, const shbim_phys& ph, const double* gamma, const double* En, double* rhs_s,
               cudaStream_t s) {
  const int64_t n = ctx->ncoef, NS = ctx->nsource;
  RatesWork w;
  int rc;
  if ((rc = rates_work(ctx, &w))) return rc;
  const double R = ph.R;
  // (ii) phi_q = S_L[(1 - 1/R) E_n]
  k_lincomb<<<nb(n), 256, 0, s>>>(w.q, En, 1.0 - 1.0 / R, En, 0.0, n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  // one-shot applications (not iterated by GMRES): in mixed precision their arithmetic is the
  // context's one-shot precision (FP64-class by default: the single layer of the capillary traction
  // nearly cancels over a drop -- a sphere under uniform tension does not move -- so an FP32 sum's
  // ~1e-7 relative error of S[f/Ca_E] is a much larger relative error of the velocity); otherwise
  // the context's precision
  const int saved_prec = ctx->opts.precision;
  const int oneshot = saved_prec == SHBIM_PREC_FP32_COMP ? ctx->oneshot_prec : saved_prec;
  ctx->opts.precision = oneshot;
  rc = shbim_eval_electric(ctx, SHBIM_LAPLACE_SL, w.q, w.phi, SHBIM_OUT_COEF, s);
  ctx->opts.precision = saved_prec;
  if (rc) return rc;
  // (iii)-(v) traction on every drop's upsampled grid, projected to degree p
  PhysDev P{ph.R, ph.Q, ph.Ca_E, ph.beta, ph.x_s, ph.E_u[0], ph.E_u[1], ph.E_u[2], ph.E_q,
            1.0 + ph.beta * std::log(1.0 - ph.x_s)};
  std::memcpy(P.g, ctx->field_g, sizeof(P.g));
  P.eos = ctx->eos;
  // fields on every drop's upsampled grid, one launch per degree
  for (const DegreeGroup& G : ctx->groups) {
    const GridTables& g = G.tab->up;
    const DropList L = G.sources();
    const int nc = ncoef(G.tab->p);
    if ((rc = sht_synth(ctx, g, G.n, En, nc, 1 << 0, w.fl, 0, NS, nullptr, nullptr, s, 1, &L)) ||
        (rc = sht_synth(ctx, g, G.n, w.phi, nc, (1 << 1) | (1 << 6), w.fl + NS, 0, NS, nullptr, nullptr, s, 1, &L)) ||
        (rc = sht_synth(ctx, g, G.n, gamma, nc, (1 << 0) | (1 << 1) | (1 << 6), w.fl + 3 * NS, 0, NS, nullptr, nullptr,
                        s, 1, &L)))
      return rc;
  }
  for (auto& d : ctx->drops) {
    const int64_t o = d.src_off;
    k_traction<<<nb(d.ns), 256, 0, s>>>(ctx->xup + 3 * kNumTab * o, d.ns, w.fl + o, NS, P, w.tv + o, NS);
    SHBIM_CHECK_LAUNCH(ctx, "k_traction");
  }
  for (const DegreeGroup& G : ctx->groups) {
    const DropList L = G.sources();
    if ((rc = sht_analysis(ctx, G.tab->up, 3 * G.n, w.tv, NS, true, w.tco, ncoef(G.tab->p), s, 3, &L))) return rc;
  }
  // (vi) right-hand side of (lam_i+1) u - sum (lam_j-1) D_j[u] = -sum_j S_j[f/Ca_E - f^E]
  ctx->opts.precision = oneshot;
  rc = shbim_eval_stokes(ctx, w.tco, nullptr, rhs_s, SHBIM_OUT_COEF, s);
  ctx->opts.precision = saved_prec;
  if (rc) return rc;
  k_lincomb<<<nb(3 * n), 256, 0, s>>>(rhs_s, rhs_s, -1.0, rhs_s, 0.0, 3 * n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  return SHBIM_OK;
}

// u_guess (may be null): initial guess of the Stokes solve (the other stage's velocity in a time step)
int rates(shbim_ctx* ctx, const shbim_phys& ph, const double* gamma, double* u, double* gE, int* it_e,
          int* it_s, cudaStream_t s, const double* u_guess = nullptr) {
  const int64_t n = ctx->ncoef, NS = ctx->nsource;
  auto& W = ctx->phys;
  RatesWork w;
  int rc;
  if ((rc = rates_work(ctx, &w))) return rc;
  const double R = ph.R;
  if (R != ctx->opts.R) ctx->geom_version++;
  ctx->opts.R = R;
  // (i) E_n
  if ((rc = shbim_electric_rhs(ctx, ph.E_u, ph.E_q, w.rhs_e, s))) return rc;
  // learned initial guesses of both solves (the network only proposes; GMRES solves to its tolerance)
  const double* En0 = nullptr;
  const double* u_net = nullptr;
  if (ctx->warm_net && ctx->xcoef_cur) {
    const int64_t nf = shbim_warm_start_feature_count(ctx);
    if ((size_t)nf > W.feat_cap) {
      cudaFree(W.feat);
      W.feat = nullptr;
      W.feat_cap = 0;
      if (cudaMalloc(&W.feat, nf * sizeof(float)) != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "warm-start features");
      W.feat_cap = nf;
    }
    if ((rc = ensure_buf(ctx, &W.guess, &W.guess_cap, 4 * (size_t)n))) return rc;
    if ((rc = shbim_warm_start_features(ctx, ctx->xcoef_cur, gamma, &ph, W.feat, s)) ||
        (rc = shbim_learned_guess(ctx, ctx->warm_net, W.feat, w.rhs_e, W.guess, W.guess + n, s)))
      return rc;
    En0 = W.guess;
    u_net = W.guess + n;
  }
  if ((rc = solve(ctx, SHBIM_SYS_ELECTRIC, w.rhs_e, En0, w.En, ph.inner_tol, it_e, s))) return rc;
  // (ii)-(vi) the Stokes right-hand side, then the Stokes solve
  if ((rc = stokes_rhs(ctx, ph, gamma, w.En, w.rhs_s, s))) return rc;
  if ((rc = solve(ctx, SHBIM_SYS_STOKES, w.rhs_s, u_guess ? u_guess : u_net, u, ph.inner_tol, it_s, s))) return rc;
  // surfactant rate -Gamma div_S u, projected to degree p
  for (const DegreeGroup& G : ctx->groups) {
    const DropList L = G.sources();
    if ((rc = sht_synth(ctx, G.tab->up, 3 * G.n, u, ncoef(G.tab->p), (1 << 1) | (1 << 6), w.uf, 2 * NS, NS, nullptr,
                        nullptr, s, 3, &L)))
      return rc;
  }
  for (auto& d : ctx->drops) {
    const int64_t o = d.src_off;
    k_surf_rate<<<nb(d.ns), 256, 0, s>>>(ctx->xup + 3 * kNumTab * o, d.ns, w.uf + o, NS, w.fl + 3 * NS + o, w.gv + o);
    SHBIM_CHECK_LAUNCH(ctx, "k_surf_rate");
  }
  for (const DegreeGroup& G : ctx->groups) {
    const DropList L = G.sources();
    if ((rc = sht_analysis(ctx, G.tab->up, G.n, w.gv, 0, true, gE, ncoef(G.tab->p), s, 1, &L))) return rc;
  }
  return SHBIM_OK;
}

int laplace_beltrami(shbim_ctx* ctx, const double* coef, double* out, cudaStream_t s) {
  const int64_t NS = ctx->nsource;
  auto& W = ctx->phys;
  if (W.lb_cap < (size_t)6 * NS) {
    // only at the first use for a layout: captured operator graphs hold this workspace
    int rc = ensure_buf(ctx, &W.lb, &W.lb_cap, (size_t)6 * NS);
    if (rc) return rc;
    ctx->geom_version++;
  }
  double* fd = W.lb;
  double* lv = fd + 5 * NS;
  const int kinds = (1 << 1) | (1 << 3) | (1 << 4) | (1 << 5) | (1 << 6);
  int rc;
  for (auto& d : ctx->drops) {
    const GridTables& g = d.tab->up;
    const int64_t o = d.src_off;
    if ((rc = sht_synth(ctx, g, 1, coef + d.coef_off, d.nc, kinds, fd + o, 0, NS, nullptr, nullptr, s))) return rc;
    k_laplace_beltrami<<<nb(d.ns), 256, 0, s>>>(ctx->xup + 3 * kNumTab * o, d.ns, fd + o, NS, lv + o);
    SHBIM_CHECK_LAUNCH(ctx, "k_laplace_beltrami");
    if ((rc = sht_analysis(ctx, g, 1, lv + o, NS, true, out + d.coef_off, d.nc, s))) return rc;
  }
  return SHBIM_OK;
}

int rebuild_geometry(shbim_ctx* ctx, const double* xcoef, cudaStream_t s);

int grid_maxnorm(shbim_ctx* ctx, const double* coef, int ncomp, double* out_host, cudaStream_t s) {
  auto& W = ctx->phys;
  int rc;
  const size_t need = (size_t)3 * ctx->ntarget + 1;
  if ((rc = ensure_buf(ctx, &W.grid, &W.grid_cap, need))) return rc;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(W.grid + 3 * ctx->ntarget);
  SHBIM_CUDA(ctx, cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
  for (auto& d : ctx->drops) {
    const int64_t cstride = (int64_t)ncomp == 3 ? 3 * d.coef_off : d.coef_off;
    if ((rc = sht_synth(ctx, d.tab->base, ncomp, coef + cstride, d.nc, 1, W.grid, d.nt, 0, nullptr, nullptr, s)))
      return rc;
    k_maxnorm<<<nb(d.nt), 256, 0, s>>>(W.grid, d.nt, ncomp, d.nt, mx);
    SHBIM_CHECK_LAUNCH(ctx, "k_maxnorm");
  }
  unsigned long long h = 0;
  SHBIM_CUDA(ctx, cudaMemcpyAsync(&h, mx, sizeof(h), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  double v;
  std::memcpy(&v, &h, sizeof(v));
  *out_host = v;
  return SHBIM_OK;
}

}  // namespace shbim

using namespace shbim;

extern "C" {

int shbim_rates(shbim_ctx* ctx, const shbim_phys* ph, const double* gamma_dev, double* u_dev, double* gE_dev,
                int* iters_host, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!ph || !gamma_dev || !u_dev || !gE_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  if (!(ph->R > 0.0) || !(ph->Ca_E > 0.0) || ph->beta < 0.0 || !(ph->x_s >= 0.0 && ph->x_s < 1.0) ||
      !(ph->inner_tol > 0.0 && ph->inner_tol < 1.0) || !(ph->Pe >= 0.0))
    return fail(ctx, SHBIM_ERR_ARG, "bad physical parameters");
  int ie = 0, is = 0;
  int rc = rates(ctx, *ph, gamma_dev, u_dev, gE_dev, &ie, &is, (cudaStream_t)stream);
  if (iters_host) {
    iters_host[0] = ie;
    iters_host[1] = is;
  }
  return rc;
}

int shbim_step(shbim_ctx* ctx, const shbim_phys* ph, const double* x_dev, const double* gamma_dev, double dt,
               double* x_out_dev, double* gamma_out_dev, double* err_host, int* iters_host, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!ph || !x_dev || !gamma_dev || !x_out_dev || !gamma_out_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, SHBIM_ERR_ARG, "dt must be positive");
  if (!(ph->Pe >= 0.0)) return fail(ctx, SHBIM_ERR_ARG, "Pe must be >= 0 (0 or infinity: no diffusion)");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = ctx->ncoef;
  auto& W = ctx->phys;
  int rc;
  const bool diffuse = ph->Pe > 0.0 && std::isfinite(ph->Pe);
  if ((rc = ensure_buf(ctx, &W.state, &W.state_cap, (size_t)13 * n))) return rc;
  double* u0 = W.state;
  double* g0 = u0 + 3 * n;
  double* u1 = g0 + n;
  double* g1 = u1 + 3 * n;
  double* xh = g1 + n;  // 3n
  // the half-step surfactant shares the last n entries with nothing else
  double* gh = W.state + 11 * n;
  int its[4] = {0, 0, 0, 0};
  if ((rc = rebuild_geometry(ctx, x_dev, s))) return rc;
  if ((rc = rates(ctx, *ph, gamma_dev, u0, g0, &its[0], &its[1], s))) return rc;
  k_lincomb<<<nb(3 * n), 256, 0, s>>>(xh, x_dev, 1.0, u0, 0.5 * dt, 3 * n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  k_lincomb<<<nb(n), 256, 0, s>>>(gh, gamma_dev, 1.0, g0, 0.5 * dt, n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  if ((rc = rebuild_geometry(ctx, xh, s))) return rc;
  if (diffuse) {
    // implicit half step of the diffusion on the half-step surface (FP64 in every mode)
    if ((rc = shbim_set_diffusion(ctx, 0.5 * dt / ph->Pe))) return rc;
    if ((rc = shbim_gmres_solve(ctx, SHBIM_SYS_DIFFUSION, gh, nullptr, gh, nullptr, nullptr, s))) return rc;
  }
  // the second stage's Stokes solve starts from the first stage's velocity
  if ((rc = rates(ctx, *ph, gh, u1, g1, &its[2], &its[3], s, u0))) return rc;
  if (diffuse) {
    double* lg = W.state + 12 * n;
    if ((rc = laplace_beltrami(ctx, gh, lg, s))) return rc;
    k_lincomb<<<nb(n), 256, 0, s>>>(g1, g1, 1.0, lg, 1.0 / ph->Pe, n);
    SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  }
  k_lincomb<<<nb(3 * n), 256, 0, s>>>(x_out_dev, x_dev, 1.0, u1, dt, 3 * n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  k_lincomb<<<nb(n), 256, 0, s>>>(gamma_out_dev, gamma_dev, 1.0, g1, dt, n);
  SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
  if (err_host) {
    // err = dt * max(max |u1 - u0|, max |g1 - g0|) on the degree-p grids
    k_lincomb<<<nb(3 * n), 256, 0, s>>>(u0, u1, 1.0, u0, -1.0, 3 * n);
    SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
    k_lincomb<<<nb(n), 256, 0, s>>>(g0, g1, 1.0, g0, -1.0, n);
    SHBIM_CHECK_LAUNCH(ctx, "k_lincomb");
    double eu = 0.0, eg = 0.0;
    if ((rc = grid_maxnorm(ctx, u0, 3, &eu, s)) || (rc = grid_maxnorm(ctx, g0, 1, &eg, s))) return rc;
    *err_host = dt * std::max(eu, eg);
  }
  if (iters_host)
    for (int k = 0; k < 4; ++k) iters_host[k] = its[k];
  return SHBIM_OK;
}

int shbim_stokes_rhs(shbim_ctx* ctx, const shbim_phys* ph, const double* gamma_dev, const double* En_dev,
                     double* rhs_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!ph || !gamma_dev || !En_dev || !rhs_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  if (!(ph->R > 0.0) || !(ph->Ca_E > 0.0) || ph->beta < 0.0 || !(ph->x_s >= 0.0 && ph->x_s < 1.0))
    return fail(ctx, SHBIM_ERR_ARG, "bad physical parameters");
  if (ph->R != ctx->opts.R) ctx->geom_version++;
  ctx->opts.R = ph->R;
  return stokes_rhs(ctx, *ph, gamma_dev, En_dev, rhs_dev, (cudaStream_t)stream);
}

int shbim_laplace_beltrami(shbim_ctx* ctx, const double* coef_dev, double* out_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!coef_dev || !out_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  return laplace_beltrami(ctx, coef_dev, out_dev, (cudaStream_t)stream);
}

}  // extern "C"
