// Transform and quadrature tables, computed on the host in FP64 once per degree.
//
// * Gauss-Legendre nodes and weights (Newton on P_N) for the latitudes of the Gaussian grid
//   (Section 2, Eq. spharm_ex).
// * Normalised associated Legendre functions with the Condon-Shortley phase
//   (Eqs. normalized_spharm, pneg) and the derivative tables the transforms need,
//   d/dtheta Pbar_n^m = (n t Pbar_n^m - sqrt((2n+1)/(2n-1) (n^2-m^2)) Pbar_{n-1}^m) / sin,
//   the second derivative from the associated Legendre equation, and the m / m^2 factors of
//   the phi derivatives, tabulated at the grid latitudes (never at a pole).
// * Regular weights omega_j = (pi/(q+1)) w_j^G (Eq. reg_quadrature with the 2q+2 point
//   trapezoid spacing) and modified weights mu_j = omega_j 2 sin(theta_j/2) sum_{n<=q} P_n(t_j)
//   (Eq. mod_weights on the degree-q grid).
// * The real-basis rotation matrix of the fixed rotation Rx(pi/2), per degree n, obtained
//   exactly by quadrature of S_nm(Q y) S_nm'(y) on the degree-p grid. Composed with
//   z-rotations it rotates any target to the north pole (Section 2.1).
#include <cmath>
#include <cstring>
#include <mutex>
#include <omp.h>

#include "internal.h"

namespace shbim {

namespace {

void gauss_legendre(int N, std::vector<double>& t, std::vector<double>& w) {
  t.assign(N, 0.0);
  w.assign(N, 0.0);
  for (int i = 0; i < N; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (N + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= N; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = N * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // final derivative at the converged node
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= N; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = N * (z * p1 - p0) / (z * z - 1.0);
    t[i] = z;  // i = 0 is the node closest to +1: t decreasing, theta increasing
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

inline int tri_off(int p, int m) { return m * (p + 1) - m * (m - 1) / 2; }

// Pbar_n^m(t) for n <= nmax, m-major triangular layout of degree nmax.
void alf_values(int nmax, double t, double s, double* P) {
  // sectoral seeds
  double pmm = 1.0 / std::sqrt(4.0 * kPi);
  for (int m = 0; m <= nmax; ++m) {
    if (m > 0) pmm *= -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
    double* col = P + tri_off(nmax, m);
    col[0] = pmm;
    if (m + 1 <= nmax) col[1] = std::sqrt(2.0 * m + 3.0) * t * pmm;
    for (int n = m + 2; n <= nmax; ++n) {
      double a = std::sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
      double b = std::sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
      col[n - m] = a * (t * col[n - 1 - m] - b * col[n - 2 - m]);
    }
  }
}

int upload(shbim_ctx* ctx, double** dst, const std::vector<double>& src) {
  cudaError_t e = cudaMalloc(dst, src.size() * sizeof(double));
  if (e != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc for tables failed");
  e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy tables");
  return SHBIM_OK;
}

// (hi, lo) = (fl32(v), fl32(v - hi)): the double-float copy of an FP64 value
float2 split_df(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}

int upload_df(shbim_ctx* ctx, float2** dst, const std::vector<float2>& src) {
  cudaError_t e = cudaMalloc(dst, src.size() * sizeof(float2));
  if (e != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc for tables failed");
  e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy tables");
  return SHBIM_OK;
}

// alf_df / trig_df (optional): double-float copies of the kinds 0..2 and of the trig table
int upload_f(shbim_ctx* ctx, float** dst, const std::vector<float>& src) {
  cudaError_t e = cudaMalloc(dst, src.size() * sizeof(float));
  if (e != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc for tables failed");
  e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy tables");
  return SHBIM_OK;
}

// alf_df / trig_df (optional): double-float copies of the kinds 0..2 and of the trig table;
// f32: FP32 copies of kind 0 and of the trig table
int build_grid(shbim_ctx* ctx, int p, int q, GridTables& g, float2** alf_df = nullptr,
               float2** trig_df = nullptr, bool f32 = false, std::vector<double>* alf0_out = nullptr) {
  g.p = p;
  g.q = q;
  std::vector<double> t, wg;
  gauss_legendre(q + 1, t, wg);
  const int nt = ntri(p);
  std::vector<double> alf((size_t)(q + 1) * kNumTab * nt);
  std::vector<double> om(q + 1), mu(q + 1), th(q + 1);
  std::vector<double> P(nt);
  for (int j = 0; j <= q; ++j) {
    double tj = t[j];
    double sj = std::sqrt((1.0 - tj) * (1.0 + tj));
    th[j] = std::acos(tj);
    alf_values(p, tj, sj, P.data());
    double* A = &alf[(size_t)j * kNumTab * nt];
    for (int m = 0; m <= p; ++m) {
      for (int n = m; n <= p; ++n) {
        int o = tri_off(p, m) + (n - m);
        double v = P[o];
        double prev = (n - 1 >= m) ? P[o - 1] : 0.0;
        double c = std::sqrt((2.0 * n + 1.0) / (2.0 * n - 1.0) * ((double)n * n - (double)m * m));
        const double d1 = (n * tj * v - (n > 0 ? c * prev : 0.0)) / sj;
        A[o] = v;
        A[nt + o] = d1;
        A[2 * nt + o] = m * v / sj;
        // associated Legendre equation in theta: P'' = -cot P' - (n(n+1) - m^2/sin^2) P
        A[3 * nt + o] = -(tj / sj) * d1 - (n * (n + 1.0) - (double)m * m / (sj * sj)) * v;
        A[4 * nt + o] = m * d1;
        A[5 * nt + o] = -(double)m * m * v;
        A[6 * nt + o] = m * v;
      }
    }
    om[j] = kPi / (q + 1) * wg[j];
    // sum_{n=0}^{q} P_n(t) by the Bonnet recurrence
    double p0 = 1.0, p1 = tj, sum = 1.0 + (q >= 1 ? tj : 0.0);
    for (int n = 1; n < q; ++n) {
      double p2 = ((2.0 * n + 1.0) * tj * p1 - n * p0) / (n + 1.0);
      sum += p2;
      p0 = p1;
      p1 = p2;
    }
    mu[j] = om[j] * 2.0 * std::sqrt(0.5 * (1.0 - tj)) * sum;
  }
  const int N = 2 * q + 2;
  std::vector<double> trig(2 * N);
  for (int k = 0; k < N; ++k) {
    trig[k] = std::cos(2.0 * kPi * k / N);
    trig[N + k] = std::sin(2.0 * kPi * k / N);
  }
  int rc;
  if (alf0_out) {
    alf0_out->assign((size_t)(q + 1) * nt, 0.0);
    for (int j = 0; j <= q; ++j)
      for (int o = 0; o < nt; ++o) (*alf0_out)[(size_t)j * nt + o] = alf[(size_t)j * kNumTab * nt + o];
  }
  if (alf_df) {
    std::vector<float2> a((size_t)(q + 1) * 3 * nt);
    for (int j = 0; j <= q; ++j)
      for (int k = 0; k < 3; ++k)
        for (int o = 0; o < nt; ++o)
          a[((size_t)j * 3 + k) * nt + o] = split_df(alf[((size_t)j * kNumTab + k) * nt + o]);
    if ((rc = upload_df(ctx, alf_df, a))) return rc;
  }
  if (trig_df) {
    std::vector<float2> tr(2 * N);
    for (int k = 0; k < 2 * N; ++k) tr[k] = split_df(trig[k]);
    if ((rc = upload_df(ctx, trig_df, tr))) return rc;
  }
  if (f32) {
    std::vector<float> a((size_t)(q + 1) * nt), tr(2 * N);
    for (int j = 0; j <= q; ++j)
      for (int o = 0; o < nt; ++o) a[(size_t)j * nt + o] = (float)alf[(size_t)j * kNumTab * nt + o];
    for (int k = 0; k < 2 * N; ++k) tr[k] = (float)trig[k];
    if ((rc = upload_f(ctx, &g.alf32, a)) || (rc = upload_f(ctx, &g.trig32, tr))) return rc;
  }
  if ((rc = upload(ctx, &g.alf, alf))) return rc;
  if ((rc = upload(ctx, &g.omega, om))) return rc;
  if ((rc = upload(ctx, &g.mu, mu))) return rc;
  if ((rc = upload(ctx, &g.trig, trig))) return rc;
  if ((rc = upload(ctx, &g.theta, th))) return rc;
  return SHBIM_OK;
}

// Real basis value S_nm at a point (n fixed, all m), given the degree-n ALF column data.
// Fills S[m + n] for m = -n..n.
void real_basis_degree(int n, const double* Pn /* Pbar_n^m, m = 0..n */, double phi, double* S) {
  S[n] = Pn[0];
  for (int m = 1; m <= n; ++m) {
    S[n + m] = kSqrt2 * Pn[m] * std::cos(m * phi);
    S[n - m] = kSqrt2 * Pn[m] * std::sin(m * phi);
  }
}

// Pbar_n^m for a single degree n and all m (fresh recurrence per call).
void alf_degree(int n, double t, double s, double* out /* n+1 */) {
  double pmm = 1.0 / std::sqrt(4.0 * kPi);
  for (int m = 0; m <= n; ++m) {
    if (m > 0) pmm *= -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) * s;
    if (m == n) { out[m] = pmm; continue; }
    double a0 = pmm;
    double a1 = std::sqrt(2.0 * m + 3.0) * t * pmm;
    for (int k = m + 2; k <= n; ++k) {
      double a = std::sqrt((4.0 * k * k - 1.0) / ((double)k * k - (double)m * m));
      double b = std::sqrt(((k - 1.0) * (k - 1.0) - (double)m * m) / (4.0 * (k - 1.0) * (k - 1.0) - 1.0));
      double a2 = a * (t * a1 - b * a0);
      a0 = a1;
      a1 = a2;
    }
    out[m] = a1;
  }
}

int build_rotation(shbim_ctx* ctx, int p, DegreeTables& T) {
  // D[n][m][m'] = int S_nm(Q y) S_nm'(y) dOmega on the degree-p grid, Q = Rx(pi/2):
  // Q (x, y, z) = (x, -z, y). Exact because the integrand has degree 2n <= 2p.
  std::vector<double> t, wg;
  gauss_legendre(p + 1, t, wg);
  const int nphi = 2 * p + 2;
  T.dq_off.assign(p + 2, 0);
  for (int n = 0; n <= p; ++n) T.dq_off[n + 1] = T.dq_off[n] + (2 * n + 1) * (2 * n + 1);
  std::vector<double> D(T.dq_off[p + 1], 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int n = p; n >= 0; --n) {
    std::vector<double> Pa(n + 1), Pb(n + 1), Sa(2 * n + 1), Sb(2 * n + 1);
    double* Dn = &D[T.dq_off[n]];
    const int w = 2 * n + 1;
    for (int j = 0; j <= p; ++j) {
      double tj = t[j], sj = std::sqrt((1.0 - tj) * (1.0 + tj));
      double om = kPi / (p + 1) * wg[j];
      alf_degree(n, tj, sj, Pb.data());
      for (int k = 0; k < nphi; ++k) {
        double ph = kPi * k / (p + 1);
        double y0 = sj * std::cos(ph), y1 = sj * std::sin(ph), y2 = tj;
        double q0 = y0, q1 = -y2, q2 = y1;  // Q y
        double ct = q2, st = std::sqrt(q0 * q0 + q1 * q1);
        double qph = std::atan2(q1, q0);
        alf_degree(n, ct, st, Pa.data());
        real_basis_degree(n, Pa.data(), qph, Sa.data());
        real_basis_degree(n, Pb.data(), ph, Sb.data());
        for (int a = 0; a < w; ++a) {
          double f = om * Sa[a];
          for (int b = 0; b < w; ++b) Dn[a * w + b] += f * Sb[b];
        }
      }
    }
  }
  int rc = upload(ctx, &T.dq, D);
  if (rc) return rc;
  {
    std::vector<float2> Ddf(D.size());
    for (size_t i = 0; i < D.size(); ++i) Ddf[i] = split_df(D[i]);
    if ((rc = upload_df(ctx, &T.dq_df, Ddf))) return rc;
    // nonzero progressions of every row and column (zeros of the block are exact, the quadrature
    // leaves rounding noise far below the threshold); a row that is not a progression is dense
    std::vector<int4> rows((size_t)(p + 1) * (p + 1)), cols((size_t)(p + 1) * (p + 1));
    auto progression = [](const std::vector<int>& idx, int w) {
      if (idx.empty()) return make_int4(0, 0, 1, 0);
      const int step = idx.size() > 1 ? idx[1] - idx[0] : 1;
      for (size_t k = 1; k < idx.size(); ++k)
        if (idx[k] - idx[k - 1] != step) return make_int4(0, w, 1, 0);
      return make_int4(idx[0], (int)idx.size(), step, 0);
    };
    for (int n = 0; n <= p; ++n) {
      const int w = 2 * n + 1, o = T.dq_off[n];
      for (int a = 0; a < w; ++a) {
        std::vector<int> r, c;
        for (int b = 0; b < w; ++b) {
          if (std::fabs(D[o + a * w + b]) > 1e-12) r.push_back(b);
          if (std::fabs(D[o + b * w + a]) > 1e-12) c.push_back(b);
        }
        rows[(size_t)n * n + a] = progression(r, w);
        cols[(size_t)n * n + a] = progression(c, w);
      }
    }
    for (auto* pr : {&rows, &cols}) {
      int4** dst = pr == &rows ? &T.dq_rows : &T.dq_cols;
      if (cudaMalloc(dst, pr->size() * sizeof(int4)) != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc Dq pattern");
      if (cudaMemcpy(*dst, pr->data(), pr->size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(ctx, SHBIM_ERR_CUDA, "cudaMemcpy Dq pattern");
    }
    // cos / sin (m alpha) at the base-grid latitudes and longitudes (the targets' rotation angles)
    std::vector<double> tb, wb;
    gauss_legendre(p + 1, tb, wb);
    std::vector<float2> cth((size_t)(p + 1) * 2 * (p + 1)), cph((size_t)(2 * p + 2) * 2 * (p + 1));
    for (int j = 0; j <= p; ++j) {
      const double th = std::acos(tb[j]);
      for (int m = 0; m <= p; ++m) {
        cth[((size_t)j * 2) * (p + 1) + m] = split_df(std::cos(m * th));
        cth[((size_t)j * 2 + 1) * (p + 1) + m] = split_df(std::sin(m * th));
      }
    }
    for (int k = 0; k < 2 * p + 2; ++k) {
      const double ph = kPi * k / (p + 1);
      for (int m = 0; m <= p; ++m) {
        cph[((size_t)k * 2) * (p + 1) + m] = split_df(std::cos(m * ph));
        cph[((size_t)k * 2 + 1) * (p + 1) + m] = split_df(std::sin(m * ph));
      }
    }
    if ((rc = upload_df(ctx, &T.cs_theta_df, cth)) || (rc = upload_df(ctx, &T.cs_phi_df, cph))) return rc;
    std::vector<double> theta(p + 1);
    for (int j = 0; j <= p; ++j) theta[j] = std::acos(tb[j]);
    if ((rc = rot_tc_digits(ctx, p, D, theta, T))) return rc;
  }
  cudaError_t e = cudaMalloc(&T.dq_off_dev, T.dq_off.size() * sizeof(int));
  if (e != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc rotation offsets");
  e = cudaMemcpy(T.dq_off_dev, T.dq_off.data(), T.dq_off.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy rotation offsets");
  return SHBIM_OK;
}

}  // namespace

int build_degree_tables(shbim_ctx* ctx, int p, DegreeTables** out) {
  DegreeTables* T = new DegreeTables();
  T->p = p;
  int rc;
  std::vector<double> alf_up;
  if ((rc = build_grid(ctx, p, p, T->base)) ||
      (rc = build_grid(ctx, p, 2 * p + 1, T->up, &T->up_alf_df, &T->up_trig_df, true, &alf_up)) ||
      (rc = leg_tc_digits(ctx, p, alf_up, *T)) ||
      (rc = build_grid(ctx, p, 4 * (2 * p + 2) - 1, T->fine, nullptr, nullptr, true)) || (rc = build_rotation(ctx, p, *T)) ||
      (rc = dft_tc_digits(ctx, p, *T))) {
    free_degree_tables(T);
    return rc;
  }
  *out = T;
  return SHBIM_OK;
}

static void free_grid(GridTables& g) {
  cudaFree(g.alf32);
  cudaFree(g.trig32);
  cudaFree(g.alf);
  cudaFree(g.omega);
  cudaFree(g.mu);
  cudaFree(g.trig);
  cudaFree(g.theta);
}

void free_degree_tables(DegreeTables* t) {
  if (!t) return;
  free_grid(t->base);
  free_grid(t->up);
  free_grid(t->fine);
  cudaFree(t->dq);
  cudaFree(t->dq_off_dev);
  cudaFree(t->up_alf_df);
  cudaFree(t->up_trig_df);
  cudaFree(t->dq_df);
  cudaFree(t->dq_rows);
  cudaFree(t->dq_cols);
  cudaFree(t->dft_digits);
  cudaFree(t->rot_digits);
  cudaFree(t->rot_toff);
  cudaFree(t->rot_exp);
  cudaFree(t->leg_digits);
  cudaFree(t->leg_toff);
  cudaFree(t->leg_exp);
  cudaFree(t->cs_theta_df);
  cudaFree(t->cs_phi_df);
  delete t;
}

}  // namespace shbim
