// Reparametrisation of the drop surfaces (Section 2.2; applied after every accepted step of
// Algorithm 1).
//
// The nodes of each drop move along its surface so as to lower the spectral energy of the
// parametrisation, E = sum over components, degrees n >= 1 and orders m of n^a |x_nm|^2. One step
// is an explicit step of the tangential gradient flow, on each drop's degree 2p+1 grid:
//   h = sum n^a x_nm S_nm (half the energy gradient as a field),  t = h - (h . n) n,
//   x <- x - tau t,  tau = c / p^a,
// and the moved grid positions are projected back to degree p by the regular rule. The surfactant
// concentration lives on the same nodes and is carried with them: the node now sits where the
// surface point x - tau t was, so
//   Gamma <- Gamma - tau grad_S Gamma . t,  grad_S Gamma . t = [G_a G_b] M^-1 [a . t, b . t]^T,
// with the tangents a = x_theta, b = x_phi / sin(theta), their Gram matrix M and G_a, G_b the
// matching derivatives of Gamma. Everything runs in FP64: the work per step is a few transforms.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace shbim {

namespace {

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// wx = w3 * x elementwise (w3: n^a of each coefficient in the position layout)
__global__ void k_rep_weight(const double* __restrict__ x, const double* __restrict__ w3, double* __restrict__ wx,
                             int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wx[i] = w3[i] * x[i];
}

// e[0] = sum w3 x^2, one block (fixed summation order)
__global__ void k_rep_energy(const double* __restrict__ x, const double* __restrict__ w3, int64_t n,
                             double* __restrict__ e) {
  __shared__ double part[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += w3[i] * x[i] * x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) e[0] = s;
  }
}

// The moved node values of one degree group: blockIdx.y = drop of the group, nodes of its
// degree 2p+1 grid. Layouts (NS = all drops' grid nodes, off = the drop's first node):
//   xs[(kind * 3 + c) NS + off + i]  x, x_theta, x_phi/sin (kind 0, 1, 2) of component c
//   h[c NS + off + i];  gs[kind NS + off + i] Gamma and its two derivatives (may be null)
//   vals[c NS + off + i] moved positions, vals[3 NS + off + i] carried Gamma
__global__ void k_rep_move(const int64_t* __restrict__ src_off, int ns, int64_t NS, const double* __restrict__ xs,
                           const double* __restrict__ h, const double* __restrict__ gs, double tau,
                           double* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ns) return;
  const int64_t o = src_off[blockIdx.y] + i;
  double X[3], A[3], B[3], H[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X[c] = xs[(0 * 3 + c) * NS + o];
    A[c] = xs[(1 * 3 + c) * NS + o];
    B[c] = xs[(2 * 3 + c) * NS + o];
    H[c] = h[c * NS + o];
  }
  double nv[3] = {A[1] * B[2] - A[2] * B[1], A[2] * B[0] - A[0] * B[2], A[0] * B[1] - A[1] * B[0]};
  const double inv = 1.0 / sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
#pragma unroll
  for (int c = 0; c < 3; ++c) nv[c] *= inv;
  const double hn = H[0] * nv[0] + H[1] * nv[1] + H[2] * nv[2];
  double T[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T[c] = H[c] - hn * nv[c];
    vals[c * NS + o] = X[c] - tau * T[c];
  }
  if (gs) {
    const double maa = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
    const double mab = A[0] * B[0] + A[1] * B[1] + A[2] * B[2];
    const double mbb = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const double at = A[0] * T[0] + A[1] * T[1] + A[2] * T[2];
    const double bt = B[0] * T[0] + B[1] * T[1] + B[2] * T[2];
    const double ga = gs[NS + o], gb = gs[2 * NS + o];
    const double dg = (ga * (mbb * at - mab * bt) + gb * (maa * bt - mab * at)) / (maa * mbb - mab * mab);
    vals[3 * NS + o] = gs[o] - tau * dg;
  }
}

int ensure_rep(shbim_ctx* ctx, size_t need, cudaStream_t s) {
  auto& W = ctx->phys;
  if (need <= W.rep_cap) return SHBIM_OK;
  if (W.rep) {
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    cudaFree(W.rep);
    W.rep = nullptr;
    W.rep_cap = 0;
  }
  if (cudaMalloc(&W.rep, need * sizeof(double)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc reparametrisation workspace");
  W.rep_cap = need;
  return SHBIM_OK;
}

}  // namespace

int reparametrize(shbim_ctx* ctx, int steps, double a, double c, double* x, double* gamma, double* energy_host,
                  cudaStream_t s) {
  const int64_t NS = ctx->nsource, n3 = 3 * ctx->ncoef;
  // workspace: xs 9 NS | h 3 NS | gs 3 NS | vals 4 NS | w3 n3 | wx n3 | energies steps+1
  const size_t need = (size_t)19 * NS + 2 * (size_t)n3 + (size_t)steps + 1;
  int rc;
  if ((rc = ensure_rep(ctx, need, s))) return rc;
  double* xs = ctx->phys.rep;
  double* h = xs + 9 * NS;
  double* gs = h + 3 * NS;
  double* vals = gs + 3 * NS;
  double* w3 = vals + 4 * NS;
  double* wx = w3 + n3;
  double* en = wx + n3;
  std::vector<double> w3h((size_t)n3);
  for (const Drop& d : ctx->drops)
    for (int cc = 0; cc < 3; ++cc)
      for (int n = 0; n <= d.p; ++n)
        for (int o = n * n; o < (n + 1) * (n + 1); ++o) w3h[3 * d.coef_off + (int64_t)cc * d.nc + o] = std::pow((double)n, a) * (n > 0);
  SHBIM_CUDA(ctx, cudaMemcpyAsync(w3, w3h.data(), n3 * sizeof(double), cudaMemcpyHostToDevice, s));
  k_rep_energy<<<1, 1024, 0, s>>>(x, w3, n3, en);
  SHBIM_CHECK_LAUNCH(ctx, "k_rep_energy");
  for (int it = 0; it < steps; ++it) {
    k_rep_weight<<<blocks(n3, 256), 256, 0, s>>>(x, w3, wx, n3);
    SHBIM_CHECK_LAUNCH(ctx, "k_rep_weight");
    for (const DegreeGroup& G : ctx->groups) {
      const GridTables& g = G.tab->up;
      const DropList L = G.sources();
      const int p = G.tab->p, nc = ncoef(p), ns = npts(g.q);
      const double tau = c / std::pow((double)p, a);
      if ((rc = sht_synth(ctx, g, 3 * G.n, x, nc, 7, xs, NS, 3 * NS, nullptr, nullptr, s, 3, &L)) ||
          (rc = sht_synth(ctx, g, 3 * G.n, wx, nc, 1, h, NS, 0, nullptr, nullptr, s, 3, &L)))
        return rc;
      if (gamma && (rc = sht_synth(ctx, g, G.n, gamma, nc, 7, gs, 0, NS, nullptr, nullptr, s, 1, &L))) return rc;
      k_rep_move<<<dim3(blocks(ns, 128), G.n), 128, 0, s>>>(G.src, ns, NS, xs, h, gamma ? gs : nullptr, tau, vals);
      SHBIM_CHECK_LAUNCH(ctx, "k_rep_move");
      if ((rc = sht_analysis(ctx, g, 3 * G.n, vals, NS, true, x, nc, s, 3, &L))) return rc;
      if (gamma && (rc = sht_analysis(ctx, g, G.n, vals + 3 * NS, 0, true, gamma, nc, s, 1, &L))) return rc;
    }
    k_rep_energy<<<1, 1024, 0, s>>>(x, w3, n3, en + it + 1);
    SHBIM_CHECK_LAUNCH(ctx, "k_rep_energy");
  }
  if (energy_host)
    SHBIM_CUDA(ctx, cudaMemcpyAsync(energy_host, en, (size_t)(steps + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  return SHBIM_OK;
}

}  // namespace shbim

using namespace shbim;

extern "C" {

int shbim_reparametrize(shbim_ctx* ctx, int steps, double a, double c, double* x_dev, double* gamma_dev,
                        double* energy_host, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (!x_dev) return fail(ctx, SHBIM_ERR_ARG, "null position coefficients");
  if (steps < 0 || steps > 100000) return fail(ctx, SHBIM_ERR_ARG, "steps outside 0..100000");
  if (!(a >= 0.0 && a <= 8.0)) return fail(ctx, SHBIM_ERR_ARG, "energy exponent a outside [0, 8]");
  if (!(c > 0.0 && c <= 1.0)) return fail(ctx, SHBIM_ERR_ARG, "step factor c outside (0, 1]");
  if (gamma_dev) {
    const char* x0 = reinterpret_cast<const char*>(x_dev);
    const char* g0 = reinterpret_cast<const char*>(gamma_dev);
    const size_t xb = 3 * (size_t)ctx->ncoef * sizeof(double), gb = (size_t)ctx->ncoef * sizeof(double);
    if (g0 < x0 + xb && x0 < g0 + gb) return fail(ctx, SHBIM_ERR_ARG, "gamma and positions overlap");
  }
  return reparametrize(ctx, steps, a, c, x_dev, gamma_dev, energy_host, (cudaStream_t)stream);
}

}  // extern "C"
