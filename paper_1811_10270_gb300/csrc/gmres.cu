// Restarted GMRES on the Galerkin systems, FP64 on the device.
//
// The paper solves the Galerkin systems of Eqs. BIM_galerkin and galerkin_En without naming
// a solver; this is restarted GMRES(m) (Saad & Schultz) with classical Gram-Schmidt applied
// twice per Arnoldi step (every projection is one kernel, so a step costs a fixed number of
// launches), Givens rotations for the small least-squares problem on the host, and one
// device-to-host read of the new Hessenberg column per step.
//   electric: A s = 1/2 s - (R-1)/(R+1) L[s]           (Eq. galerkin_En)
//   Stokes:   A u = (lam_i + 1) u - sum_j (lam_j-1) D_j[u]   (Eq. main_eq, Galerkin form)
//   diffusion: (I - c Delta_S) G = b on every drop (implicit surfactant diffusion of Algorithm 1),
//             solved right-preconditioned, A y = M^{-1} y - c P[Delta_S M^{-1} y], G = M^{-1} y, with
//             M^{-1} = diag(1/(1 + c n(n+1)/a_i^2)), a_i^2 = area_i/(4 pi): the exact inverse on a
//             sphere of radius a_i, where Delta_S Y_nm = -n(n+1)/a^2 Y_nm.
#include <algorithm>
#include <cmath>

#include <vector>

#include "internal.h"

namespace shbim {

namespace {

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// h[i] = V_i . w for i < nvec (one block per vector, fixed summation order)
__global__ void k_dots(const double* __restrict__ V, int64_t n, const double* __restrict__ w,
                       double* __restrict__ h) {
  const double* v = V + (int64_t)blockIdx.x * n;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(v[e], w[e], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) h[blockIdx.x] = acc;
}

// w -= sum_i h[i] V_i ; hacc[i] += h[i]
__global__ void k_orth_update(double* __restrict__ w, const double* __restrict__ V, int64_t n, int nvec,
                              const double* __restrict__ h, double* __restrict__ hacc, int first) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    for (int i = 0; i < nvec; ++i) hacc[i] = first ? h[i] : hacc[i] + h[i];
  }
  if (e >= n) return;
  double acc = w[e];
  for (int i = 0; i < nvec; ++i) acc = fma(-h[i], V[(int64_t)i * n + e], acc);
  w[e] = acc;
}

__global__ void k_normalize(const double* __restrict__ w, const double* __restrict__ nrm2,
                            double* __restrict__ out, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
  out[e] = w[e] * s;
}

__global__ void k_system(const double* __restrict__ diag, double off, const double* __restrict__ x,
                         const double* __restrict__ Ax, double* __restrict__ y, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  y[e] = fma(diag[e], x[e], off * Ax[e]);
}

__global__ void k_sub(const double* __restrict__ b, const double* __restrict__ a, double* __restrict__ r,
                      int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  r[e] = b[e] - a[e];
}

__global__ void k_xupdate(double* __restrict__ x, const double* __restrict__ V, const double* __restrict__ y,
                          int k, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double acc = x[e];
  for (int i = 0; i < k; ++i) acc = fma(y[i], V[(int64_t)i * n + e], acc);
  x[e] = acc;
}

__global__ void k_fill_diag(double* __restrict__ diag, const DropDev* __restrict__ drops, int n_drops,
                            int sys, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  if (sys == SHBIM_SYS_ELECTRIC) {
    diag[e] = 0.5;
    return;
  }
  int i = 0;
  while (i + 1 < n_drops && 3 * drops[i + 1].coef_off <= e) ++i;
  diag[e] = drops[i].lam + 1.0;
}

// Diffusion preconditioner: one block per drop sums the area (weights omega J of the source
// grid) and writes 1/(1 + c n(n+1)/a^2) for the drop's coefficients (index n*n + n + m).
__global__ void k_fill_minv(double* __restrict__ minv, const DropDev* __restrict__ drops,
                            const double* __restrict__ src, int64_t nsource, double c) {
  const DropDev D = drops[blockIdx.x];
  double a = 0.0;
  for (int64_t e = threadIdx.x; e < D.ns; e += blockDim.x) a += src[6 * nsource + D.src_off + e];
  a = block_sum(a);
  __shared__ double area;
  if (threadIdx.x == 0) area = a;
  __syncthreads();
  const double a2 = area / (4.0 * 3.14159265358979323846);
  for (int k = threadIdx.x; k < D.nc; k += blockDim.x) {
    int n = (int)sqrt((double)k);
    while (n * n > k) --n;
    while ((n + 1) * (n + 1) <= k) ++n;
    minv[D.coef_off + k] = 1.0 / (1.0 + c * n * (n + 1.0) / a2);
  }
}

__global__ void k_mul(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                      int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = a[e] * b[e];
}

__global__ void k_div(double* __restrict__ y, const double* __restrict__ a, const double* __restrict__ b,
                      int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] = a[e] / b[e];
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// ---- GMRES cycles on the device (the state of a cycle lives in device memory; every kernel reads the
// Arnoldi index k from it, so one captured graph serves every step of a cycle)
struct DevCycle {
  double* H;    // (m+1) x m, column-major: column k at k (m+1)
  double* cs;   // m
  double* sn;   // m
  double* g;    // m+1
  double* y;    // m
  double* sc;   // 0 residual estimate, 1 ||b||, 2 tolerance, 3 beta
  int* is;      // 0 k, 1 total Arnoldi steps, 2 flags (bit 0: non-finite), 3 step budget
  int m;
};

DevCycle dev_cycle(double* dstate, int* istate, int m) {
  DevCycle C;
  C.H = dstate;
  C.cs = C.H + (size_t)(m + 1) * m;
  C.sn = C.cs + m;
  C.g = C.sn + m;
  C.y = C.g + m + 1;
  C.sc = C.y + m;
  C.is = istate;
  C.m = m;
  return C;
}

size_t dev_cycle_doubles(int m) { return (size_t)(m + 1) * m + 3 * (size_t)m + (m + 1) + 8; }

__device__ __forceinline__ unsigned cycle_go(const DevCycle& C) {
  return (C.is[2] == 0 && C.sc[0] > C.sc[2] && C.is[0] < C.m && C.is[1] < C.is[3]) ? 1u : 0u;
}

__global__ void k_cycle_cond(cudaGraphConditionalHandle h, DevCycle C) { cudaGraphSetConditional(h, cycle_go(C)); }

__global__ void k_stage_vk(const double* __restrict__ V, int64_t n, const int* __restrict__ is, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = V[(int64_t)is[0] * n + e];
}

// h[i] = V_i . w for i <= k (one block per vector; blocks past k return)
__global__ void k_dots_k(const double* __restrict__ V, int64_t n, const double* __restrict__ w,
                         double* __restrict__ h, const int* __restrict__ is) {
  if ((int)blockIdx.x > is[0]) return;
  const double* v = V + (int64_t)blockIdx.x * n;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(v[e], w[e], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) h[blockIdx.x] = acc;
}

__global__ void k_orth_update_k(double* __restrict__ w, const double* __restrict__ V, int64_t n,
                                const double* __restrict__ h, double* __restrict__ hacc, int first,
                                const int* __restrict__ is) {
  const int nvec = is[0] + 1;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    for (int i = 0; i < nvec; ++i) hacc[i] = first ? h[i] : hacc[i] + h[i];
  }
  if (e >= n) return;
  double acc = w[e];
  for (int i = 0; i < nvec; ++i) acc = fma(-h[i], V[(int64_t)i * n + e], acc);
  w[e] = acc;
}

__global__ void k_norm2_k(const double* __restrict__ w, int64_t n, double* __restrict__ hacc, const int* __restrict__ is) {
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc = fma(w[e], w[e], acc);
  acc = block_sum(acc);
  if (threadIdx.x == 0) hacc[is[0] + 1] = acc;
}

__global__ void k_normalize_k(const double* __restrict__ w, const double* __restrict__ hacc, double* __restrict__ V,
                              int64_t n, const int* __restrict__ is) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double nr = hacc[is[0] + 1];
  const double sc = nr > 0.0 ? 1.0 / sqrt(nr) : 0.0;
  V[(int64_t)(is[0] + 1) * n + e] = w[e] * sc;
}

// the new Hessenberg column, its Givens rotation, the residual estimate and the loop condition
__global__ void k_givens(cudaGraphConditionalHandle h, DevCycle C, const double* __restrict__ hacc) {
  const int k = C.is[0], ld = C.m + 1;
  double* Hc = C.H + (size_t)k * ld;
  for (int i = 0; i <= k; ++i) Hc[i] = hacc[i];
  Hc[k + 1] = sqrt(fmax(0.0, hacc[k + 1]));
  bool finite = true;
  for (int i = 0; i <= k + 1; ++i) finite = finite && isfinite(Hc[i]);
  for (int i = 0; i < k; ++i) {
    const double a = Hc[i], b = Hc[i + 1];
    Hc[i] = C.cs[i] * a + C.sn[i] * b;
    Hc[i + 1] = -C.sn[i] * a + C.cs[i] * b;
  }
  const double den = hypot(Hc[k], Hc[k + 1]);
  C.cs[k] = den > 0.0 ? Hc[k] / den : 1.0;
  C.sn[k] = den > 0.0 ? Hc[k + 1] / den : 0.0;
  Hc[k] = den;
  Hc[k + 1] = 0.0;
  C.g[k + 1] = -C.sn[k] * C.g[k];
  C.g[k] = C.cs[k] * C.g[k];
  C.is[0] = k + 1;
  C.is[1] += 1;
  C.sc[0] = C.sc[1] > 0.0 ? fabs(C.g[k + 1]) / C.sc[1] : 0.0;
  if (!finite || !isfinite(C.sc[0])) C.is[2] |= 1;
  cudaGraphSetConditional(h, cycle_go(C));
}

// y = R^{-1} g for the current k
__global__ void k_backsolve(DevCycle C) {
  const int k = C.is[0], ld = C.m + 1;
  for (int i = k - 1; i >= 0; --i) {
    double acc = C.g[i];
    for (int c = i + 1; c < k; ++c) acc -= C.H[(size_t)c * ld + i] * C.y[c];
    C.y[i] = acc / C.H[(size_t)i * ld + i];
  }
}

__global__ void k_xupdate_k(double* __restrict__ x, const double* __restrict__ V, const double* __restrict__ y,
                            const int* __restrict__ is, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = is[0];
  double acc = x[e];
  for (int i = 0; i < k; ++i) acc = fma(y[i], V[(int64_t)i * n + e], acc);
  x[e] = acc;
}

// ---- Stokes preconditioner (right). On drop i the self part of the Stokes system,
// (lam_i+1) u - (lam_i-1) D_i[u], maps the six rigid-body motions of the drop to 2 u (D reproduces a
// rigid motion on a closed surface) and, on a sphere, the normal field to 2 lam_i u (the double layer's
// eigenvalue -1); the other modes have eigenvalues (lam_i+1) - (lam_i-1) mu with |mu| <= 3/5, clustered
// near lam_i + 1. With Q_i an orthonormal basis of the rigid motions (coefficient inner product) and r_i
// the unit normal mode of the parameter sphere orthogonalised against them,
//   P_i^{-1} v = v/(lam_i+1) + (1/2 - 1/(lam_i+1)) Q_i Q_i^T v + (1/(2 lam_i) - 1/(lam_i+1)) r_i r_i^T v
// maps those outlying eigenvalues to 1 and the cluster near 1 (P_i is the same form with the inverse
// factors). GMRES iterates y = P x and applies A P^{-1}; the solution is x = P^{-1} y.

// dots[drop][k] = basis_k . v over the drop's 3 nc coefficients (one block per drop, fixed order)
__global__ void k_prec_dots(const double* __restrict__ v, const double* __restrict__ basis,
                            const DropDev* __restrict__ drops, double* __restrict__ dots) {
  __shared__ double red[7][32];
  const DropDev D = drops[blockIdx.x];
  const int64_t n3 = 3 * (int64_t)D.nc;
  const double* vv = v + 3 * D.coef_off;
  const double* B = basis + 21 * D.coef_off;
  double acc[7];
#pragma unroll
  for (int k = 0; k < 7; ++k) acc[k] = 0.0;
  for (int64_t e = threadIdx.x; e < n3; e += blockDim.x) {
    const double x = vv[e];
#pragma unroll
    for (int k = 0; k < 7; ++k) acc[k] = fma(B[k * n3 + e], x, acc[k]);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double a = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[k][wid] = a;
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    double a = 0.0;
    for (int w = 0; w < nw; ++w) a += red[threadIdx.x][w];
    dots[7 * blockIdx.x + threadIdx.x] = a;
  }
}

// out = f0 v + f1 Q Q^T v + f2 r r^T v per drop (f: inverse or forward factors)
__global__ void k_prec_apply(const double* __restrict__ v, const double* __restrict__ basis,
                             const DropDev* __restrict__ drops, const double* __restrict__ dots,
                             const double* __restrict__ fac, int forward, double* __restrict__ out) {
  const DropDev D = drops[blockIdx.y];
  const int64_t n3 = 3 * (int64_t)D.nc;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n3) return;
  const double* f = fac + 6 * blockIdx.y + (forward ? 3 : 0);
  const double* B = basis + 21 * D.coef_off;
  const double* z = dots + 7 * blockIdx.y;
  double q = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) q = fma(z[k], B[k * n3 + e], q);
  const int64_t o = 3 * D.coef_off + e;
  out[o] = f[0] * v[o] + f[1] * q + f[2] * (z[6] * B[6 * n3 + e]);
}

int prec_apply(shbim_ctx* ctx, const double* v, double* out, bool forward, cudaStream_t s) {
  int maxn3 = 0;
  for (const auto& d : ctx->drops) maxn3 = std::max(maxn3, 3 * d.nc);
  k_prec_dots<<<ctx->n_drops, 256, 0, s>>>(v, ctx->prec_basis, ctx->drops_dev, ctx->prec_dots);
  SHBIM_CHECK_LAUNCH(ctx, "k_prec_dots");
  k_prec_apply<<<dim3((unsigned)((maxn3 + 255) / 256), (unsigned)ctx->n_drops), 256, 0, s>>>(
      v, ctx->prec_basis, ctx->drops_dev, ctx->prec_dots, ctx->prec_fac, forward ? 1 : 0, out);
  SHBIM_CHECK_LAUNCH(ctx, "k_prec_apply");
  return SHBIM_OK;
}

inline int64_t system_size(const shbim_ctx* ctx, int sys) {
  return sys == SHBIM_SYS_STOKES ? 3 * ctx->ncoef : ctx->ncoef;
}

int matvec_eager(shbim_ctx* ctx, const double* v, double* out, cudaStream_t s) {
  auto& G = ctx->gm;
  if (G.sys == SHBIM_SYS_DIFFUSION) {
    k_mul<<<nb(G.n), 256, 0, s>>>(G.tmp, G.diag, v, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_mul");
    int rc = laplace_beltrami(ctx, G.tmp, G.Av, s);
    if (rc) return rc;
    k_system<<<nb(G.n), 256, 0, s>>>(G.diag, G.offdiag, v, G.Av, out, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_system");
    return SHBIM_OK;  // not a layer-operator application
  }
  if (G.sys == SHBIM_SYS_STOKES && G.prec && !G.raw) {
    // A P^{-1} v
    int rc = prec_apply(ctx, v, G.tmp, false, s);
    if (rc || (rc = shbim_eval_stokes(ctx, nullptr, G.tmp, G.Av, SHBIM_OUT_COEF, s))) return rc;
    k_system<<<nb(G.n), 256, 0, s>>>(G.diag, G.offdiag, G.tmp, G.Av, out, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_system");
    return SHBIM_OK;
  }
  int rc = G.sys == SHBIM_SYS_ELECTRIC
               ? shbim_eval_electric(ctx, SHBIM_LAPLACE_DL, v, G.Av, SHBIM_OUT_COEF, s)
               : shbim_eval_stokes(ctx, nullptr, v, G.Av, SHBIM_OUT_COEF, s);
  if (rc) return rc;
  k_system<<<nb(G.n), 256, 0, s>>>(G.diag, G.offdiag, v, G.Av, out, G.n);
  SHBIM_CHECK_LAUNCH(ctx, "k_system");
  return SHBIM_OK;
}

// Operator application of the current system. With graphs on, the second application for a
// given geometry, system and precision is captured on the library's stream (input and output
// through fixed staging buffers) and later ones replay the graph on the caller's stream.
int system_matvec(shbim_ctx* ctx, const double* v, double* out, cudaStream_t s) {
  auto& G = ctx->gm;
  // applications of the system itself (refinement residuals) are not the captured preconditioned form
  if (!ctx->graphs_on || G.raw) return matvec_eager(ctx, v, out, s);
  auto& GR = ctx->graphs[G.sys * 3 + ctx->opts.precision];
  if (GR.version != ctx->geom_version || GR.n != G.n) {
    if (GR.exec) cudaGraphExecDestroy(GR.exec);
    GR.exec = nullptr;
    GR.warm = false;
    GR.version = ctx->geom_version;
    if (GR.n < G.n) {
      cudaFree(GR.in);
      cudaFree(GR.out);
      GR.in = GR.out = nullptr;
      if (cudaMalloc(&GR.in, G.n * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&GR.out, G.n * sizeof(double)) != cudaSuccess)
        return fail(ctx, SHBIM_ERR_NOMEM, "graph staging buffers");
    }
    GR.n = G.n;
  }
  if (!GR.exec) {
    if (!GR.warm) {  // first application: eager, sizes every workspace
      GR.warm = true;
      return matvec_eager(ctx, v, out, s);
    }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      return matvec_eager(ctx, v, out, s);
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    cudaGraph_t graph = nullptr;
    const int64_t l0 = ctx->launches, a0 = ctx->applications;
    SHBIM_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = matvec_eager(ctx, GR.in, GR.out, ctx->cap_stream);
    const cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    GR.kernels = ctx->launches - l0;
    ctx->launches = l0;
    ctx->applications = a0;
    if (rc || ce != cudaSuccess || !graph) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      ctx->graphs_on = false;  // fall back to eager launches for this context
      return matvec_eager(ctx, v, out, s);
    }
    const cudaError_t ie = cudaGraphInstantiate(&GR.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      GR.exec = nullptr;
      cudaGetLastError();
      ctx->graphs_on = false;
      return matvec_eager(ctx, v, out, s);
    }
  }
  SHBIM_CUDA(ctx, cudaMemcpyAsync(GR.in, v, G.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SHBIM_CUDA(ctx, cudaGraphLaunch(GR.exec, s));
  SHBIM_CUDA(ctx, cudaMemcpyAsync(out, GR.out, G.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ctx->launches += GR.kernels;
  if (G.sys != SHBIM_SYS_DIFFUSION) ctx->applications += 1;
  return SHBIM_OK;
}

double* hacc_ptr(shbim_ctx* ctx) { return ctx->gm.h + (ctx->gm.m + 2); }

// ||src||^2 into hacc[slot] and src/||src|| into dst; returns the norm read back on the host
int normalize_into(shbim_ctx* ctx, const double* src, double* dst, int slot, double* norm, cudaStream_t s) {
  auto& G = ctx->gm;
  double* hacc = hacc_ptr(ctx);
  k_dots<<<1, 256, 0, s>>>(src, G.n, src, hacc + slot);
  SHBIM_CHECK_LAUNCH(ctx, "k_dots");
  k_normalize<<<nb(G.n), 256, 0, s>>>(src, hacc + slot, dst, G.n);
  SHBIM_CHECK_LAUNCH(ctx, "k_normalize");
  SHBIM_CUDA(ctx, cudaMemcpyAsync(G.h_host, hacc + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  *norm = std::sqrt(std::max(0.0, G.h_host[0]));
  if (!std::isfinite(*norm)) return fail(ctx, SHBIM_ERR_NONFINITE, "non-finite norm in GMRES");
  return SHBIM_OK;
}

// start a cycle from the current x: V0 = (b - A x)/beta
int start_cycle(shbim_ctx* ctx, bool x_is_zero, cudaStream_t s) {
  auto& G = ctx->gm;
  int rc;
  if (x_is_zero) {
    SHBIM_CUDA(ctx, cudaMemcpyAsync(G.w, G.b, G.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    if ((rc = system_matvec(ctx, G.x, G.w, s))) return rc;
    k_sub<<<nb(G.n), 256, 0, s>>>(G.b, G.w, G.w, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_sub");
  }
  double beta = 0.0;
  if ((rc = normalize_into(ctx, G.w, G.V, 0, &beta, s))) return rc;
  std::fill(G.g.begin(), G.g.end(), 0.0);
  G.g[0] = beta;
  G.k = 0;
  G.resid = G.bnorm > 0.0 ? beta / G.bnorm : 0.0;
  return SHBIM_OK;
}

// Build (or reuse) the graph of one device cycle of the current system at the context's precision:
// a kernel that sets the loop condition, the conditional 'while' node whose body is one Arnoldi step
// (stage V_k, operator application, two Gram-Schmidt passes, norm, normalisation, Givens rotation and
// the convergence test that sets the condition), then the back substitution and the update of x.
// Returns false (and marks the slot) if the graph cannot be built; the caller then steps on the host.
bool cycle_graph(shbim_ctx* ctx, cudaStream_t s) {
  auto& G = ctx->gm;
  auto& CG = ctx->cycles[G.sys * 3 + ctx->opts.precision];
  if (CG.failed) return false;
  if (CG.exec && CG.version == ctx->geom_version && CG.n == G.n && CG.m == G.m) return true;
  if (CG.exec) cudaGraphExecDestroy(CG.exec);
  CG.exec = nullptr;
  // the operator's workspaces must exist before capture: one eager application per slot and geometry
  auto& GR = ctx->graphs[G.sys * 3 + ctx->opts.precision];
  if (GR.version != ctx->geom_version || !GR.warm) return false;
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    CG.failed = true;
    return false;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return false;
  const DevCycle C = dev_cycle(G.dstate, G.istate, G.m);
  const int64_t n = G.n;
  double* hacc = hacc_ptr(ctx);
  double* htmp = G.h;
  cudaGraph_t graph = nullptr;
  cudaGraphConditionalHandle handle;
  cudaGraphNode_t pre = nullptr, cond = nullptr;
  size_t nn = 1;
  const int64_t l0 = ctx->launches, a0 = ctx->applications;
  bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess &&
            cudaGraphConditionalHandleCreate(&handle, graph, 0, cudaGraphCondAssignDefault) == cudaSuccess;
  // the condition for the first step
  ok = ok && cudaStreamBeginCaptureToGraph(ctx->cap_stream, graph, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    k_cycle_cond<<<1, 1, 0, ctx->cap_stream>>>(handle, C);
    ok = cudaStreamEndCapture(ctx->cap_stream, &graph) == cudaSuccess;
  }
  ok = ok && cudaGraphGetNodes(graph, &pre, &nn) == cudaSuccess && nn == 1;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  ok = ok && cudaGraphAddNode(&cond, graph, &pre, nullptr, 1, &cp) == cudaSuccess;
  int64_t body_kernels = 0;
  if (ok) {
    // the body: one Arnoldi step
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    ok = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      cudaStream_t cs = ctx->cap_stream;
      const int64_t b0 = ctx->launches;
      k_stage_vk<<<nb(n), 256, 0, cs>>>(G.V, n, G.istate, G.vstage);
      int rc = matvec_eager(ctx, G.vstage, G.w, cs);
      for (int pass = 0; pass < 2 && rc == SHBIM_OK; ++pass) {
        k_dots_k<<<G.m + 1, 256, 0, cs>>>(G.V, n, G.w, htmp, G.istate);
        k_orth_update_k<<<nb(n), 256, 0, cs>>>(G.w, G.V, n, htmp, hacc, pass == 0, G.istate);
      }
      k_norm2_k<<<1, 256, 0, cs>>>(G.w, n, hacc, G.istate);
      k_normalize_k<<<nb(n), 256, 0, cs>>>(G.w, hacc, G.V, n, G.istate);
      k_givens<<<1, 1, 0, cs>>>(handle, C, hacc);
      body_kernels = ctx->launches - b0 + 8;
      cudaGraph_t b2 = nullptr;
      const cudaError_t e = cudaStreamEndCapture(cs, &b2);
      ok = rc == SHBIM_OK && e == cudaSuccess;
    }
  }
  // back substitution and the update of x after the loop
  ok = ok && cudaStreamBeginCaptureToGraph(ctx->cap_stream, graph, &cond, nullptr, 1,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    k_backsolve<<<1, 1, 0, ctx->cap_stream>>>(C);
    k_xupdate_k<<<nb(n), 256, 0, ctx->cap_stream>>>(G.x, G.V, C.y, G.istate, n);
    ok = cudaStreamEndCapture(ctx->cap_stream, &graph) == cudaSuccess;
  }
  ok = ok && cudaGraphInstantiate(&CG.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  ctx->launches = l0;
  ctx->applications = a0;
  if (!ok) {
    if (CG.exec) cudaGraphExecDestroy(CG.exec);
    CG.exec = nullptr;
    CG.failed = true;
    cudaGetLastError();
    return false;
  }
  CG.version = ctx->geom_version;
  CG.n = G.n;
  CG.m = G.m;
  CG.body_kernels = body_kernels;
  return true;
}

// Run the current solve's remaining steps as device cycles, from whatever state the host holds (the
// Hessenberg columns, rotations and g of the cycle so far are copied to the device first). *done = true
// when the solve converged; false when the graph is unavailable (nothing changed: the caller steps on
// the host).
int device_cycles(shbim_ctx* ctx, cudaStream_t s, bool* done) {
  auto& G = ctx->gm;
  *done = false;
  if (G.resid <= ctx->opts.gmres_tol) {
    *done = true;
    return SHBIM_OK;
  }
  if (!cycle_graph(ctx, s)) return SHBIM_OK;
  auto& CG = ctx->cycles[G.sys * 3 + ctx->opts.precision];
  const DevCycle C = dev_cycle(G.dstate, G.istate, G.m);
  double* sc_h = G.h_host + 2 * (G.m + 2);
  int* is_h = reinterpret_cast<int*>(sc_h + 4);
  for (;;) {
    // the host's state of the current cycle
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.H, G.H.data(), G.H.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.cs, G.cs.data(), G.m * sizeof(double), cudaMemcpyHostToDevice, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.sn, G.sn.data(), G.m * sizeof(double), cudaMemcpyHostToDevice, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.g, G.g.data(), (G.m + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
    sc_h[0] = G.resid;
    sc_h[1] = G.bnorm;
    sc_h[2] = ctx->opts.gmres_tol;
    sc_h[3] = G.g[0];
    is_h[0] = G.k;
    is_h[1] = G.total;
    is_h[2] = 0;
    is_h[3] = ctx->opts.gmres_maxiter;
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.sc, sc_h, 4 * sizeof(double), cudaMemcpyHostToDevice, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(C.is, is_h, 4 * sizeof(int), cudaMemcpyHostToDevice, s));
    SHBIM_CUDA(ctx, cudaGraphLaunch(CG.exec, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(is_h, C.is, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    SHBIM_CUDA(ctx, cudaMemcpyAsync(sc_h, C.sc, sizeof(double), cudaMemcpyDeviceToHost, s));
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    const int steps = is_h[1] - G.total;
    G.total = is_h[1];
    G.resid = sc_h[0];
    G.k = 0;  // the graph has already added V y to x
    ctx->launches += 3 + (int64_t)steps * CG.body_kernels;
    if (G.sys != SHBIM_SYS_DIFFUSION) ctx->applications += steps;
    if (is_h[2] & 1) return fail(ctx, SHBIM_ERR_NONFINITE, "non-finite Arnoldi column");
    if (G.resid <= ctx->opts.gmres_tol) break;
    if (G.total >= ctx->opts.gmres_maxiter)
      return fail(ctx, SHBIM_ERR_NOT_CONVERGED, "GMRES reached its iteration limit");
    // Krylov space full: restart from the true residual
    int rc = start_cycle(ctx, false, s);
    if (rc) return rc;
    if (G.resid <= ctx->opts.gmres_tol) break;
  }
  *done = true;
  return SHBIM_OK;
}

// y = R^{-1} g for the rotated Hessenberg matrix of the current cycle, x += V y
int update_x(shbim_ctx* ctx, cudaStream_t s) {
  auto& G = ctx->gm;
  const int k = G.k;
  if (k == 0) return SHBIM_OK;
  const int ld = G.m + 1;
  std::vector<double> y(k);
  for (int i = k - 1; i >= 0; --i) {
    double acc = G.g[i];
    for (int c = i + 1; c < k; ++c) acc -= G.H[(size_t)c * ld + i] * y[c];
    y[i] = acc / G.H[(size_t)i * ld + i];
  }
  std::copy(y.begin(), y.end(), G.h_host);
  SHBIM_CUDA(ctx, cudaMemcpyAsync(G.y, G.h_host, k * sizeof(double), cudaMemcpyHostToDevice, s));
  k_xupdate<<<nb(G.n), 256, 0, s>>>(G.x, G.V, G.y, k, G.n);
  SHBIM_CHECK_LAUNCH(ctx, "k_xupdate");
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));  // h_host is reused by the next read-back
  G.k = 0;
  return SHBIM_OK;
}

}  // namespace

// Basis of the Stokes preconditioner for the current geometry: per drop the translations e_k (constant
// fields, coefficient sqrt(4 pi) on Y_00), the rotations e_k x x (from the position coefficients) and
// the parameter sphere's radial field r^ (degree 1), orthonormalised in that order in FP64 (modified
// Gram-Schmidt, twice); factors from the drop's viscosity ratio.
int build_stokes_preconditioner(shbim_ctx* ctx, const double* xcoef_dev, cudaStream_t s) {
  const int64_t nc_all = ctx->ncoef;
  if (!ctx->prec_basis) {
    if (cudaMalloc(&ctx->prec_basis, (size_t)21 * nc_all * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->prec_dots, (size_t)7 * ctx->n_drops * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->prec_fac, (size_t)6 * ctx->n_drops * sizeof(double)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "Stokes preconditioner allocation failed");
  }
  std::vector<double> x((size_t)3 * nc_all), B((size_t)21 * nc_all, 0.0), F((size_t)6 * ctx->n_drops);
  SHBIM_CUDA(ctx, cudaMemcpyAsync(x.data(), xcoef_dev, x.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  const double s4pi = std::sqrt(4.0 * kPi), s4pi3 = std::sqrt(4.0 * kPi / 3.0);
  for (int i = 0; i < ctx->n_drops; ++i) {
    const Drop& d = ctx->drops[i];
    const int64_t nc = d.nc, n3 = 3 * nc;
    const double* xc = x.data() + 3 * d.coef_off;
    double* b = B.data() + 21 * d.coef_off;
    for (int k = 0; k < 3; ++k) b[k * n3 + k * nc] = s4pi;
    for (int k = 0; k < 3; ++k) {
      double* v = b + (3 + k) * n3;
      const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      // (e_k x x)_{k1} = -x_{k2}, (e_k x x)_{k2} = x_{k1}
      for (int64_t j = 0; j < nc; ++j) {
        v[k1 * nc + j] = -xc[k2 * nc + j];
        v[k2 * nc + j] = xc[k1 * nc + j];
      }
    }
    double* r = b + 6 * n3;
    r[0 * nc + 3] = -s4pi3;   // x: -sqrt(4 pi/3) on the (1, 1) harmonic
    r[1 * nc + 1] = -s4pi3;   // y: -sqrt(4 pi/3) on the (1, -1) harmonic
    r[2 * nc + 2] = s4pi3;    // z:  sqrt(4 pi/3) on the (1, 0) harmonic
    for (int k = 0; k < 7; ++k) {
      double* v = b + k * n3;
      for (int pass = 0; pass < 2; ++pass)
        for (int l = 0; l < k; ++l) {
          const double* u = b + l * n3;
          double dot = 0.0;
          for (int64_t j = 0; j < n3; ++j) dot += u[j] * v[j];
          for (int64_t j = 0; j < n3; ++j) v[j] -= dot * u[j];
        }
      double nrm = 0.0;
      for (int64_t j = 0; j < n3; ++j) nrm += v[j] * v[j];
      nrm = std::sqrt(nrm);
      if (!(nrm > 1e-12)) return fail(ctx, SHBIM_ERR_ARG, "degenerate drop shape for the Stokes preconditioner");
      for (int64_t j = 0; j < n3; ++j) v[j] /= nrm;
    }
    const double lam = d.lam, a = 1.0 / (lam + 1.0);
    double* f = F.data() + 6 * i;
    f[0] = a;
    f[1] = 0.5 - a;
    f[2] = 0.5 / lam - a;
    f[3] = lam + 1.0;
    f[4] = 2.0 - (lam + 1.0);
    f[5] = 2.0 * lam - (lam + 1.0);
  }
  SHBIM_CUDA(ctx, cudaMemcpy(ctx->prec_basis, B.data(), B.size() * sizeof(double), cudaMemcpyHostToDevice));
  SHBIM_CUDA(ctx, cudaMemcpy(ctx->prec_fac, F.data(), F.size() * sizeof(double), cudaMemcpyHostToDevice));
  return SHBIM_OK;
}

}  // namespace shbim

using namespace shbim;

extern "C" {

int shbim_set_stokes_preconditioner(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->stokes_prec = on != 0;
  ctx->geom_version++;  // captured applications and device cycles hold the other form
  return SHBIM_OK;
}

int shbim_gmres_begin(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (sys != SHBIM_SYS_ELECTRIC && sys != SHBIM_SYS_STOKES && sys != SHBIM_SYS_DIFFUSION)
    return fail(ctx, SHBIM_ERR_ARG, "bad system");
  if (!rhs_dev) return fail(ctx, SHBIM_ERR_ARG, "null right-hand side");
  cudaStream_t s = (cudaStream_t)stream;
  auto& G = ctx->gm;
  const int64_t n = system_size(ctx, sys);
  const int m = ctx->opts.gmres_restart;
  if (n * (m + 1) > G.cap || m != G.m || !G.V) {
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    cudaFree(G.V); cudaFree(G.w); cudaFree(G.x); cudaFree(G.b); cudaFree(G.h); cudaFree(G.Av);
    cudaFree(G.diag); cudaFree(G.tmp); cudaFree(G.y); cudaFree(G.dstate); cudaFree(G.istate); cudaFree(G.vstage);
    if (G.h_host) cudaFreeHost(G.h_host);
    G.V = G.w = G.x = G.b = G.h = G.Av = G.diag = G.tmp = G.y = G.h_host = G.dstate = G.vstage = nullptr;
    G.istate = nullptr;
    const int64_t ncap = std::max<int64_t>(n, 3 * ctx->ncoef);
    if (cudaMalloc(&G.V, (size_t)ncap * (m + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.w, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.x, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.b, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.Av, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.diag, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.tmp, ncap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.y, (m + 2) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.h, 2 * (m + 2) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.dstate, dev_cycle_doubles(m) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.istate, 4 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&G.vstage, ncap * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&G.h_host, (2 * (m + 2) + 8) * sizeof(double)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "GMRES workspace allocation failed");
    G.cap = ncap * (m + 1);
    G.m = m;
    ctx->geom_version++;  // captured operator graphs referenced the old workspaces
  }
  G.sys = sys;
  G.n = n;
  G.H.assign((size_t)(m + 1) * m, 0.0);
  G.cs.assign(m, 0.0);
  G.sn.assign(m, 0.0);
  G.g.assign(m + 1, 0.0);
  G.total = 0;
  G.k = 0;
  const double R = ctx->opts.R;
  if (sys == SHBIM_SYS_DIFFUSION) {
    G.offdiag = -ctx->diff_c;
    k_fill_minv<<<ctx->n_drops, 256, 0, s>>>(G.diag, ctx->drops_dev, ctx->geo.src, ctx->nsource, ctx->diff_c);
    SHBIM_CHECK_LAUNCH(ctx, "k_fill_minv");
  } else {
    G.offdiag = sys == SHBIM_SYS_ELECTRIC ? -(R - 1.0) / (R + 1.0) : -1.0;
    k_fill_diag<<<nb(n), 256, 0, s>>>(G.diag, ctx->drops_dev, ctx->n_drops, sys, n);
    SHBIM_CHECK_LAUNCH(ctx, "k_fill_diag");
  }
  G.raw = false;
  G.prec = sys == SHBIM_SYS_STOKES && ctx->stokes_prec && ctx->prec_basis;
  SHBIM_CUDA(ctx, cudaMemcpyAsync(G.b, rhs_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (x0_dev && sys == SHBIM_SYS_DIFFUSION) {  // the iterate is y = M x
    k_div<<<nb(n), 256, 0, s>>>(G.x, x0_dev, G.diag, n);
    SHBIM_CHECK_LAUNCH(ctx, "k_div");
  } else if (x0_dev && G.prec) {  // the iterate is y = P x
    if (int rc = prec_apply(ctx, x0_dev, G.x, true, s)) return rc;
  } else if (x0_dev) {
    SHBIM_CUDA(ctx, cudaMemcpyAsync(G.x, x0_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    SHBIM_CUDA(ctx, cudaMemsetAsync(G.x, 0, n * sizeof(double), s));
  }
  // ||b||
  double* hacc = hacc_ptr(ctx);
  k_dots<<<1, 256, 0, s>>>(G.b, n, G.b, hacc);
  SHBIM_CHECK_LAUNCH(ctx, "k_dots");
  SHBIM_CUDA(ctx, cudaMemcpyAsync(G.h_host, hacc, sizeof(double), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  G.bnorm = std::sqrt(std::max(0.0, G.h_host[0]));
  if (!std::isfinite(G.bnorm)) return fail(ctx, SHBIM_ERR_NONFINITE, "non-finite right-hand side");
  if (G.bnorm == 0.0) {
    SHBIM_CUDA(ctx, cudaMemsetAsync(G.x, 0, n * sizeof(double), s));
    G.resid = 0.0;
    return SHBIM_OK;
  }
  return start_cycle(ctx, x0_dev == nullptr, s);
}

int shbim_gmres_step(shbim_ctx* ctx, double* resid_host, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  auto& G = ctx->gm;
  if (G.sys < 0) return fail(ctx, SHBIM_ERR_ARG, "shbim_gmres_begin was not called");
  cudaStream_t s = (cudaStream_t)stream;
  if (resid_host) *resid_host = G.resid;
  if (G.resid <= ctx->opts.gmres_tol) return SHBIM_CONVERGED;
  if (G.total >= ctx->opts.gmres_maxiter)
    return fail(ctx, SHBIM_ERR_NOT_CONVERGED, "GMRES reached its iteration limit");
  int rc;
  const int k = G.k;
  const int64_t n = G.n;
  double* vk = G.V + (int64_t)k * n;
  if ((rc = system_matvec(ctx, vk, G.w, s))) return rc;
  double* htmp = G.h;
  double* hacc = hacc_ptr(ctx);
  for (int pass = 0; pass < 2; ++pass) {
    k_dots<<<k + 1, 256, 0, s>>>(G.V, n, G.w, htmp);
    SHBIM_CHECK_LAUNCH(ctx, "k_dots");
    k_orth_update<<<nb(n), 256, 0, s>>>(G.w, G.V, n, k + 1, htmp, hacc, pass == 0);
    SHBIM_CHECK_LAUNCH(ctx, "k_orth_update");
  }
  k_dots<<<1, 256, 0, s>>>(G.w, n, G.w, hacc + k + 1);
  SHBIM_CHECK_LAUNCH(ctx, "k_dots");
  k_normalize<<<nb(n), 256, 0, s>>>(G.w, hacc + k + 1, G.V + (int64_t)(k + 1) * n, n);
  SHBIM_CHECK_LAUNCH(ctx, "k_normalize");
  SHBIM_CUDA(ctx, cudaMemcpyAsync(G.h_host, hacc, (k + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  const int ld = G.m + 1;
  double* Hc = &G.H[(size_t)k * ld];
  for (int i = 0; i <= k; ++i) Hc[i] = G.h_host[i];
  Hc[k + 1] = std::sqrt(std::max(0.0, G.h_host[k + 1]));
  for (int i = 0; i <= k + 1; ++i)
    if (!std::isfinite(Hc[i])) return fail(ctx, SHBIM_ERR_NONFINITE, "non-finite Arnoldi column");
  for (int i = 0; i < k; ++i) {
    const double a = Hc[i], b = Hc[i + 1];
    Hc[i] = G.cs[i] * a + G.sn[i] * b;
    Hc[i + 1] = -G.sn[i] * a + G.cs[i] * b;
  }
  const double den = std::hypot(Hc[k], Hc[k + 1]);
  G.cs[k] = den > 0.0 ? Hc[k] / den : 1.0;
  G.sn[k] = den > 0.0 ? Hc[k + 1] / den : 0.0;
  Hc[k] = den;
  Hc[k + 1] = 0.0;
  G.g[k + 1] = -G.sn[k] * G.g[k];
  G.g[k] = G.cs[k] * G.g[k];
  G.k = k + 1;
  G.total++;
  G.resid = std::fabs(G.g[k + 1]) / G.bnorm;
  if (resid_host) *resid_host = G.resid;
  if (G.resid <= ctx->opts.gmres_tol) return SHBIM_CONVERGED;
  if (G.k == G.m) {
    // restart from the true residual of the updated iterate
    if ((rc = update_x(ctx, s))) return rc;
    if ((rc = start_cycle(ctx, false, s))) return rc;
    if (resid_host) *resid_host = G.resid;
    if (G.resid <= ctx->opts.gmres_tol) return SHBIM_CONVERGED;
  }
  if (G.total >= ctx->opts.gmres_maxiter)
    return fail(ctx, SHBIM_ERR_NOT_CONVERGED, "GMRES reached its iteration limit");
  return SHBIM_CONTINUE;
}

int shbim_gmres_finish(shbim_ctx* ctx, double* x_dev, int* iters_host, void* stream) {
  if (!ctx || !x_dev) return SHBIM_ERR_ARG;
  auto& G = ctx->gm;
  if (G.sys < 0) return fail(ctx, SHBIM_ERR_ARG, "shbim_gmres_begin was not called");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = update_x(ctx, s);
  if (rc) return rc;
  if (G.sys == SHBIM_SYS_DIFFUSION) {
    k_mul<<<nb(G.n), 256, 0, s>>>(x_dev, G.diag, G.x, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_mul");
  } else if (G.sys == SHBIM_SYS_STOKES && G.prec) {
    if ((rc = prec_apply(ctx, G.x, x_dev, false, s))) return rc;
  } else {
    SHBIM_CUDA(ctx, cudaMemcpyAsync(x_dev, G.x, G.n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  if (iters_host) *iters_host = G.total;
  return SHBIM_OK;
}

int shbim_gmres_solve(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev, double* x_dev,
                      int* iters_host, double* resid_host, void* stream) {
  int rc = shbim_gmres_begin(ctx, sys, rhs_dev, x0_dev, stream);
  if (rc) return rc;
  bool done = false;
  if (ctx->graphs_on && ctx->device_gmres) {
    // the first step on the host warms the operator's graph slot (workspaces, captured application);
    // the rest of the solve runs as device cycles
    rc = shbim_gmres_step(ctx, nullptr, stream);
    if (rc == SHBIM_CONVERGED) done = true;
    else if (rc != SHBIM_CONTINUE) return rc;
    if (!done && (rc = device_cycles(ctx, (cudaStream_t)stream, &done))) return rc;
  }
  while (!done) {
    rc = shbim_gmres_step(ctx, nullptr, stream);
    if (rc == SHBIM_CONVERGED) break;
    if (rc != SHBIM_CONTINUE) return rc;
  }
  if ((rc = shbim_gmres_finish(ctx, x_dev, iters_host, stream))) return rc;
  if (resid_host) {
    auto& G = ctx->gm;
    cudaStream_t s = (cudaStream_t)stream;
    if (G.bnorm == 0.0) {
      *resid_host = 0.0;
      return SHBIM_OK;
    }
    if ((rc = system_matvec(ctx, G.x, G.w, s))) return rc;
    k_sub<<<nb(G.n), 256, 0, s>>>(G.b, G.w, G.w, G.n);
    SHBIM_CHECK_LAUNCH(ctx, "k_sub");
    double* hacc = hacc_ptr(ctx);
    k_dots<<<1, 256, 0, s>>>(G.w, G.n, G.w, hacc);
    SHBIM_CHECK_LAUNCH(ctx, "k_dots");
    SHBIM_CUDA(ctx, cudaMemcpyAsync(G.h_host, hacc, sizeof(double), cudaMemcpyDeviceToHost, s));
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    *resid_host = std::sqrt(std::max(0.0, G.h_host[0])) / G.bnorm;
  }
  return SHBIM_OK;
}

int shbim_set_outer_precision(shbim_ctx* ctx, int precision) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (precision != SHBIM_PREC_FP64 && precision != SHBIM_PREC_DF64)
    return fail(ctx, SHBIM_ERR_ARG, "outer precision must be SHBIM_PREC_FP64 or SHBIM_PREC_DF64");
  ctx->outer_prec = precision;
  return SHBIM_OK;
}

int shbim_set_device_gmres(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->device_gmres = on != 0;
  return SHBIM_OK;
}

int shbim_set_oneshot_precision(shbim_ctx* ctx, int precision) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (precision != SHBIM_PREC_FP64 && precision != SHBIM_PREC_DF64 && precision != SHBIM_PREC_FP32_COMP)
    return fail(ctx, SHBIM_ERR_ARG, "one-shot precision must be SHBIM_PREC_FP64, SHBIM_PREC_DF64 or SHBIM_PREC_FP32_COMP");
  ctx->oneshot_prec = precision;
  return SHBIM_OK;
}

int shbim_set_diffusion(shbim_ctx* ctx, double c) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (!(c >= 0.0) || !std::isfinite(c)) return fail(ctx, SHBIM_ERR_ARG, "diffusion coefficient must be >= 0");
  if (c != ctx->diff_c) ctx->geom_version++;  // the factor is a parameter of captured graphs
  ctx->diff_c = c;
  return SHBIM_OK;
}

}  // extern "C"

namespace shbim {
namespace {
__global__ void k_add(double* __restrict__ x, const double* __restrict__ d, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) x[e] += d[e];
}
}  // namespace
}  // namespace shbim

extern "C" int shbim_gmres_solve_refined(shbim_ctx* ctx, int sys, const double* rhs_dev, const double* x0_dev,
                                         double* x_dev, double inner_tol, int max_outer, int* inner_iters_host,
                                         int* outer_iters_host, double* resid_host, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (sys != SHBIM_SYS_ELECTRIC && sys != SHBIM_SYS_STOKES) return fail(ctx, SHBIM_ERR_ARG, "bad system");
  if (!rhs_dev || !x_dev) return fail(ctx, SHBIM_ERR_ARG, "null pointer");
  if (!(inner_tol > 0.0 && inner_tol < 1.0) || max_outer < 1)
    return fail(ctx, SHBIM_ERR_ARG, "need 0 < inner_tol < 1 and max_outer >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = system_size(ctx, sys);
  auto& G = ctx->gm;
  // outer buffers (sized for the larger system)
  if (!G.xr) {
    const int64_t cap = 3 * ctx->ncoef;
    if (cudaMalloc(&G.xr, cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.rr, cap * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&G.dr, cap * sizeof(double)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "refinement buffers");
  }
  const int saved_prec = ctx->opts.precision;
  const double saved_tol = ctx->opts.gmres_tol;
  const double tol = saved_tol;
  int inner_total = 0, outer = 0, rc = SHBIM_OK;
  double rel = 1.0;
  bool attempted_direct = false;
  if (x0_dev) {
    SHBIM_CUDA(ctx, cudaMemcpyAsync(G.xr, x0_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    SHBIM_CUDA(ctx, cudaMemsetAsync(G.xr, 0, n * sizeof(double), s));
  }
  // ||b||, through the GMRES set-up of the system (FP64 residual)
  double bnorm = 0.0;
  for (;;) {
    // FP64-class residual r = b - A x (FP64 or double-float sums)
    ctx->opts.precision = ctx->outer_prec;
    rc = shbim_gmres_begin(ctx, sys, rhs_dev, nullptr, stream);  // sets diag/offdiag, b, ||b||
    if (rc) break;
    bnorm = G.bnorm;
    if (bnorm == 0.0) {
      rel = 0.0;
      SHBIM_CUDA(ctx, cudaMemsetAsync(G.xr, 0, n * sizeof(double), s));
      break;
    }
    if (outer == 0 && !x0_dev) {
      // x = 0: the residual is b itself, no operator application needed
      SHBIM_CUDA(ctx, cudaMemcpyAsync(G.rr, rhs_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      // the first residual of an initial guess is formed in FP32: the first inner solve only has to
      // bring the residual down to the FP32 operator's accuracy, and the FP64-class residuals that
      // follow are the same as from a zero start (one for a system that finishes in one step, two
      // otherwise)
      if (outer == 0) ctx->opts.precision = SHBIM_PREC_FP32_COMP;
      G.raw = true;
      rc = system_matvec(ctx, G.xr, G.w, s);
      G.raw = false;
      ctx->opts.precision = ctx->outer_prec;
      if (rc) break;
      k_sub<<<nb(n), 256, 0, s>>>(rhs_dev, G.w, G.rr, n);
      SHBIM_CHECK_LAUNCH(ctx, "k_sub");
    }
    double* hacc = hacc_ptr(ctx);
    k_dots<<<1, 256, 0, s>>>(G.rr, n, G.rr, hacc);
    SHBIM_CHECK_LAUNCH(ctx, "k_dots");
    SHBIM_CUDA(ctx, cudaMemcpyAsync(G.h_host, hacc, sizeof(double), cudaMemcpyDeviceToHost, s));
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    rel = std::sqrt(std::max(0.0, G.h_host[0])) / bnorm;
    if (!std::isfinite(rel)) {
      rc = fail(ctx, SHBIM_ERR_NONFINITE, "non-finite residual in refinement");
      break;
    }
    if (outer == 1 && attempted_direct && rel > tol) ctx->refine_direct[sys] = false;
    // an FP32 first residual (see above) cannot end the solve: only an FP64-class one can
    if (rel <= tol && !(outer == 0 && x0_dev)) break;
    if (outer >= max_outer) {
      rc = fail(ctx, SHBIM_ERR_NOT_CONVERGED, "refinement reached max_outer");
      break;
    }
    // inner solve A d = r with FP32 sums. The tolerance that would finish in this step is
    // 0.5 tol / rel: when it is looser than inner_tol (typically the last step) it is used as is;
    // otherwise the step reduces the residual by inner_tol. The first inner solve (from a zero start
    // or from an initial guess) aims straight at the end (one FP64-class residual instead of two) while
    // this system's FP32 operator has been accurate enough for that; the first time the FP64-class
    // check after such a step misses the tolerance, later solves of the system go back to the
    // two-step form.
    const double need = 0.5 * tol / rel;
    const bool direct = outer == 0 && ctx->refine_direct[sys];
    const double tau = direct ? std::min(need, 0.5) : (need >= inner_tol ? std::min(need, 0.5) : inner_tol);
    attempted_direct = direct;
    ctx->opts.precision = SHBIM_PREC_FP32_COMP;
    ctx->opts.gmres_tol = tau;
    int it = 0;
    rc = shbim_gmres_solve(ctx, sys, G.rr, nullptr, G.dr, &it, nullptr, stream);
    ctx->opts.gmres_tol = saved_tol;
    if (rc) break;
    inner_total += it;
    k_add<<<nb(n), 256, 0, s>>>(G.xr, G.dr, n);
    SHBIM_CHECK_LAUNCH(ctx, "k_add");
    ++outer;
  }
  ctx->opts.precision = saved_prec;
  ctx->opts.gmres_tol = saved_tol;
  if (rc) return rc;
  SHBIM_CUDA(ctx, cudaMemcpyAsync(x_dev, G.xr, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (inner_iters_host) *inner_iters_host = inner_total;
  if (outer_iters_host) *outer_iters_host = outer;
  if (resid_host) *resid_host = rel;
  return SHBIM_OK;
}
