// Geometry and the singular self-integration (Section 2.1), FP64.
//
// Geometry: x, x_theta, x_phi/sin(theta) on a grid by synthesis with derivative tables;
// n = (x_theta x x_phi/sin) / J with J = |x_theta x x_phi/sin| the area element relative to
// the unit sphere (W / sin theta in the notation of Eq. reg_quadrature).
//
// Singular rows. For a target on drop i at parameter direction (theta_a, phi_b) let
// R = Rz(phi_b) Ry(theta_a), which takes the north pole to the target. The rotated-pole rule
// (Eq. mod_weights, degree-q grid y_jk) integrates K(x0, x(R y)) rho(R y) J(R y) with the
// modified weights mu_j. Because the rule is linear in the density, it equals
// row . rho_coef with
//     row_nm = sum_jk mu_j J K S_nm(R y_jk) / (4 pi),
// and the rows are built once per geometry:
//   1. rotate the position coefficients: b = D_R^T a, so that x(R y) = sum b_nm S_nm(y)
//      (real-basis rotation matrices D, S(R y) = D_R S(y), D_R = Dz(phi_b) Dq^T Dz(theta_a) Dq
//      with Dq the fixed matrix of Rx(pi/2), since Ry(t) = Rx(pi/2)^-1 Rz(t) Rx(pi/2));
//   2. synthesise x, x_theta, x_phi/sin of the rotated expansion on the degree-q grid and form
//      the weights w = mu_j J K / (4 pi) for every kernel component;
//   3. analyse: v_nm = sum_jk w S_nm(y_jk)  (plain sum, no regular weights);
//   4. rotate back: row = D_R v.
// The matvec then applies the rows as a dense FP64 GEMV (HBM-bound).
#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "internal.h"
#include "fourier.cuh"

namespace shbim {

// tmp[c * nkind * n + slot * n + i]: slots 0, 1, 2 = x, x_theta, x_phi / sin
__global__ void k_geometry(const double* __restrict__ tmp, int n, int nkind, int N,
                           const double* __restrict__ omega, int weighted, double* __restrict__ out,
                           int64_t ld, int64_t off, float* __restrict__ out32, double cx, double cy,
                           double cz, float* __restrict__ out32lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double X[3], Xt[3], Xp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X[c] = tmp[(int64_t)(c * nkind + 0) * n + i];
    Xt[c] = tmp[(int64_t)(c * nkind + 1) * n + i];
    Xp[c] = tmp[(int64_t)(c * nkind + 2) * n + i];
  }
  const double c0 = Xt[1] * Xp[2] - Xt[2] * Xp[1];
  const double c1 = Xt[2] * Xp[0] - Xt[0] * Xp[2];
  const double c2 = Xt[0] * Xp[1] - Xt[1] * Xp[0];
  const double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
  const double inv = 1.0 / J;
  const double w = weighted ? omega[i / N] * J : J;
  const double v[7] = {X[0], X[1], X[2], c0 * inv, c1 * inv, c2 * inv, w};
#pragma unroll
  for (int k = 0; k < 7; ++k) out[k * ld + off + i] = v[k];
  if (out32) {
    const double r[7] = {X[0] - cx, X[1] - cy, X[2] - cz, v[3], v[4], v[5], w};
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const float h = (float)r[k];
      out32[k * ld + off + i] = h;
      if (out32lo) out32lo[k * ld + off + i] = (float)(r[k] - (double)h);
    }
  }
}

int geometry_kernel(shbim_ctx* ctx, const double* buf, int64_t n, int nkind, const GridTables& g, double* out,
                    int64_t ld, int64_t off, cudaStream_t s) {
  k_geometry<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(buf, (int)n, nkind, 2 * g.q + 2, g.omega, 1, out, ld, off,
                                                         nullptr, 0.0, 0.0, 0.0, nullptr);
  SHBIM_CHECK_LAUNCH(ctx, "k_geometry");
  return SHBIM_OK;
}

int geometry_kernel32(shbim_ctx* ctx, const double* buf, int64_t n, int nkind, const GridTables& g, double* out,
                      float* out32, int64_t ld, int64_t off, const double* centre, cudaStream_t s,
                      float* out32lo) {
  k_geometry<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(buf, (int)n, nkind, 2 * g.q + 2, g.omega, 1, out, ld, off,
                                                         out32, centre[0], centre[1], centre[2], out32lo);
  SHBIM_CHECK_LAUNCH(ctx, "k_geometry");
  return SHBIM_OK;
}

int build_geometry(shbim_ctx* ctx, const double* xcoef, cudaStream_t s) {
  // scratch for the 9 synthesised fields of the largest grid
  int64_t maxn = 0;
  for (auto& d : ctx->drops) maxn = std::max<int64_t>(maxn, d.nt);
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, (size_t)9 * maxn * sizeof(double)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc geometry scratch");
  int rc = SHBIM_OK;
  for (auto& d : ctx->drops) {
    const double* xc = xcoef + 3 * d.coef_off;
    for (int pass = 0; pass < 2 && rc == SHBIM_OK; ++pass) {
      const GridTables& g = pass == 0 ? d.tab->base : d.tab->up;
      const int n = npts(g.q);
      // targets: x, x_theta, x_phi/sin into scratch; sources: all derivative kinds kept in xup
      const int nkind = pass == 0 ? 3 : kNumTab;
      double* buf = pass == 0 ? tmp : ctx->xup + 3 * kNumTab * d.src_off;
      rc = sht_synth(ctx, g, 3, xc, d.nc, (1 << nkind) - 1, buf, (int64_t)nkind * n, n, nullptr, nullptr, s);
      if (rc) break;
      double* out = pass == 0 ? ctx->geo.tgt : ctx->geo.src;
      float* out32 = pass == 0 ? ctx->geo.tgt32 : ctx->geo.src32;
      const int64_t ld = pass == 0 ? ctx->ntarget : ctx->nsource;
      const int64_t off = pass == 0 ? d.tgt_off : d.src_off;
      k_geometry<<<(n + 127) / 128, 128, 0, s>>>(buf, n, nkind, 2 * g.q + 2, g.omega, pass == 1 ? 1 : 0,
                                                 out, ld, off, out32, d.centre[0], d.centre[1],
                                                 d.centre[2], pass == 0 ? nullptr : ctx->geo.src32lo);
      ctx->launches++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(ctx, e, "k_geometry");
    }
    if (rc) break;
  }
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  return rc;
}

// ---------------------------------------------------------------- rotations

__device__ __forceinline__ int isqrt_d(int o) {
  int n = (int)sqrt((double)o);
  while ((n + 1) * (n + 1) <= o) ++n;
  while (n * n > o) --n;
  return n;
}

// cos(m alpha), sin(m alpha) for m = 0..p into shared memory (one sincos per order)
__device__ void trig_table(double* cz, double* sz, int p, double alpha) {
  for (int m = threadIdx.x; m <= p; m += blockDim.x) sincos(m * alpha, &sz[m], &cz[m]);
}

// v <- Dz(alpha) v in the real basis: S(Rz(alpha) y) = Dz(alpha) S(y); sgn = -1 applies
// Dz(-alpha) from the same table.
__device__ void dz_apply(double* v, int p, const double* cz, const double* sz, double sgn) {
  const int nc = (p + 1) * (p + 1);
  for (int o = threadIdx.x; o < nc; o += blockDim.x) {
    const int n = isqrt_d(o);
    const int m = o - n * n - n;
    if (m <= 0) continue;
    const double ca = cz[m], sa = sgn * sz[m];
    const double a = v[o];
    const double b = v[o - 2 * m];
    v[o] = ca * a - sa * b;
    v[o - 2 * m] = sa * a + ca * b;
  }
}

// out <- Dq in   (transpose: Dq^T in)
__device__ void dq_apply(const double* __restrict__ in, double* __restrict__ out, int p,
                         const double* __restrict__ dq, const int* __restrict__ dq_off, bool transpose) {
  const int nc = (p + 1) * (p + 1);
  for (int o = threadIdx.x; o < nc; o += blockDim.x) {
    const int n = isqrt_d(o);
    const int m = o - n * n - n;
    const int w = 2 * n + 1;
    const double* B = dq + dq_off[n];
    const double* x = in + n * n;
    double acc = 0.0;
    if (!transpose) {
      const double* row = B + (m + n) * w;
      for (int c = 0; c < w; ++c) acc = fma(row[c], x[c], acc);
    } else {
      const double* col = B + (m + n);
      for (int c = 0; c < w; ++c) acc = fma(col[c * w], x[c], acc);
    }
    out[o] = acc;
  }
}

// b = D_R^T a for the position coefficients of one target (blockIdx.x) and component (blockIdx.y)
__global__ void k_rotate_fwd(const double* __restrict__ xc, int nc, int p, int t_begin,
                             const double* __restrict__ theta_base, const double* __restrict__ dq,
                             const int* __restrict__ dq_off, double* __restrict__ out) {
  extern __shared__ double sm[];
  double* b0 = sm;
  double* b1 = sm + nc;
  double* ct = b1 + nc;
  double* st = ct + (p + 1);
  double* cp = st + (p + 1);
  double* sp = cp + (p + 1);
  const int tl = t_begin + blockIdx.x;
  const int f = blockIdx.y;
  const int nlon = 2 * p + 2;
  const double th = theta_base[tl / nlon];
  const double ph = 3.14159265358979323846 * (tl % nlon) / (p + 1);
  trig_table(ct, st, p, th);
  trig_table(cp, sp, p, ph);
  for (int o = threadIdx.x; o < nc; o += blockDim.x) b0[o] = xc[(int64_t)f * nc + o];
  __syncthreads();
  dz_apply(b0, p, cp, sp, -1.0);
  __syncthreads();
  dq_apply(b0, b1, p, dq, dq_off, false);
  __syncthreads();
  dz_apply(b1, p, ct, st, -1.0);
  __syncthreads();
  dq_apply(b1, out + ((int64_t)blockIdx.x * 3 + f) * nc, p, dq, dq_off, true);
}

// row = D_R v for target blockIdx.x and component blockIdx.y
__global__ void k_rotate_adj(const double* __restrict__ vbuf, int nc, int p, int t_begin, int ncomp,
                             const double* __restrict__ theta_base, const double* __restrict__ dq,
                             const int* __restrict__ dq_off, float* __restrict__ rows_lap,
                             float* __restrict__ rows_sto, int nt_drop) {
  extern __shared__ double sm[];
  double* b0 = sm;
  double* b1 = sm + nc;
  double* ct = b1 + nc;
  double* st = ct + (p + 1);
  double* cp = st + (p + 1);
  double* sp = cp + (p + 1);
  const int tl = t_begin + blockIdx.x;
  const int c = blockIdx.y;
  const int nlon = 2 * p + 2;
  const double th = theta_base[tl / nlon];
  const double ph = 3.14159265358979323846 * (tl % nlon) / (p + 1);
  trig_table(ct, st, p, th);
  trig_table(cp, sp, p, ph);
  const double* v = vbuf + ((int64_t)blockIdx.x * ncomp + c) * nc;
  dq_apply(v, b1, p, dq, dq_off, false);
  __syncthreads();
  dz_apply(b1, p, ct, st, 1.0);
  __syncthreads();
  dq_apply(b1, b0, p, dq, dq_off, true);
  __syncthreads();
  dz_apply(b0, p, cp, sp, 1.0);
  __syncthreads();
  float* dst = c < kNumLap ? rows_lap + ((int64_t)tl * kNumLap + c) * nc
                           : rows_sto + ((int64_t)tl * kNumSto + (c - kNumLap)) * nc;
  const int64_t plane = (int64_t)nt_drop * (c < kNumLap ? kNumLap : kNumSto) * nc;
  for (int o = threadIdx.x; o < nc; o += blockDim.x) {
    const float h = (float)b0[o];
    dst[o] = h;
    dst[plane + o] = (float)(b0[o] - (double)h);
  }
}

// ---------------------------------------------------------------- rotated-grid weights

__device__ __forceinline__ int tri_off_s(int p, int m) { return m * (p + 1) - m * (m - 1) / 2; }

// For target blockIdx.x (chunk-local) and up-grid latitude blockIdx.y: synthesise the rotated
// position and its tangents, then write the 14 kernel weights of every node of the latitude.
__global__ void k_self_weights(const double* __restrict__ rot, int p, int q,
                               const double* __restrict__ alf, const double* __restrict__ trig,
                               const double* __restrict__ mu, const double* __restrict__ tgt,
                               int64_t ntarget, int64_t tgt0, double* __restrict__ wbuf) {
  extern __shared__ double sm[];
  const int t = blockIdx.x;
  const int j = blockIdx.y;
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  const int nc = P1 * P1;
  const int nt = P1 * (p + 2) / 2;
  double* A = sm;             // [3 f][3 kind][2][P1]
  double* tc = A + 18 * P1;
  double* ts = tc + N;
  double* V = ts + N;         // [9][N] rotated x, x_theta, x_phi/sin on this latitude
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tc[i] = trig[i];
    ts[i] = trig[N + i];
  }
  const double* T = alf + (int64_t)j * kNumTab * nt;
  const double* cf = rot + (int64_t)t * 3 * nc;
  for (int task = threadIdx.x; task < 18 * P1; task += blockDim.x) {
    const int fk = task / (2 * P1);      // f * 3 + kind
    const int r = task - fk * 2 * P1;
    const int m = r >> 1;
    const int cs = r & 1;
    const int f = fk / 3, kind = fk - f * 3;
    double acc = 0.0;
    if (!(cs == 1 && m == 0)) {
      const double* col = T + kind * nt + tri_off_s(p, m);
      const double* c = cf + f * nc;
      const int sg = cs ? -m : m;
      for (int n = m; n <= p; ++n) acc = fma(c[n * n + n + sg], col[n - m], acc);
    }
    A[(fk * 2 + cs) * P1 + m] = acc;
  }
  __syncthreads();
  // Fourier synthesis, four longitudes per task (N = 4(p+1) on the upsampled grid)
  const int Q4 = N >> 2;
  for (int task = threadIdx.x; task < 9 * (Q4 + 1); task += blockDim.x) {
    const int fk = task / (Q4 + 1);
    const int k = task - fk * (Q4 + 1);
    const double* Ac = A + (fk * 2) * P1;
    const double* As = Ac + P1;
    if (fk % 3 != 2)
      synth4(Ac, As, Ac[0], 1.0, p, k, N, tc, ts, V + fk * N);
    else
      synth4(As, Ac, 0.0, -1.0, p, k, N, tc, ts, V + fk * N);
  }
  __syncthreads();
  const int64_t tg = tgt0 + t;
  const double x0 = tgt[tg], y0 = tgt[ntarget + tg], z0 = tgt[2 * ntarget + tg];
  const double n0x = tgt[3 * ntarget + tg], n0y = tgt[4 * ntarget + tg], n0z = tgt[5 * ntarget + tg];
  const double w0 = mu[j] * 0.07957747154594766788;
  const int64_t Ns = (int64_t)(q + 1) * N;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    // V[f*3 + kind]: f = x,y,z ; kind = value, d/dtheta, (1/sin) d/dphi
    const double xt0 = V[1 * N + k], xt1 = V[4 * N + k], xt2 = V[7 * N + k];
    const double xp0 = V[2 * N + k], xp1 = V[5 * N + k], xp2 = V[8 * N + k];
    const double c0 = xt1 * xp2 - xt2 * xp1;
    const double c1 = xt2 * xp0 - xt0 * xp2;
    const double c2 = xt0 * xp1 - xt1 * xp0;
    const double J = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    const double nx = c0 / J, ny = c1 / J, nz = c2 / J;
    const double hx = x0 - V[k], hy = y0 - V[3 * N + k], hz = z0 - V[6 * N + k];
    const double r2 = hx * hx + hy * hy + hz * hz;
    const double ri = 1.0 / sqrt(r2);
    const double ri2 = ri * ri;
    const double ri3 = ri2 * ri;
    const double w = w0 * J;
    const double hn = hx * nx + hy * ny + hz * nz;
    const double d5 = -6.0 * w * hn * ri3 * ri2;
    const double s3 = w * ri3;
    const double wr = w * ri;
    double out[14];
    out[0] = w * (hx * n0x + hy * n0y + hz * n0z) * ri3;
    out[1] = wr;
    out[2] = wr + s3 * hx * hx;
    out[3] = s3 * hx * hy;
    out[4] = s3 * hx * hz;
    out[5] = wr + s3 * hy * hy;
    out[6] = s3 * hy * hz;
    out[7] = wr + s3 * hz * hz;
    out[8] = d5 * hx * hx;
    out[9] = d5 * hx * hy;
    out[10] = d5 * hx * hz;
    out[11] = d5 * hy * hy;
    out[12] = d5 * hy * hz;
    out[13] = d5 * hz * hz;
    const int64_t node = (int64_t)j * N + k;
#pragma unroll
    for (int c = 0; c < 14; ++c) wbuf[((int64_t)t * 14 + c) * Ns + node] = out[c];
  }
}

static int ensure(shbim_ctx* ctx, double** buf, size_t* cap, size_t need, const char* what) {
  if (need <= *cap) return SHBIM_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, need * sizeof(double)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, std::string("cudaMalloc ") + what);
  *cap = need;
  return SHBIM_OK;
}

int build_singular_rows(shbim_ctx* ctx, const double* xcoef, cudaStream_t s) {
  const int ncomp = kNumLap + kNumSto;
  for (auto& d : ctx->drops) {
    const GridTables& up = d.tab->up;
    const int64_t Ns = d.ns;
    const int nc = d.nc;
    // chunk of targets so that the weight buffer stays near 256 MB
    int CT = (int)std::max<int64_t>(1, std::min<int64_t>(d.nt, (256ll << 20) / (ncomp * Ns * 8)));
    int rc;
    if ((rc = ensure(ctx, &ctx->rot_coef, &ctx->rot_elems, (size_t)CT * 3 * nc, "rotation buffer")) ||
        (rc = ensure(ctx, &ctx->wbuf, &ctx->wbuf_elems, (size_t)CT * ncomp * Ns, "weight buffer")) ||
        (rc = ensure(ctx, &ctx->vbuf, &ctx->vbuf_elems, (size_t)CT * ncomp * nc, "row buffer")))
      return rc;
    const double* xc = xcoef + 3 * d.coef_off;
    const int rot_smem = (2 * nc + 4 * (d.p + 1)) * (int)sizeof(double);
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, rot_smem));
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, rot_smem));
    for (int t0 = 0; t0 < d.nt; t0 += CT) {
      const int ct = std::min(CT, d.nt - t0);
      k_rotate_fwd<<<dim3(ct, 3), 128, rot_smem, s>>>(
          xc, nc, d.p, t0, d.tab->base.theta, d.tab->dq, d.tab->dq_off_dev, ctx->rot_coef);
      SHBIM_CHECK_LAUNCH(ctx, "k_rotate_fwd");
      const size_t smem = (size_t)(18 * (d.p + 1) + 11 * (2 * d.q + 2)) * sizeof(double);
      {
        TimeScope ts(ctx, SHBIM_K_SELF_WEIGHTS, s);
        k_self_weights<<<dim3(ct, d.q + 1), 128, smem, s>>>(ctx->rot_coef, d.p, d.q, up.alf, up.trig,
                                                            up.mu, ctx->geo.tgt, ctx->ntarget,
                                                            d.tgt_off + t0, ctx->wbuf);
        SHBIM_CHECK_LAUNCH(ctx, "k_self_weights");
      }
      {
        TimeScope ts(ctx, SHBIM_K_SELF_ANALYSIS, s);
        rc = sht_analysis(ctx, up, ct * ncomp, ctx->wbuf, Ns, false, ctx->vbuf, nc, s);
        if (rc) return rc;
      }
      k_rotate_adj<<<dim3(ct, ncomp), 128, rot_smem, s>>>(
          ctx->vbuf, nc, d.p, t0, ncomp, d.tab->base.theta, d.tab->dq, d.tab->dq_off_dev,
          d.rows_lap, d.rows_sto, d.nt);
      SHBIM_CHECK_LAUNCH(ctx, "k_rotate_adj");
    }
  }
  return SHBIM_OK;
}

// ---------------------------------------------------------------- self GEMV

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Self GEMVs over the FP32 row planes. FP32 path (DF = false): hi plane and the FP32 copy of the
// density, FP32 accumulation. FP64-class path (DF = true): both planes and both density planes,
// double-float accumulation. One warp per target; HBM-bound in both forms (in FP64 arithmetic the
// GEMV would be bound by the FP64 pipe: 2 flops per 8 bytes is above this GPU's FP64 balance).
__global__ void k_split_density(const double* __restrict__ x, int64_t n, float* __restrict__ hi,
                                float* __restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float h = (float)x[e];
  hi[e] = h;
  lo[e] = (float)(x[e] - (double)h);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <bool DF>
__global__ void k_self_lap(const DropDev* __restrict__ drops, const int* __restrict__ tgt_drop,
                           int64_t ntarget, int which, const float* __restrict__ xh,
                           const float* __restrict__ xl, double* __restrict__ out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntarget) return;
  const DropDev D = drops[tgt_drop[t]];
  const int64_t tl = t - D.tgt_off;
  const int64_t plane = (int64_t)D.nt * kNumLap * D.nc;
  const float* rh = D.rows_lap + (tl * kNumLap + which) * D.nc;
  const float* x = xh + D.coef_off;
  double v;
  if (!DF) {
    float acc = 0.f;
    for (int e = lane; e < D.nc; e += 32) acc = fmaf(rh[e], x[e], acc);
    v = (double)warp_sum_f(acc);
  } else {
    const float* rl = rh + plane;
    const float* x2 = xl + D.coef_off;
    dfl::acc acc;
    for (int e = lane; e < D.nc; e += 32) acc.add_prod(dfl::df{rh[e], rl[e]}, dfl::df{x[e], x2[e]});
    v = warp_sum(dfl::to_double(acc.value()));
  }
  if (lane == 0) out[t] = v;
}

template <bool DF>
__global__ void k_self_sto(const DropDev* __restrict__ drops, const int* __restrict__ tgt_drop,
                           int64_t ntarget, const float* __restrict__ fh, const float* __restrict__ fl,
                           const float* __restrict__ uh, const float* __restrict__ ul, double* __restrict__ out) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ntarget) return;
  const DropDev D = drops[tgt_drop[t]];
  const int64_t tl = t - D.tgt_off;
  const int nc = D.nc;
  const int64_t plane = (int64_t)D.nt * kNumSto * nc;
  const float* rows = D.rows_sto + tl * kNumSto * nc;
  double res[3] = {0.0, 0.0, 0.0};
  for (int part = 0; part < 2; ++part) {
    const float* vh = part == 0 ? fh : uh;
    if (!vh || (part == 1 && D.lam == 1.0)) continue;
    const float* vl = part == 0 ? fl : ul;
    const float* r = rows + part * 6 * nc;
    const float* Xh = vh + 3 * D.coef_off;
    double s3[3];
    if (!DF) {
      float a0 = 0.f, a1 = 0.f, a2 = 0.f;
      for (int e = lane; e < nc; e += 32) {
        const float X = Xh[e], Y = Xh[nc + e], Z = Xh[2 * nc + e];
        const float xx = r[e], xy = r[nc + e], xz = r[2 * nc + e];
        const float yy = r[3 * nc + e], yz = r[4 * nc + e], zz = r[5 * nc + e];
        a0 = fmaf(xx, X, fmaf(xy, Y, fmaf(xz, Z, a0)));
        a1 = fmaf(xy, X, fmaf(yy, Y, fmaf(yz, Z, a1)));
        a2 = fmaf(xz, X, fmaf(yz, Y, fmaf(zz, Z, a2)));
      }
      s3[0] = warp_sum_f(a0);
      s3[1] = warp_sum_f(a1);
      s3[2] = warp_sum_f(a2);
    } else {
      const float* Xl = vl + 3 * D.coef_off;
      const float* q = r + plane;
      dfl::acc a0, a1, a2;
      for (int e = lane; e < nc; e += 32) {
        const dfl::df X{Xh[e], Xl[e]}, Y{Xh[nc + e], Xl[nc + e]}, Z{Xh[2 * nc + e], Xl[2 * nc + e]};
        const dfl::df xx{r[e], q[e]}, xy{r[nc + e], q[nc + e]}, xz{r[2 * nc + e], q[2 * nc + e]};
        const dfl::df yy{r[3 * nc + e], q[3 * nc + e]}, yz{r[4 * nc + e], q[4 * nc + e]};
        const dfl::df zz{r[5 * nc + e], q[5 * nc + e]};
        a0.add_prod(xx, X);
        a0.add_prod(xy, Y);
        a0.add_prod(xz, Z);
        a1.add_prod(xy, X);
        a1.add_prod(yy, Y);
        a1.add_prod(yz, Z);
        a2.add_prod(xz, X);
        a2.add_prod(yz, Y);
        a2.add_prod(zz, Z);
      }
      s3[0] = warp_sum(dfl::to_double(a0.value()));
      s3[1] = warp_sum(dfl::to_double(a1.value()));
      s3[2] = warp_sum(dfl::to_double(a2.value()));
    }
    const double w = part == 0 ? 1.0 : D.lam - 1.0;
    for (int c = 0; c < 3; ++c) res[c] += w * s3[c];
  }
  if (lane == 0) {
    double* o = out + 3 * D.tgt_off + tl;
    o[0] = res[0];
    o[D.nt] = res[1];
    o[2 * D.nt] = res[2];
  }
}

namespace {
// hi / lo planes of n doubles into slot 0 or 1 (3 ncoef floats each) of the context's split buffer
int split_density(shbim_ctx* ctx, const double* x, int64_t n, int slot, float** hi, float** lo, cudaStream_t s) {
  const size_t need = (size_t)12 * ctx->ncoef;   // [hi, lo][slot 0, slot 1][3 ncoef]
  if (ctx->dens_split_cap < need) {
    cudaFree(ctx->dens_split);
    ctx->dens_split = nullptr;
    ctx->dens_split_cap = 0;
    if (cudaMalloc(&ctx->dens_split, need * sizeof(float)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc density split");
    ctx->dens_split_cap = need;
    ctx->geom_version++;  // captured operator graphs referenced the old buffer
  }
  *hi = ctx->dens_split + (int64_t)slot * 3 * ctx->ncoef;
  *lo = *hi + 6 * ctx->ncoef;
  k_split_density<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, *hi, *lo);
  SHBIM_CHECK_LAUNCH(ctx, "k_split_density");
  return SHBIM_OK;
}
}  // namespace

int apply_self_laplace(shbim_ctx* ctx, int which, const double* dens, double* out, cudaStream_t s) {
  float *xh, *xl;
  int rc = split_density(ctx, dens, ctx->ncoef, 0, &xh, &xl, s);
  if (rc) return rc;
  const int64_t threads = ctx->ntarget * 32;
  const unsigned g = (unsigned)((threads + 255) / 256);
  if (ctx->opts.precision == SHBIM_PREC_FP32_COMP && ctx->self_prec == SHBIM_PREC_FP32_COMP)
    k_self_lap<false><<<g, 256, 0, s>>>(ctx->drops_dev, ctx->geo.tgt_drop, ctx->ntarget, which, xh, xl, out);
  else
    k_self_lap<true><<<g, 256, 0, s>>>(ctx->drops_dev, ctx->geo.tgt_drop, ctx->ntarget, which, xh, xl, out);
  SHBIM_CHECK_LAUNCH(ctx, "k_self_lap");
  return SHBIM_OK;
}

int apply_self_stokes(shbim_ctx* ctx, const double* f, const double* u, double* out, cudaStream_t s) {
  float *fh = nullptr, *fl = nullptr, *uh = nullptr, *ul = nullptr;
  int rc;
  const int64_t n3 = 3 * ctx->ncoef;
  if (f && (rc = split_density(ctx, f, n3, 0, &fh, &fl, s))) return rc;
  if (u && (rc = split_density(ctx, u, n3, 1, &uh, &ul, s))) return rc;
  const int64_t threads = ctx->ntarget * 32;
  const unsigned g = (unsigned)((threads + 255) / 256);
  if (ctx->opts.precision == SHBIM_PREC_FP32_COMP && ctx->self_prec == SHBIM_PREC_FP32_COMP)
    k_self_sto<false><<<g, 256, 0, s>>>(ctx->drops_dev, ctx->geo.tgt_drop, ctx->ntarget, fh, fl, uh, ul, out);
  else
    k_self_sto<true><<<g, 256, 0, s>>>(ctx->drops_dev, ctx->geo.tgt_drop, ctx->ntarget, fh, fl, uh, ul, out);
  SHBIM_CHECK_LAUNCH(ctx, "k_self_sto");
  return SHBIM_OK;
}

}  // namespace shbim
