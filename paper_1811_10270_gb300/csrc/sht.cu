// Spherical-harmonic transforms on Gaussian grids (Section 2, Eq. spharm_ex), FP64.
//
// Synthesis splits into a Legendre stage (per latitude j and order m: sum over degree n of
// coefficient x table) and a Fourier stage (per longitude: sum over m of cos / sin terms),
// both inside one CTA per (item, latitude). Analysis is the adjoint: a Fourier stage per
// (item, latitude) writing 2(p+1) partial sums to scratch, then a Legendre stage per
// (item, coefficient) summing over latitudes in a fixed order (deterministic).
#include <algorithm>

#include "internal.h"
#include "fourier.cuh"

namespace shbim {

__device__ __forceinline__ int tri_off_d(int p, int m) { return m * (p + 1) - m * (m - 1) / 2; }

// kinds bitmask -> table index of the slot-th set bit
__device__ __forceinline__ int kind_of_slot(int kinds, int slot) {
  int k = 0;
  for (int b = 0; b < kNumTab; ++b) {
    if (kinds & (1 << b)) {
      if (k == slot) return b;
      ++k;
    }
  }
  return 0;
}

// Items are (drop d, component c) with item = d kpd + c: coefficients at item * coef_stride,
// values at d drop_stride + c item_stride (+ kind slot * kind_stride), the per-node scale at
// d drop_stride, the factor alpha (times alpha_drop[d] when given).
__global__ void k_synth(const double* __restrict__ coef, int64_t coef_stride, int p, int q,
                        const double* __restrict__ alf, const double* __restrict__ trig, int kinds,
                        double* __restrict__ out, int64_t item_stride, int64_t kind_stride,
                        const double* __restrict__ scale, double alpha, float* __restrict__ out32,
                        float* __restrict__ out32lo, int kpd, int64_t drop_stride,
                        const double* __restrict__ alpha_drop, DropList L) {
  extern __shared__ double sm[];
  const int item = blockIdx.x;
  const int dl = item / kpd, ci = item - dl * kpd;
  const int64_t dbase = L.idx ? L.val_off[dl] : (int64_t)dl * drop_stride;
  const int64_t obase = dbase + (int64_t)ci * item_stride;
  if (scale) scale += dbase;
  if (alpha_drop) alpha *= alpha_drop[L.idx ? L.idx[dl] : dl];
  const int j = blockIdx.y;
  const int nk = __popc(kinds);
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  double* A = sm;                    // [nk][2][P1]
  double* tc = A + nk * 2 * P1;      // [N]
  double* ts = tc + N;               // [N]
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tc[i] = trig[i];
    ts[i] = trig[N + i];
  }
  const double* c = coef + (L.idx ? (int64_t)kpd * L.coef_off[dl] + (int64_t)ci * coef_stride
                                   : (int64_t)item * coef_stride);
  const int nt = (p + 1) * (p + 2) / 2;
  const double* T = alf + (int64_t)j * kNumTab * nt;
  const int ntask = nk * 2 * P1;
  for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
    const int slot = task / (2 * P1);
    const int r = task - slot * 2 * P1;
    const int m = r >> 1;
    const int cs = r & 1;
    double acc = 0.0;
    if (!(cs == 1 && m == 0)) {
      const double* col = T + kind_of_slot(kinds, slot) * nt + tri_off_d(p, m);
      const int sgn = cs ? -m : m;
      for (int n = m; n <= p; ++n) acc = fma(__ldg(c + n * n + n + sgn), col[n - m], acc);
    }
    A[(slot * 2 + cs) * P1 + m] = acc;
  }
  __syncthreads();
  const double s2 = 1.41421356237309504880;
  if ((N & 3) == 0) {
    double* V = ts + N;  // [nk][N]
    const int Q4 = N >> 2;
    for (int task = threadIdx.x; task < nk * (Q4 + 1); task += blockDim.x) {
      const int slot = task / (Q4 + 1);
      const int k = task - slot * (Q4 + 1);
      const int kind = kind_of_slot(kinds, slot);
      const double* Ac = A + (slot * 2) * P1;
      const double* As = Ac + P1;
      if (!((kPhiTypeMask >> kind) & 1))
        synth4(Ac, As, Ac[0], 1.0, p, k, N, tc, ts, V + slot * N);
      else
        synth4(As, Ac, 0.0, -1.0, p, k, N, tc, ts, V + slot * N);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
      const int64_t node = (int64_t)j * N + k;
      for (int slot = 0; slot < nk; ++slot) {
        const int kind = kind_of_slot(kinds, slot);
        double v = V[slot * N + k];
        if (kind == 0 && scale) v *= scale[node] * alpha;
        const int64_t o = obase + (int64_t)slot * kind_stride + node;
        out[o] = v;
        if (out32) {
          const float h = (float)v;
          out32[o] = h;
          if (out32lo) out32lo[o] = (float)(v - (double)h);
        }
      }
    }
    return;
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int64_t node = (int64_t)j * N + k;
    for (int slot = 0; slot < nk; ++slot) {
      const int kind = kind_of_slot(kinds, slot);
      const double* Ac = A + (slot * 2) * P1;
      const double* As = Ac + P1;
      double v = 0.0;
      int id = 0;
      if (!((kPhiTypeMask >> kind) & 1)) {
        for (int m = 1; m <= p; ++m) {
          id += k;
          if (id >= N) id -= N;
          v = fma(Ac[m], tc[id], v);
          v = fma(As[m], ts[id], v);
        }
        v = Ac[0] + s2 * v;
      } else {
        for (int m = 1; m <= p; ++m) {
          id += k;
          if (id >= N) id -= N;
          v = fma(-Ac[m], ts[id], v);
          v = fma(As[m], tc[id], v);
        }
        v = s2 * v;
      }
      if (kind == 0 && scale) v *= scale[node] * alpha;
      const int64_t o = obase + (int64_t)slot * kind_stride + node;
      out[o] = v;
      if (out32) {
        const float h = (float)v;
        out32[o] = h;
        if (out32lo) out32lo[o] = (float)(v - (double)h);
      }
    }
  }
}

// Dynamic shared memory above the 48 KB default needs the kernel's opt-in (up to 227 KB per CTA).
int synth_smem_ok(shbim_ctx* ctx, size_t smem) {
  if (smem <= 48 * 1024) return SHBIM_OK;
  if (smem > 227 * 1024) return fail(ctx, SHBIM_ERR_ARG, "synthesis grid too large for shared memory");
  SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  return SHBIM_OK;
}

int sht_synth(shbim_ctx* ctx, const GridTables& g, int n_items, const double* coef,
              int64_t coef_stride, int kinds, double* out, int64_t item_stride,
              int64_t kind_stride, const double* scale, float* out32, cudaStream_t s, int kpd,
              const DropList* L) {
  if (n_items <= 0) return SHBIM_OK;
  const int nk = __builtin_popcount(kinds);
  const size_t smem = (size_t)(nk * 2 * (g.p + 1) + (2 + nk) * (2 * g.q + 2)) * sizeof(double);
  if (int rc = synth_smem_ok(ctx, smem)) return rc;
  dim3 grid(n_items, g.q + 1);
  k_synth<<<grid, 128, smem, s>>>(coef, coef_stride, g.p, g.q, g.alf, g.trig, kinds, out,
                                  item_stride, kind_stride, scale, 1.0, out32, nullptr, L ? kpd : n_items, 0, nullptr,
                                  L ? *L : DropList{});
  SHBIM_CHECK_LAUNCH(ctx, "k_synth");
  return SHBIM_OK;
}

// FP32 synthesis of values only, scaled per node, for the FP32 copies the FP32 sums read:
// out32[item][node] = fl32(alpha scale[node]) * sum_nm c_nm S_nm(node), Legendre and four-fold Fourier
// sums in FP32 (relative error ~1e-7, as the FP32 path allows).
__global__ void k_synth32(const double* __restrict__ coef, int64_t coef_stride, int p, int q,
                          const float* __restrict__ alf32, const float* __restrict__ trig32, float* __restrict__ out32,
                          int64_t item_stride, const double* __restrict__ scale, double alpha, int kpd,
                          int64_t drop_stride, const double* __restrict__ alpha_drop, DropList L) {
  extern __shared__ float smf32[];
  const int item = blockIdx.x, j = blockIdx.y;
  const int dl = item / kpd, ci = item - dl * kpd;
  const int64_t dbase = L.idx ? L.val_off[dl] : (int64_t)dl * drop_stride;
  scale += dbase;
  if (alpha_drop) alpha *= alpha_drop[L.idx ? L.idx[dl] : dl];
  const int N = 2 * q + 2, P1 = p + 1, Q4 = N >> 2, h = N >> 1;
  float* A = smf32;          // [2][P1]
  float* tc = A + 2 * P1;    // [N]
  float* ts = tc + N;        // [N]
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tc[i] = trig32[i];
    ts[i] = trig32[N + i];
  }
  const double* c = coef + (L.idx ? (int64_t)kpd * L.coef_off[dl] + (int64_t)ci * coef_stride
                                   : (int64_t)item * coef_stride);
  const int nt = P1 * (p + 2) / 2;
  const float* T = alf32 + (int64_t)j * nt;
  for (int task = threadIdx.x; task < 2 * P1; task += blockDim.x) {
    const int m = task >> 1, cs = task & 1;
    float acc = 0.f;
    if (!(cs == 1 && m == 0)) {
      const float* col = T + tri_off_d(p, m);
      const int sgn = cs ? -m : m;
      for (int n = m; n <= p; ++n) acc = fmaf((float)__ldg(c + n * n + n + sgn), col[n - m], acc);
    }
    A[cs * P1 + m] = acc;
  }
  __syncthreads();
  const float* Ac = A;
  const float* As = A + P1;
  const float s2 = 1.41421356f;
  float* out = out32 + dbase + (int64_t)ci * item_stride + (int64_t)j * N;
  const double* sc = scale + (int64_t)j * N;
  for (int k = threadIdx.x; k <= Q4; k += blockDim.x) {
    float ce = 0.f, co = 0.f, se = 0.f, so = 0.f;
    int id = 0, m = 1;
    for (; m + 1 <= p; m += 2) {
      id += k;
      if (id >= N) id -= N;
      co = fmaf(Ac[m], tc[id], co);
      so = fmaf(As[m], ts[id], so);
      id += k;
      if (id >= N) id -= N;
      ce = fmaf(Ac[m + 1], tc[id], ce);
      se = fmaf(As[m + 1], ts[id], se);
    }
    if (m <= p) {
      id += k;
      if (id >= N) id -= N;
      co = fmaf(Ac[m], tc[id], co);
      so = fmaf(As[m], ts[id], so);
    }
    const float c1 = ce + co, s1 = se + so, c2 = ce - co, s2v = so - se;
    const int ks[4] = {k, (N - k) % N, h - k, h + k};
    const float vs[4] = {Ac[0] + s2 * (c1 + s1), Ac[0] + s2 * (c1 - s1), Ac[0] + s2 * (c2 + s2v),
                         Ac[0] + s2 * (c2 - s2v)};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      // k = 0 and k = N/4 produce some longitudes twice with equal values
      out[ks[u]] = vs[u] * (float)(alpha * sc[ks[u]]);
    }
  }
}

// Synthesis with a scalar factor on the scaled values (used for (lam_j - 1) strengths).
int sht_synth_scaled(shbim_ctx* ctx, const GridTables& g, int n_items, const double* coef,
                     int64_t coef_stride, double* out, int64_t item_stride, const double* scale,
                     double alpha, float* out32, cudaStream_t s, float* out32lo) {
  return sht_synth_drops(ctx, g, 1, n_items, coef, coef_stride, out, item_stride, 0, scale, alpha, nullptr, out32, s,
                         out32lo);
}

// The same for nb consecutive drops of one degree in one launch: kpd items per drop, component c
// of drop d at d drop_stride + c comp_stride in the value arrays, the scale at d drop_stride, the
// factor alpha alpha_drop[d] (alpha_drop may be null).
int sht_synth_drops(shbim_ctx* ctx, const GridTables& g, int nb, int kpd, const double* coef, int64_t coef_stride,
                    double* out, int64_t comp_stride, int64_t drop_stride, const double* scale, double alpha,
                    const double* alpha_drop, float* out32, cudaStream_t s, float* out32lo, const DropList* L) {
  const DropList list = L ? *L : DropList{};
  const int n_items = nb * kpd;
  const int64_t item_stride = comp_stride;
  if (n_items <= 0) return SHBIM_OK;
  if (ctx->opts.precision == SHBIM_PREC_FP32_COMP && out32 && !out32lo && g.alf32 && ((2 * g.q + 2) & 3) == 0) {
    // only the FP32 copies are read in this mode: FP32 arithmetic
    const size_t smem32 = (size_t)(2 * (g.p + 1) + 2 * (2 * g.q + 2)) * sizeof(float);
    k_synth32<<<dim3(n_items, g.q + 1), 128, smem32, s>>>(coef, coef_stride, g.p, g.q, g.alf32, g.trig32, out32,
                                                          item_stride, scale, alpha, kpd, drop_stride, alpha_drop,
                                                          list);
    SHBIM_CHECK_LAUNCH(ctx, "k_synth32");
    return SHBIM_OK;
  }
  const size_t smem = (size_t)(2 * (g.p + 1) + 3 * (2 * g.q + 2)) * sizeof(double);
  if (int rc = synth_smem_ok(ctx, smem)) return rc;
  dim3 grid(n_items, g.q + 1);
  k_synth<<<grid, 128, smem, s>>>(coef, coef_stride, g.p, g.q, g.alf, g.trig, 1, out, item_stride,
                                  0, scale, alpha, out32, out32 ? out32lo : nullptr, kpd, drop_stride, alpha_drop,
                                  list);
  SHBIM_CHECK_LAUNCH(ctx, "k_synth");
  return SHBIM_OK;
}

// Fourier stage of the analysis: F[item][j][cs][m] = (omega_j) sum_k v[j][k] (cos|sin)(m phi_k)
__global__ void k_analysis_fourier(const double* __restrict__ vals, int64_t val_stride, int p, int q,
                                   const double* __restrict__ trig, const double* __restrict__ omega,
                                   int weighted, double* __restrict__ F, int kpd, DropList L) {
  extern __shared__ double sm[];
  const int item = blockIdx.x;
  const int j = blockIdx.y;
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  double* row = sm;
  double* tc = row + N;
  double* ts = tc + N;
  const int64_t ib = L.idx ? L.val_off[item / kpd] + (int64_t)(item % kpd) * val_stride : (int64_t)item * val_stride;
  const double* v = vals + ib + (int64_t)j * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    row[i] = v[i];
    tc[i] = trig[i];
    ts[i] = trig[N + i];
  }
  __syncthreads();
  const double w = weighted ? omega[j] : 1.0;
  double* out = F + ((int64_t)item * (q + 1) + j) * 2 * P1;
  for (int task = threadIdx.x; task < 2 * P1; task += blockDim.x) {
    const int cs = task / P1;
    const int m = task - cs * P1;
    const double* tb = cs ? ts : tc;
    double acc = 0.0;
    int id = 0;
    for (int k = 0; k < N; ++k) {
      acc = fma(row[k], tb[id], acc);
      id += m;
      if (id >= N) id -= N;
    }
    out[task] = w * acc;
  }
}

// Fourier stage for N divisible by 4, `rows` (item, latitude) rows per block. Each row is
// folded twice -- k with N-k (even / odd part in phi) and k with N/2-k (parity of m) -- so every
// output sums N/4-1 terms instead of N: four times fewer FP64 FMAs than the plain sum.
__global__ void k_analysis_fourier4(const double* __restrict__ vals, int64_t val_stride, int p, int q,
                                    const double* __restrict__ trig, const double* __restrict__ omega,
                                    int weighted, int64_t nrows, int rows, double* __restrict__ F, int kpd,
                                    DropList L) {
  extern __shared__ double sm[];
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  const int Q4 = N >> 2;
  const int h = N >> 1;
  double* tc = sm;
  double* ts = tc + N;
  double* R = ts + N;  // per row: x[N] then ee, eo, oe, oo [Q4 each]
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int nr = (int)min((int64_t)rows, nrows - r0);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tc[i] = trig[i];
    ts[i] = trig[N + i];
  }
  for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
    const int r = e / N, k = e - r * N;
    const int64_t row = r0 + r;
    const int64_t item = row / (q + 1), j = row - item * (q + 1);
    const int64_t ib = L.idx ? L.val_off[item / kpd] + (item % kpd) * val_stride : item * val_stride;
    R[r * 2 * N + k] = vals[ib + j * N + k];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * Q4; e += blockDim.x) {
    const int r = e / Q4, k = e - r * Q4;
    if (k == 0) continue;
    const double* x = R + r * 2 * N;
    double* ee = R + r * 2 * N + N;
    const double ek = x[k] + x[N - k], ok = x[k] - x[N - k];
    const double e2 = x[h - k] + x[h + k], o2 = x[h - k] - x[h + k];
    ee[k] = ek + e2;
    ee[Q4 + k] = ek - e2;
    ee[2 * Q4 + k] = ok + o2;
    ee[3 * Q4 + k] = ok - o2;
  }
  __syncthreads();
  for (int task = threadIdx.x; task < nr * 2 * P1; task += blockDim.x) {
    const int r = task / (2 * P1);
    const int tt = task - r * 2 * P1;
    const int cs = tt / P1;
    const int m = tt - cs * P1;
    const double* x = R + r * 2 * N;
    const double* fold = x + N;
    const bool odd = m & 1;
    const int r4 = m & 3;
    double acc;
    const double* src;
    const double* tb;
    if (cs == 0) {
      const double eq = x[Q4] + x[3 * Q4];
      acc = x[0] + (odd ? -x[h] : x[h]) + (r4 == 0 ? eq : (r4 == 2 ? -eq : 0.0));
      src = odd ? fold + Q4 : fold;
      tb = tc;
    } else {
      const double oq = x[Q4] - x[3 * Q4];
      acc = (r4 == 1 ? oq : (r4 == 3 ? -oq : 0.0));
      src = odd ? fold + 2 * Q4 : fold + 3 * Q4;
      tb = ts;
    }
    int id = 0;
    for (int k = 1; k < Q4; ++k) {
      id += m;
      if (id >= N) id -= N;
      acc = fma(src[k], tb[id], acc);
    }
    const int64_t row = r0 + r;
    const int64_t j = row % (q + 1);
    F[row * 2 * P1 + tt] = (weighted ? omega[j] : 1.0) * acc;
  }
}

// Legendre stage: coef[item][n^2+n+-m] = s_m sum_j F[item][j][cs][m] Pbar_n^m(t_j)
__global__ void k_analysis_legendre(const double* __restrict__ F, int p, int q,
                                    const double* __restrict__ alf, double* __restrict__ coef,
                                    int64_t coef_stride, int kpd, DropList L) {
  const int item = blockIdx.x;
  const int nt = (p + 1) * (p + 2) / 2;
  const int o = blockIdx.y * blockDim.x + threadIdx.x;
  if (o >= nt) return;
  int m = 0;
  while (m < p && tri_off_d(p, m + 1) <= o) ++m;
  const int n = m + (o - tri_off_d(p, m));
  const int P1 = p + 1;
  const double* Fi = F + (int64_t)item * (q + 1) * 2 * P1;
  double ac = 0.0, as = 0.0;
  for (int j = 0; j <= q; ++j) {
    const double a = alf[(int64_t)j * kNumTab * nt + o];
    ac = fma(Fi[(int64_t)j * 2 * P1 + m], a, ac);
    as = fma(Fi[(int64_t)j * 2 * P1 + P1 + m], a, as);
  }
  double* c = coef + (L.idx ? (int64_t)kpd * L.coef_off[item / kpd] + (int64_t)(item % kpd) * coef_stride
                             : (int64_t)item * coef_stride);
  if (m == 0) {
    c[n * n + n] = ac;
  } else {
    const double s2 = 1.41421356237309504880;
    c[n * n + n + m] = s2 * ac;
    c[n * n + n - m] = s2 * as;
  }
}

int sht_analysis(shbim_ctx* ctx, const GridTables& g, int n_items, const double* vals,
                 int64_t val_stride, bool weighted, double* coef, int64_t coef_stride,
                 cudaStream_t s, int kpd, const DropList* L) {
  if (n_items <= 0) return SHBIM_OK;
  const DropList list = L ? *L : DropList{};
  const size_t need = (size_t)n_items * (g.q + 1) * 2 * (g.p + 1);
  if (need > ctx->sht_scratch_elems) {
    // growing scratch: wait for queued users of the old buffer before freeing it
    if (ctx->sht_scratch) {
      SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
      cudaFree(ctx->sht_scratch);
      ctx->sht_scratch = nullptr;
    }
    if (cudaMalloc(&ctx->sht_scratch, need * sizeof(double)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc transform scratch");
    ctx->sht_scratch_elems = need;
    ctx->geom_version++;  // captured operator graphs referenced the old scratch
  }
  const int N = 2 * g.q + 2;
  if ((N & 3) == 0) {
    const int budget = 46 * 1024 / (int)sizeof(double) - 2 * N;  // stay below the 48 KB default
    const int rows = std::max(1, std::min(8, budget / (2 * N)));
    const int64_t nrows = (int64_t)n_items * (g.q + 1);
    const size_t smem = (size_t)(2 * N + rows * 2 * N) * sizeof(double);
    k_analysis_fourier4<<<(unsigned)((nrows + rows - 1) / rows), 128, smem, s>>>(
        vals, val_stride, g.p, g.q, g.trig, g.omega, weighted ? 1 : 0, nrows, rows, ctx->sht_scratch, kpd, list);
    SHBIM_CHECK_LAUNCH(ctx, "k_analysis_fourier4");
  } else {
    dim3 g1(n_items, g.q + 1);
    k_analysis_fourier<<<g1, 64, 3 * N * sizeof(double), s>>>(vals, val_stride, g.p, g.q, g.trig,
                                                              g.omega, weighted ? 1 : 0,
                                                              ctx->sht_scratch, kpd, list);
    SHBIM_CHECK_LAUNCH(ctx, "k_analysis_fourier");
  }
  const int nt = ntri(g.p);
  dim3 g2(n_items, (nt + 127) / 128);
  k_analysis_legendre<<<g2, 128, 0, s>>>(ctx->sht_scratch, g.p, g.q, g.alf, coef, coef_stride, kpd, list);
  SHBIM_CHECK_LAUNCH(ctx, "k_analysis_legendre");
  return SHBIM_OK;
}

}  // namespace shbim
