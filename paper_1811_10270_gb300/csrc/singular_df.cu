// Singular self rows (rotated-pole rule, Eq. mod_weights and Section 2.1) built in double-float
// arithmetic on the FP32 pipe. Same algorithm as singular.cu, stage for stage:
//   1. rotate the position coefficients so that the target is the north pole
//      (b = D_R^T x with D_R = Dz(phi) Dq^T Dz(theta) Dq);
//   2. synthesise the rotated x, x_theta, x_phi / sin on the degree 2p+1 grid and form the 14
//      kernel weights mu J K / (4 pi) at every node (Laplace DL and SL, 6 Stokeslet and 6
//      stresslet components);
//   3. analyse the weights (Fourier stage on the tensor cores, dft_tc.cu, or folded four ways in
//      double-float; then the Legendre stage, here or, opt-in, on the tensor cores, leg_tc.cu);
//   4. rotate the coefficient rows back (row = D_R v) and store them as (hi, lo) FP32 planes.
// The rotations of steps 1 and 4 run on the tensor cores (rot_tc.cu) where the degree fits.
// Every sum and every pointwise operation here is double-float (hi + lo FP32 pairs; Dekker
// products, Knuth sums, Newton square roots), ~2^-44 relative per operation; the tensor-core stages
// split their operands into exact digit products (~2^-40 of the sum of magnitudes). The rows agree
// with the FP64 build to rounding level while the FP64 pipe (1/64 of the FP32 rate here) stays idle.
#include <algorithm>

#include "dfloat.cuh"
#include "fourier.cuh"
#include "internal.h"

namespace shbim {

namespace {

using dfl::df;

__device__ __forceinline__ df ld(const float2* p, int64_t i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void st(float2* p, int64_t i, df v) { p[i] = make_float2(v.hi, v.lo); }

__device__ __forceinline__ int tri_off_i(int p, int m) { return m * (p + 1) - m * (m - 1) / 2; }

__global__ void k_to_df(const double* __restrict__ x, int64_t n, float2* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) st(out, e, dfl::from_double(x[e]));
}

// Rotation of all components of TPB targets per CTA, degree by degree (degrees n_begin .. p; the lower
// ones may have gone to the tensor-core kernel): every stage of
// D_R = Dz(phi) Dq^T Dz(theta) Dq acts within a degree block, so the block Dq_n is staged in shared
// memory once and applied to the TPB x ncomp vectors of the CTA.
//   forward (ADJ = false): out = Dq^T Dz(-theta) Dq Dz(-phi) in   (position coefficients)
//   adjoint (ADJ = true):  out = Dz(phi) Dq^T Dz(theta) Dq in     (rows, FP32 planes)
template <bool ADJ>
__global__ void __launch_bounds__(256)
k_rotate_deg_df(const float2* __restrict__ vin, int64_t in_stride, int nc, int p, int n_begin, int t_begin, int t_count,
                int tpb, int ncomp, const float2* __restrict__ cs_theta, const float2* __restrict__ cs_phi,
                const float2* __restrict__ dq, const int* __restrict__ dq_off, const int4* __restrict__ dq_rows,
                const int4* __restrict__ dq_cols, float2* __restrict__ vout, float* __restrict__ rows_lap,
                float* __restrict__ rows_sto, int nt_drop) {
  extern __shared__ float2 smf[];
  const int wmax = 2 * p + 1;
  const int b0 = blockIdx.x * tpb;                      // first chunk-local target of the CTA
  const int nb = min(tpb, t_count - b0);                // targets of this CTA
  const int nv = nb * ncomp;                            // vectors
  float2* D = smf;                                      // [w][w] Dq_n
  float2* X = D + wmax * wmax;                          // [tpb * ncomp][w]
  float2* Y = X + tpb * ncomp * wmax;                   // [tpb * ncomp][w]
  const int nlon = 2 * p + 2;
  auto cs_of = [&](int v, bool theta) {
    const int tl = t_begin + b0 + v / ncomp;
    return theta ? cs_theta + (int64_t)(tl / nlon) * 2 * (p + 1) : cs_phi + (int64_t)(tl % nlon) * 2 * (p + 1);
  };
  // Dz on the degree-n block of every vector, in place: (v[m], v[-m]) rotated by m alpha
  auto dz = [&](float2* V, int n, bool theta, bool neg) {
    const int w = 2 * n + 1;
    for (int task = threadIdx.x; task < nv * n; task += blockDim.x) {
      const int v = task / n, m = task - v * n + 1;
      const float2* cs = cs_of(v, theta);
      const df ca = ld(cs, m);
      df sa = ld(cs, p + 1 + m);
      if (neg) sa = dfl::neg(sa);
      float2* x = V + v * w;
      const df a = ld(x, n + m), b = ld(x, n - m);
      st(x, n + m, dfl::sub(dfl::mul(ca, a), dfl::mul(sa, b)));
      st(x, n - m, dfl::add(dfl::mul(sa, a), dfl::mul(ca, b)));
    }
  };
  // out[v][m] = sum_k M[m][k] in[v][k] with M = Dq_n (trans = false) or Dq_n^T (trans = true)
  auto apply_dq = [&](const float2* in, float2* out, int n, bool trans) {
    const int w = 2 * n + 1;
    for (int task = threadIdx.x; task < nv * w; task += blockDim.x) {
      const int v = task / w, m = task - v * w;
      const float2* x = in + v * w;
      dfl::acc acc;
      // only the nonzero entries of row m (column m for the transpose)
      const int4 pr = (trans ? dq_cols : dq_rows)[n * n + m];
      if (!trans)
        for (int i = 0, k = pr.x; i < pr.y; ++i, k += pr.z) acc.add_prod(ld(D, m * w + k), ld(x, k));
      else
        for (int i = 0, k = pr.x; i < pr.y; ++i, k += pr.z) acc.add_prod(ld(D, k * w + m), ld(x, k));
      st(out, v * w + m, acc.value());
    }
  };
  for (int n = n_begin; n <= p; ++n) {
    const int w = 2 * n + 1;
    __syncthreads();
    for (int i = threadIdx.x; i < w * w; i += blockDim.x) D[i] = dq[dq_off[n] + i];
    for (int i = threadIdx.x; i < nv * w; i += blockDim.x) {
      const int v = i / w, k = i - v * w;
      const int b = v / ncomp, c = v - b * ncomp;
      X[i] = vin[(int64_t)(b0 + b) * in_stride + (int64_t)c * nc + n * n + k];
    }
    __syncthreads();
    if (!ADJ) {
      dz(X, n, false, true);
      __syncthreads();
    }
    apply_dq(X, Y, n, false);
    __syncthreads();
    dz(Y, n, true, !ADJ);
    __syncthreads();
    apply_dq(Y, X, n, true);
    __syncthreads();
    if (ADJ) {
      dz(X, n, false, false);
      __syncthreads();
    }
    for (int i = threadIdx.x; i < nv * w; i += blockDim.x) {
      const int v = i / w, k = i - v * w;
      const int b = v / ncomp, c = v - b * ncomp;
      const df x = ld(X, i);
      if (!ADJ) {
        vout[((int64_t)(b0 + b) * ncomp + c) * nc + n * n + k] = make_float2(x.hi, x.lo);
      } else {
        const int tl = t_begin + b0 + b;
        float* dst = c < kNumLap ? rows_lap + ((int64_t)tl * kNumLap + c) * nc
                                 : rows_sto + ((int64_t)tl * kNumSto + (c - kNumLap)) * nc;
        const int64_t plane = (int64_t)nt_drop * (c < kNumLap ? kNumLap : kNumSto) * nc;
        dst[n * n + k] = x.hi;
        dst[plane + n * n + k] = x.lo;
      }
    }
  }
}

// Four-longitude Fourier synthesis (the parity folding of synth4) in double-float.
__device__ void synth4_df(const float2* __restrict__ a, const float2* __restrict__ b, df a0, float beta, int p,
                          int k, int N, const float2* __restrict__ tc, const float2* __restrict__ ts,
                          float2* __restrict__ dst) {
  dfl::acc ce, co, se, so;
  int id = 0;
  int m = 1;
  for (; m + 1 <= p; m += 2) {
    id += k;
    if (id >= N) id -= N;
    co.add_prod(ld(a, m), ld(tc, id));
    so.add_prod(ld(b, m), ld(ts, id));
    id += k;
    if (id >= N) id -= N;
    ce.add_prod(ld(a, m + 1), ld(tc, id));
    se.add_prod(ld(b, m + 1), ld(ts, id));
  }
  if (m <= p) {
    id += k;
    if (id >= N) id -= N;
    co.add_prod(ld(a, m), ld(tc, id));
    so.add_prod(ld(b, m), ld(ts, id));
  }
  const df s2{1.41421353816986084f, 2.4203234971764687e-08f};  // sqrt(2) as hi + lo
  const df CE = ce.value(), CO = co.value();
  df SE = se.value(), SO = so.value();
  if (beta < 0) {
    SE = dfl::neg(SE);
    SO = dfl::neg(SO);
  } else if (beta == 0) {
    SE = df{0.f, 0.f};
    SO = df{0.f, 0.f};
  }
  const df c1 = dfl::add(CE, CO), s1 = dfl::add(SE, SO);
  const df c2 = dfl::sub(CE, CO), s2v = dfl::sub(SO, SE);
  const int h = N >> 1;
  st(dst, k, dfl::add(a0, dfl::mul(s2, dfl::add(c1, s1))));
  st(dst, (N - k) % N, dfl::add(a0, dfl::mul(s2, dfl::sub(c1, s1))));
  st(dst, h - k, dfl::add(a0, dfl::mul(s2, dfl::add(c2, s2v))));
  st(dst, h + k, dfl::add(a0, dfl::mul(s2, dfl::sub(c2, s2v))));
}

// For target blockIdx.x (chunk-local) and up-grid latitude blockIdx.y: synthesise the rotated
// position and tangents, then the 14 kernel weights of every node of the latitude.
__global__ void k_self_weights_df(const float2* __restrict__ rot, int p, int q, const float2* __restrict__ alf,
                                  const float2* __restrict__ trig, const double* __restrict__ mu,
                                  const double* __restrict__ tgt, int64_t ntarget, int64_t tgt0,
                                  float2* __restrict__ wbuf, int* __restrict__ rexp) {
  extern __shared__ float2 smf[];
  const int t = blockIdx.x;
  const int j = blockIdx.y;
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  const int nc = P1 * P1;
  const int nt = P1 * (p + 2) / 2;
  float2* A = smf;            // [3 f][3 kind][2][P1]
  float2* tc = A + 18 * P1;
  float2* ts = tc + N;
  float2* V = ts + N;         // [9][N]
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tc[i] = trig[i];
    ts[i] = trig[N + i];
  }
  const float2* T = alf + (int64_t)j * 3 * nt;
  const float2* cf = rot + (int64_t)t * 3 * nc;
  // order m-major, so that the 32 lanes of a warp hold sums of (nearly) equal length p + 1 - m
  for (int task = threadIdx.x; task < 18 * P1; task += blockDim.x) {
    const int m = task / 18;
    const int r = task - m * 18;
    const int fk = r >> 1;
    const int cs = r & 1;
    const int f = fk / 3, kind = fk - f * 3;
    dfl::acc acc;
    if (!(cs == 1 && m == 0)) {
      const float2* col = T + kind * nt + tri_off_i(p, m);
      const float2* c = cf + f * nc;
      const int sg = cs ? -m : m;
      for (int n = m; n <= p; ++n) acc.add_prod(ld(c, n * n + n + sg), ld(col, n - m));
    }
    st(A, (fk * 2 + cs) * P1 + m, acc.value());
  }
  __syncthreads();
  const int Q4 = N >> 2;
  // field fastest: the lanes of a warp read the same few trig entries (broadcasts) instead of
  // entries m k apart (bank conflicts)
  for (int task = threadIdx.x; task < 9 * (Q4 + 1); task += blockDim.x) {
    const int k = task / 9;
    const int fk = task - k * 9;
    const float2* Ac = A + (fk * 2) * P1;
    const float2* As = Ac + P1;
    // the phi-derivative kind swaps the cos / sin roles: selected per lane, one code path
    const bool dphi = fk % 3 == 2;
    synth4_df(dphi ? As : Ac, dphi ? Ac : As, dphi ? df{0.f, 0.f} : ld(Ac, 0), dphi ? -1.f : 1.f, p, k, N, tc, ts,
              V + fk * N);
  }
  __syncthreads();
  // the target's position and normal and mu_j / (4 pi) as double-float, converted once per block
  // (FP64 conversions run on the FP64 pipe)
  __shared__ float2 tv[7];
  if (threadIdx.x < 7) {
    const int64_t tg = tgt0 + t;
    const double v = threadIdx.x < 6 ? tgt[threadIdx.x * ntarget + tg] : mu[j] * 0.07957747154594766788;
    st(tv, threadIdx.x, dfl::from_double(v));
  }
  __syncthreads();
  const df x0 = ld(tv, 0), y0 = ld(tv, 1), z0 = ld(tv, 2);
  const df n0x = ld(tv, 3), n0y = ld(tv, 4), n0z = ld(tv, 5);
  const df w0 = ld(tv, 6);
  const int64_t Ns = (int64_t)(q + 1) * N;
  float mx[14];
#pragma unroll
  for (int c = 0; c < 14; ++c) mx[c] = 0.f;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const df xt0 = ld(V, 1 * N + k), xt1 = ld(V, 4 * N + k), xt2 = ld(V, 7 * N + k);
    const df xp0 = ld(V, 2 * N + k), xp1 = ld(V, 5 * N + k), xp2 = ld(V, 8 * N + k);
    const df c0 = dfl::sub(dfl::mul(xt1, xp2), dfl::mul(xt2, xp1));
    const df c1 = dfl::sub(dfl::mul(xt2, xp0), dfl::mul(xt0, xp2));
    const df c2 = dfl::sub(dfl::mul(xt0, xp1), dfl::mul(xt1, xp0));
    const df J2 = dfl::dot3(c0, c1, c2, c0, c1, c2);
    const df rJ = dfl::rsqrt(J2);
    const df J = dfl::mul(J2, rJ);
    const df nx = dfl::mul(c0, rJ), ny = dfl::mul(c1, rJ), nz = dfl::mul(c2, rJ);
    const df hx = dfl::diff(x0, ld(V, k)), hy = dfl::diff(y0, ld(V, 3 * N + k)), hz = dfl::diff(z0, ld(V, 6 * N + k));
    const df r2 = dfl::dot3(hx, hy, hz, hx, hy, hz);
    const df ri = dfl::rsqrt(r2);
    const df ri2 = dfl::sqr(ri);
    const df ri3 = dfl::mul(ri2, ri);
    const df w = dfl::mul(w0, J);
    const df hn = dfl::dot3(hx, hy, hz, nx, ny, nz);
    const df d5 = dfl::mul(dfl::mul(dfl::mul_f(w, -6.f), hn), dfl::mul(ri3, ri2));
    const df s3 = dfl::mul(w, ri3);
    const df wr = dfl::mul(w, ri);
    df out[14];
    out[0] = dfl::mul(dfl::mul(w, dfl::dot3(hx, hy, hz, n0x, n0y, n0z)), ri3);
    out[1] = wr;
    const df sx = dfl::mul(s3, hx), sy = dfl::mul(s3, hy), sz = dfl::mul(s3, hz);
    out[2] = dfl::add(wr, dfl::mul(sx, hx));
    out[3] = dfl::mul(sx, hy);
    out[4] = dfl::mul(sx, hz);
    out[5] = dfl::add(wr, dfl::mul(sy, hy));
    out[6] = dfl::mul(sy, hz);
    out[7] = dfl::add(wr, dfl::mul(sz, hz));
    const df dx = dfl::mul(d5, hx), dy = dfl::mul(d5, hy), dz = dfl::mul(d5, hz);
    out[8] = dfl::mul(dx, hx);
    out[9] = dfl::mul(dx, hy);
    out[10] = dfl::mul(dx, hz);
    out[11] = dfl::mul(dy, hy);
    out[12] = dfl::mul(dy, hz);
    out[13] = dfl::mul(dz, hz);
    const int64_t node = (int64_t)j * N + k;
#pragma unroll
    for (int c = 0; c < 14; ++c) {
      st(wbuf, ((int64_t)t * 14 + c) * Ns + node, out[c]);
      mx[c] = fmaxf(mx[c], fabsf(out[c].hi));
    }
  }
  // power-of-two scale of each (component, latitude) row for the tensor-core analysis: max |hi|
  // < 2^e over the row's N nodes
  if (rexp) {
    __shared__ float red[4][14];   // blockDim.x <= 128
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 14; ++c) {
      float v = mx[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red[wp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 14) {
      float v = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w][threadIdx.x]);
      int e = 0;
      frexpf(v, &e);
      rexp[((int64_t)t * 14 + threadIdx.x) * (q + 1) + j] = max(e, -120);
    }
  }
}

// Fourier stage of the analysis, N divisible by 4, `rows` (item, latitude) rows per block:
// F[row][cs][m] = sum_k v[k] (cos|sin)(m phi_k), folded k <-> N-k and k <-> N/2-k (unweighted).
__global__ void k_analysis_f4_df(const float2* __restrict__ vals, int64_t val_stride, int p, int q,
                                 const float2* __restrict__ trig, int64_t nrows, int rows, float2* __restrict__ F) {
  extern __shared__ float2 smf[];
  const int N = 2 * q + 2;
  const int P1 = p + 1;
  const int Q4 = N >> 2;
  const int h = N >> 1;
  float2* tc = smf;
  float2* ts = tc + N;
  float2* R = ts + N;  // per row: x[N] then the four folds [Q4 each]
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
    R[r * 2 * N + k] = vals[item * val_stride + j * N + k];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * Q4; e += blockDim.x) {
    const int r = e / Q4, k = e - r * Q4;
    if (k == 0) continue;
    const float2* x = R + r * 2 * N;
    float2* ee = R + r * 2 * N + N;
    const df xk = ld(x, k), xn = ld(x, N - k), xa = ld(x, h - k), xb = ld(x, h + k);
    const df ek = dfl::add(xk, xn), ok = dfl::sub(xk, xn);
    const df e2 = dfl::add(xa, xb), o2 = dfl::sub(xa, xb);
    st(ee, k, dfl::add(ek, e2));
    st(ee, Q4 + k, dfl::sub(ek, e2));
    st(ee, 2 * Q4 + k, dfl::add(ok, o2));
    st(ee, 3 * Q4 + k, dfl::sub(ok, o2));
  }
  __syncthreads();
  for (int task = threadIdx.x; task < nr * 2 * P1; task += blockDim.x) {
    const int r = task / (2 * P1);
    const int tt = task - r * 2 * P1;
    const int cs = tt / P1;
    const int m = tt - cs * P1;
    const float2* x = R + r * 2 * N;
    const float2* fold = x + N;
    const bool odd = m & 1;
    const int r4 = m & 3;
    dfl::acc acc;
    const float2* src;
    const float2* tb;
    if (cs == 0) {
      const df eq = dfl::add(ld(x, Q4), ld(x, 3 * Q4));
      const df xh = ld(x, h);
      acc.add(ld(x, 0));
      acc.add(odd ? dfl::neg(xh) : xh);
      if (r4 == 0) acc.add(eq);
      if (r4 == 2) acc.add(dfl::neg(eq));
      src = odd ? fold + Q4 : fold;
      tb = tc;
    } else {
      const df oq = dfl::sub(ld(x, Q4), ld(x, 3 * Q4));
      if (r4 == 1) acc.add(oq);
      if (r4 == 3) acc.add(dfl::neg(oq));
      src = odd ? fold + 2 * Q4 : fold + 3 * Q4;
      tb = ts;
    }
    int id = 0;
    for (int k = 1; k < Q4; ++k) {
      id += m;
      if (id >= N) id -= N;
      acc.add_prod(ld(src, k), ld(tb, id));
    }
    st(F, (r0 + r) * 2 * P1 + tt, acc.value());
  }
}

// Legendre stage: coef[item][n^2+n+-m] = s_m sum_j F[item][j][cs][m] Pbar_n^m(t_j), one CTA per
// item: the item's Fourier coefficients (q + 1 latitudes x 2 x (p + 1) double-float values) are
// copied once into shared memory, where every output reads them as broadcasts; the Legendre table
// comes through L1 (shared by all CTAs).
__global__ void __launch_bounds__(288)
k_analysis_leg_item_df(const float2* __restrict__ F, int p, int q, const float2* __restrict__ alf,
                       float2* __restrict__ coef, int64_t coef_stride) {
  extern __shared__ __align__(16) float2 sF[];
  const int item = blockIdx.x;
  const int nt = (p + 1) * (p + 2) / 2;
  const int P1 = p + 1;
  const int nF = (q + 1) * 2 * P1;   // float2, a multiple of 2 (16-byte pieces)
  const float2* Fi = F + (int64_t)item * nF;
  for (int e = threadIdx.x; e < nF / 2; e += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(sF + 2 * e)),
                 "l"(Fi + 2 * e));
  asm volatile("cp.async.commit_group;\n");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  float2* c = coef + (int64_t)item * coef_stride;
  for (int o = threadIdx.x; o < nt; o += blockDim.x) {
    int m = 0;
    while (m < p && tri_off_i(p, m + 1) <= o) ++m;
    const int n = m + (o - tri_off_i(p, m));
    dfl::acc ac, as;
#pragma unroll 4
    for (int j = 0; j <= q; ++j) {
      const df a = ld(alf, (int64_t)j * 3 * nt + o);
      ac.add_prod(ld(sF, j * 2 * P1 + m), a);
      as.add_prod(ld(sF, j * 2 * P1 + P1 + m), a);
    }
    if (m == 0) {
      st(c, n * n + n, ac.value());
    } else {
      const df s2{1.41421353816986084f, 2.4203234971764687e-08f};
      st(c, n * n + n + m, dfl::mul(s2, ac.value()));
      st(c, n * n + n - m, dfl::mul(s2, as.value()));
    }
  }
}

int ensure_d(shbim_ctx* ctx, double** buf, size_t* cap, size_t need, const char* what) {
  if (need <= *cap) return SHBIM_OK;
  cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  if (cudaMalloc(buf, need * sizeof(double)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, std::string("cudaMalloc ") + what);
  *cap = need;
  return SHBIM_OK;
}

}  // namespace

// Double-float build of every drop's singular rows (same buffers and chunking as the FP64 build;
// a float2 occupies the bytes of one double).
int build_singular_rows_df(shbim_ctx* ctx, cudaStream_t s, const double* xcoef) {
  const int ncomp = kNumLap + kNumSto;
  int rc;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // chunks of targets (weights of at most 1 GB) and the lane buffers sized for the largest drop
  auto chunk_of = [&](const Drop& d) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(d.nt, (1024ll << 20) / (ncomp * (int64_t)d.ns * 8)));
  };
  size_t need_rot = 0, need_w = 0, need_F = 0, need_v = 0, need_x = 0, need_e = 0;
  int chunks = 0;
  for (auto& d : ctx->drops) {
    if ((2 * d.q + 2) % 4) return fail(ctx, SHBIM_ERR_ARG, "double-float row build needs 4 | 2q+2");
    const size_t CT = (size_t)chunk_of(d);
    need_rot = std::max(need_rot, CT * 3 * d.nc);
    need_w = std::max(need_w, CT * ncomp * d.ns);
    need_F = std::max(need_F, CT * ncomp * (d.q + 1) * 2 * (d.p + 1));
    need_v = std::max(need_v, CT * ncomp * d.nc);
    need_x = std::max(need_x, (size_t)3 * d.nc);
    need_e = std::max(need_e, (CT * ncomp * (d.q + 1) + 1) / 2);
    chunks += (int)((d.nt + CT - 1) / CT);
  }
  // with two or more chunks, odd chunks run on the library's side stream, each lane with its own
  // buffers: the latency-bound tensor-core stages of one chunk overlap the FP32-pipe stages of the
  // other; the side lane starts after everything queued on s, and s waits for it at the end
  const bool two = ctx->concurrent && chunks > 1;
  cudaStream_t ls[2] = {s, s};
  if (two) {
    if ((rc = ensure_side_stream(ctx))) return rc;
    ls[1] = ctx->side;
  }
  for (int l = 0; l < (two ? 2 : 1); ++l) {
    auto& L = ctx->lanes[l];
    if ((rc = ensure_d(ctx, &L.rot, &L.rot_n, need_rot, "rotation buffer")) ||
        (rc = ensure_d(ctx, &L.w, &L.w_n, need_w, "weight buffer")) ||
        (rc = ensure_d(ctx, &L.F, &L.F_n, need_F, "Fourier buffer")) ||
        (rc = ensure_d(ctx, &L.v, &L.v_n, need_v, "row buffer")) ||
        (rc = ensure_d(ctx, &L.xdf, &L.xdf_n, need_x, "position copy")) ||
        (rc = ensure_d(ctx, &L.rexp, &L.rexp_n, need_e, "row exponents")))
      return rc;
    L.xdrop = -1;
  }
  if (two) {
    SHBIM_CUDA(ctx, cudaEventRecord(ctx->ev_fork, s));
    SHBIM_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
  }
  int c = 0;
  for (size_t di = 0; di < ctx->drops.size(); ++di) {
    const Drop& d = ctx->drops[di];
    const GridTables& up = d.tab->up;
    const int64_t Ns = d.ns;
    const int nc = d.nc;
    const int N = 2 * d.q + 2;
    const int CT = chunk_of(d);
    const int wmax = 2 * d.p + 1;
    // targets per CTA of the FP32-pipe rotations: as many as fit beside the Dq block in ~100 KB,
    // and no more than keeps at least two CTAs per SM busy for a chunk of CT targets
    const int per_t3 = 2 * 3 * wmax * (int)sizeof(float2), per_t14 = 2 * ncomp * wmax * (int)sizeof(float2);
    const int dq_bytes = wmax * wmax * (int)sizeof(float2);
    const int occ = std::max(1, CT / (2 * nsm));
    const int tpb3 = std::max(1, std::min({16, (100 * 1024 - dq_bytes) / per_t3, occ}));
    const int tpb14 = std::max(1, std::min({8, (100 * 1024 - dq_bytes) / per_t14, occ}));
    const int deg_smem3 = dq_bytes + tpb3 * per_t3;
    const int deg_smem14 = dq_bytes + tpb14 * per_t14;
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_deg_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, deg_smem3));
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_deg_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, deg_smem14));
    const size_t w_smem = (size_t)(18 * (d.p + 1) + 11 * N) * sizeof(float2);
    const int budget = 46 * 1024 / (int)sizeof(float2) - 2 * N;
    const int rows = std::max(1, std::min(8, budget / (2 * N)));
    const size_t f_smem = (size_t)(2 * N + rows * 2 * N) * sizeof(float2);
    // tensor-core rotations for degrees 0 .. rot_n (all of them up to p = 39), the FP32-pipe kernel above
    const int rot_n = ctx->tc_rot ? rot_tc_nmax(d.p) : -1;
    const bool rot_tc = rot_n >= 0;
    const int df_n0 = rot_n + 1;
    const int leg_smem = (d.q + 1) * 2 * (d.p + 1) * (int)sizeof(float2);
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_analysis_leg_item_df, cudaFuncAttributeMaxDynamicSharedMemorySize, leg_smem));
    const bool dft_tc = ctx->tc_rows && dft_tc_fits(d.p);
    const bool leg_tc = dft_tc && ctx->tc_leg && leg_tc_fits(d.p);   // reads the order-major Fourier output
    for (int t0 = 0; t0 < d.nt; t0 += CT, ++c) {
      const int ct = std::min(CT, d.nt - t0);
      const int lane = two ? (c & 1) : 0;
      cudaStream_t st = ls[lane];
      auto& L = ctx->lanes[lane];
      float2* rot = reinterpret_cast<float2*>(L.rot);
      float2* wb = reinterpret_cast<float2*>(L.w);
      float2* vb = reinterpret_cast<float2*>(L.v);
      float2* F = reinterpret_cast<float2*>(L.F);
      float2* xc = reinterpret_cast<float2*>(L.xdf);
      // row exponents of the weights for the tensor-core analysis, written by the weights kernel
      int* rexp = dft_tc ? reinterpret_cast<int*>(L.rexp) : nullptr;
      if (L.xdrop != (int)di) {
        k_to_df<<<(unsigned)((3 * nc + 255) / 256), 256, 0, st>>>(xcoef + 3 * d.coef_off, 3 * nc, xc);
        SHBIM_CHECK_LAUNCH(ctx, "k_to_df");
        L.xdrop = (int)di;
      }
      // the position coefficients are the same for every target: zero input stride
      {
        TimeScope tr(ctx, SHBIM_K_SELF_ROTATION, st);
        if (rot_tc) {
          if ((rc = rotate_tc(ctx, *d.tab, false, xc, 0, nc, t0, ct, 3, rot, nullptr, nullptr, d.nt, st))) return rc;
        }
        if (df_n0 <= d.p) {
          k_rotate_deg_df<false><<<(ct + tpb3 - 1) / tpb3, 256, deg_smem3, st>>>(
              xc, 0, nc, d.p, df_n0, t0, ct, tpb3, 3, d.tab->cs_theta_df, d.tab->cs_phi_df, d.tab->dq_df,
              d.tab->dq_off_dev, d.tab->dq_rows, d.tab->dq_cols, rot, nullptr, nullptr, d.nt);
          SHBIM_CHECK_LAUNCH(ctx, "k_rotate_deg_df");
        }
      }
      {
        TimeScope ts(ctx, SHBIM_K_SELF_WEIGHTS, st);
        k_self_weights_df<<<dim3(ct, d.q + 1), 128, w_smem, st>>>(rot, d.p, d.q, d.tab->up_alf_df, d.tab->up_trig_df,
                                                                  up.mu, ctx->geo.tgt, ctx->ntarget, d.tgt_off + t0, wb,
                                                                  rexp);
        SHBIM_CHECK_LAUNCH(ctx, "k_self_weights_df");
      }
      {
        TimeScope ts(ctx, SHBIM_K_SELF_ANALYSIS, st);
        const int64_t nrows = (int64_t)ct * ncomp * (d.q + 1);
        if (leg_tc) {
          if ((rc = analysis_fourier_tc(ctx, *d.tab, wb, nrows, rexp, F, st, true)) ||
              (rc = analysis_legendre_tc(ctx, *d.tab, F, (int64_t)ct * ncomp, vb, nc, st)))
            return rc;
        } else if (dft_tc) {
          if ((rc = analysis_fourier_tc(ctx, *d.tab, wb, nrows, rexp, F, st))) return rc;
        } else {
          k_analysis_f4_df<<<(unsigned)((nrows + rows - 1) / rows), 128, f_smem, st>>>(wb, Ns, d.p, d.q,
                                                                                     d.tab->up_trig_df, nrows, rows, F);
          SHBIM_CHECK_LAUNCH(ctx, "k_analysis_f4_df");
        }
        if (!leg_tc) {
          k_analysis_leg_item_df<<<ct * ncomp, 288, leg_smem, st>>>(F, d.p, d.q, d.tab->up_alf_df, vb, nc);
          SHBIM_CHECK_LAUNCH(ctx, "k_analysis_leg_item_df");
        }
      }
      {
        TimeScope tr(ctx, SHBIM_K_SELF_ROTATION, st);
        if (rot_tc) {
          if ((rc = rotate_tc(ctx, *d.tab, true, vb, (int64_t)ncomp * nc, nc, t0, ct, ncomp, nullptr, d.rows_lap,
                              d.rows_sto, d.nt, st)))
            return rc;
        }
        if (df_n0 <= d.p) {
          k_rotate_deg_df<true><<<(ct + tpb14 - 1) / tpb14, 256, deg_smem14, st>>>(
              vb, (int64_t)ncomp * nc, nc, d.p, df_n0, t0, ct, tpb14, ncomp, d.tab->cs_theta_df, d.tab->cs_phi_df,
              d.tab->dq_df, d.tab->dq_off_dev, d.tab->dq_rows, d.tab->dq_cols, nullptr, d.rows_lap, d.rows_sto, d.nt);
          SHBIM_CHECK_LAUNCH(ctx, "k_rotate_deg_df");
        }
      }
    }
  }
  if (two) {
    SHBIM_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
    SHBIM_CUDA(ctx, cudaStreamWaitEvent(s, ctx->ev_join, 0));
  }
  if ((ctx->tc_rows || ctx->tc_rot || ctx->tc_leg) && ctx->tc_err) {
    int flag = 0;
    SHBIM_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
    if (flag) {
      SHBIM_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s));
      return fail(ctx, SHBIM_ERR_TIMEOUT, "tensor-core row build: a bounded wait expired");
    }
  }
  return SHBIM_OK;
}

}  // namespace shbim
