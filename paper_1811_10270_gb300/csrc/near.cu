// Nearly-singular correction (Section 2.1): targets close to another drop's surface take that
// drop's contribution from the regular rule (Eq. reg_quadrature) on its grid upsampled four
// times per direction, degree q_n = 4(q+1) - 1.
//
// Per geometry: a target x0 of drop i is near drop j when its distance to the nearest source
// node of S_j is below 6 h_j, h_j = sqrt(area_j / N_s) (k_near_detect, bounding-sphere
// culling first); the upsampled geometry (x, n, w = omega J) of every drop that has near
// targets is built once.
// Per operator application: the density of each such drop is synthesised on its upsampled
// grid (times w), and one CTA per near pair adds
//     sum over upsampled nodes of K(x0, y) s(y)  -  sum over degree-q nodes of K(x0, y) s(y)
// to the all-pairs result, replacing the degree-q regular value by the upsampled one. The
// FP32 variant uses the same centre-relative coordinates, (hi, lo) target offsets and two-sum
// accumulation as the all-pairs kernel; the FP64 variant plain FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dfloat.cuh"
#include "internal.h"
#include "pair_df.cuh"

namespace shbim {

constexpr int kNearGroup = 128;   // near targets per CTA of the tiled FP32 kernel

namespace {

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per drop: area (sum of w over the source grid) and radius (max |x - c|, one square root of the
// largest squared distance); one block per drop
__global__ void k_drop_stats(const DropDev* __restrict__ drops, const double* __restrict__ src, int64_t nsource,
                             double* __restrict__ out /* [n][2] */) {
  const DropDev D = drops[blockIdx.x];
  double a = 0.0, r2 = 0.0;
  for (int64_t e = threadIdx.x; e < D.ns; e += blockDim.x) {
    const int64_t s = D.src_off + e;
    const double dx = src[s] - D.cx, dy = src[nsource + s] - D.cy, dz = src[2 * nsource + s] - D.cz;
    a += src[6 * nsource + s];
    r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
  }
  __shared__ double sa[256], sr[256];
  sa[threadIdx.x] = a;
  sr[threadIdx.x] = r2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sr[threadIdx.x] = fmax(sr[threadIdx.x], sr[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = sa[0];
    out[2 * blockIdx.x + 1] = sqrt(sr[0]);
  }
}

// Near test in FP32 on centre-relative coordinates (a target within rounding of the 6 h_j
// threshold may land on either side; there the two rules agree to ~1e-11 anyway). One warp per
// target: for each candidate drop the lanes test 32 consecutive source nodes at a time (coalesced
// loads) and stop together at the first chunk that holds a node below the threshold.
__global__ void k_near_detect(const double* __restrict__ tgt, int64_t ntarget, const int* __restrict__ tgt_drop,
                              const DropDev* __restrict__ drops, int n_drops, const float* __restrict__ src32,
                              int64_t nsource, const double* __restrict__ stats /* area, R, lim per drop */,
                              int* __restrict__ count, int64_t* __restrict__ pair_t, int* __restrict__ pair_j,
                              int cap) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // uniform over the warp
  const int lane = threadIdx.x & 31;
  if (t >= ntarget) return;
  const int i = tgt_drop[t];
  const double x = tgt[t], y = tgt[ntarget + t], z = tgt[2 * ntarget + t];
  for (int j = 0; j < n_drops; ++j) {
    if (j == i) continue;
    const DropDev D = drops[j];
    const double R = stats[3 * j + 1], lim = stats[3 * j + 2];
    const double dcx = x - D.cx, dcy = y - D.cy, dcz = z - D.cz;
    if (sqrt(dcx * dcx + dcy * dcy + dcz * dcz) > R + lim) continue;
    const float rx = (float)dcx, ry = (float)dcy, rz = (float)dcz;
    const float lim2 = (float)(lim * lim);
    bool near = false;
    for (int64_t e0 = 0; e0 < D.ns; e0 += 32) {
      const int64_t e = e0 + lane;
      bool hit = false;
      if (e < D.ns) {
        const int64_t s = D.src_off + e;
        const float dx = rx - src32[s], dy = ry - src32[nsource + s], dz = rz - src32[2 * nsource + s];
        hit = dx * dx + dy * dy + dz * dz < lim2;
      }
      if (__any_sync(0xffffffffu, hit)) {
        near = true;
        break;
      }
    }
    if (near && lane == 0) {
      const int k = atomicAdd(count, 1);
      if (k < cap) {
        pair_t[k] = t;
        pair_j[k] = j;
      }
    }
  }
}

// Smallest distance from a near target to drop j's surface, sampled on j's upsampled grid (node
// spacing h_j / 4, so the sampled value exceeds the true distance by at most ~0.2 h_j): one warp per
// near pair, FP32 centre-relative coordinates; the squared distance and its ratio to h_j^2 are folded
// into two global minima (non-negative floats order like their bit patterns).
__global__ void k_near_min_dist(const double* __restrict__ tgt, int64_t ntarget, const int64_t* __restrict__ pair_t,
                                const int* __restrict__ pair_j, int npairs, const DropDev* __restrict__ drops,
                                int n_drops, const float* __restrict__ fgeo32, int64_t nfine,
                                const int64_t* __restrict__ foff /* [2][n_drops]: offset, count */,
                                const double* __restrict__ stats /* area, R, lim per drop */,
                                unsigned* __restrict__ mins /* d^2, d^2 / h^2 */) {
  const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // uniform over the warp
  const int lane = threadIdx.x & 31;
  if (k >= npairs) return;
  const int64_t t = pair_t[k];
  const int j = pair_j[k];
  const DropDev D = drops[j];
  const float rx = (float)(tgt[t] - D.cx), ry = (float)(tgt[ntarget + t] - D.cy), rz = (float)(tgt[2 * ntarget + t] - D.cz);
  const int64_t o = foff[j], n = foff[n_drops + j];
  float best = 3.0e38f;
  for (int64_t e = lane; e < n; e += 32) {
    const float dx = rx - fgeo32[o + e], dy = ry - fgeo32[nfine + o + e], dz = rz - fgeo32[2 * nfine + o + e];
    best = fminf(best, fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
  }
#pragma unroll
  for (int sh = 16; sh > 0; sh >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, sh));
  if (lane == 0) {
    const double h2 = stats[3 * j] / D.ns;   // h_j^2 = area_j / N_s
    atomicMin(&mins[0], __float_as_uint(best));
    atomicMin(&mins[1], __float_as_uint((float)(best / h2)));
  }
}

__device__ __forceinline__ void two_sum_f(float& hi, float& lo, float a) {
  const float s = hi + a;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (a - bp);
  hi = s;
}

__device__ __forceinline__ double block_sum_near(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

// Sum over one grid of drop j of K(x0, y) s(y) for kernel KIND (0 DL target normal, 1 SL,
// 2 Stokes with f and u strengths) into acc[3]. FP32: positions relative to drop j's centre
// (pos32, [x y z nx ny nz][stride]), strengths str32 [comp][sstride]; FP64: absolute.
template <int KIND>
__device__ void near_sum32(const float* __restrict__ pos, int64_t stride, const float* __restrict__ str,
                           int64_t sstride, int64_t n, const float th[3], const float tl[3], const float nv[3],
                           int has_f, int has_u, double acc[3]) {
  float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const float dx = (th[0] - pos[e]) + tl[0];
    const float dy = (th[1] - pos[stride + e]) + tl[1];
    const float dz = (th[2] - pos[2 * stride + e]) + tl[2];
    const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    if (KIND == 1) {
      two_sum_f(hi[0], lo[0], str[e] * ri);
    } else if (KIND == 0) {
      const float dn = fmaf(dx, nv[0], fmaf(dy, nv[1], dz * nv[2]));
      two_sum_f(hi[0], lo[0], str[e] * ri * ri * ri * dn);
    } else {
      const float fx = has_f ? str[e] : 0.f, fy = has_f ? str[sstride + e] : 0.f, fz = has_f ? str[2 * sstride + e] : 0.f;
      const float ux = has_u ? str[3 * sstride + e] : 0.f, uy = has_u ? str[4 * sstride + e] : 0.f,
                  uz = has_u ? str[5 * sstride + e] : 0.f;
      const float nx = pos[3 * stride + e], ny = pos[4 * stride + e], nz = pos[5 * stride + e];
      const float ri2 = ri * ri, ri3 = ri2 * ri;
      const float hf = fmaf(dx, fx, fmaf(dy, fy, dz * fz));
      const float hu = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
      const float hn = fmaf(dx, nx, fmaf(dy, ny, dz * nz));
      const float t = ri3 * fmaf(hu * hn, ri2, hf);
      two_sum_f(hi[0], lo[0], fmaf(fx, ri, dx * t));
      two_sum_f(hi[1], lo[1], fmaf(fy, ri, dy * t));
      two_sum_f(hi[2], lo[2], fmaf(fz, ri, dz * t));
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = (double)hi[c] + (double)lo[c];
}

template <int KIND>
__device__ void near_sum64(const double* __restrict__ pos, int64_t stride, const double* __restrict__ str,
                           int64_t sstride, int64_t n, const double x0[3], const double nv[3], int has_f,
                           int has_u, double acc[3]) {
  double a[3] = {0.0, 0.0, 0.0};
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double dx = x0[0] - pos[e], dy = x0[1] - pos[stride + e], dz = x0[2] - pos[2 * stride + e];
    const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
    if (KIND == 1) {
      a[0] = fma(str[e], ri, a[0]);
    } else if (KIND == 0) {
      a[0] = fma(str[e] * ri * ri * ri, dx * nv[0] + dy * nv[1] + dz * nv[2], a[0]);
    } else {
      const double fx = has_f ? str[e] : 0.0, fy = has_f ? str[sstride + e] : 0.0, fz = has_f ? str[2 * sstride + e] : 0.0;
      const double ux = has_u ? str[3 * sstride + e] : 0.0, uy = has_u ? str[4 * sstride + e] : 0.0,
                   uz = has_u ? str[5 * sstride + e] : 0.0;
      const double ri2 = ri * ri, ri3 = ri2 * ri;
      const double hf = dx * fx + dy * fy + dz * fz;
      const double hu = dx * ux + dy * uy + dz * uz;
      const double hn = dx * pos[3 * stride + e] + dy * pos[4 * stride + e] + dz * pos[5 * stride + e];
      const double t = ri3 * (hf + hu * hn * ri2);
      a[0] += fx * ri + dx * t;
      a[1] += fy * ri + dy * t;
      a[2] += fz * ri + dz * t;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = a[c];
}

// Double-float version (FP64-class accuracy on the FP32 pipe): positions, normals and strengths
// are (FP32 copy, low part) pairs relative to drop j's centre; T is the target offset.
template <int KIND>
__device__ void near_sum_df(const float* __restrict__ pos, const float* __restrict__ poslo, int64_t stride,
                            const float* __restrict__ str, const float* __restrict__ strlo, int64_t sstride,
                            int64_t n, const dfl::df T[3], const dfl::df nv[3], int has_f, int has_u,
                            double acc[3]) {
  using dfl::df;
  dfl::acc A[3];
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const df dx = dfl::diff(T[0], df{pos[e], poslo[e]});
    const df dy = dfl::diff(T[1], df{pos[stride + e], poslo[stride + e]});
    const df dz = dfl::diff(T[2], df{pos[2 * stride + e], poslo[2 * stride + e]});
    const df ri = dfl::rsqrt(dfl::dot3(dx, dy, dz, dx, dy, dz));
    if (KIND == 1) {
      A[0].add_prod(df{str[e], strlo[e]}, ri);
    } else if (KIND == 0) {
      const df dn = dfl::dot3(dx, dy, dz, nv[0], nv[1], nv[2]);
      A[0].add_prod(dfl::mul(df{str[e], strlo[e]}, dfl::mul(dfl::sqr(ri), ri)), dn);
    } else {
      df f[3], u[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        f[c] = has_f ? df{str[c * sstride + e], strlo[c * sstride + e]} : df{0.f, 0.f};
        u[c] = has_u ? df{str[(3 + c) * sstride + e], strlo[(3 + c) * sstride + e]} : df{0.f, 0.f};
      }
      const df nx{pos[3 * stride + e], poslo[3 * stride + e]}, ny{pos[4 * stride + e], poslo[4 * stride + e]},
          nz{pos[5 * stride + e], poslo[5 * stride + e]};
      const df hf = dfl::dot3(dx, dy, dz, f[0], f[1], f[2]);
      const df hu = dfl::dot3(dx, dy, dz, u[0], u[1], u[2]);
      const df hn = dfl::dot3(dx, dy, dz, nx, ny, nz);
      const df ri2 = dfl::sqr(ri);
      const df tt = dfl::mul(dfl::mul(ri2, ri), dfl::add(hf, dfl::mul(dfl::mul(hu, hn), ri2)));
      const df d[3] = {dx, dy, dz};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A[c].add_prod(f[c], ri);
        A[c].add_prod(d[c], tt);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = dfl::to_double(A[c].value());
}

struct NearArgs {
  const int64_t* pair_t;
  const int* pair_j;
  const int64_t* fine_off;   // per drop: offset into the upsampled arrays (-1: none)
  const int64_t* fine_n;     // per drop: upsampled node count
  const DropDev* drops;
  const int* tgt_drop;
  const double* tgt;
  int64_t ntarget;
  const double* fpos;        // [7][nfine] FP64 absolute
  const float* fpos32;       // [7][nfine] FP32 relative to the drop centre
  const double* fstr;        // [6][nfine] strengths on the upsampled grids
  const float* fstr32;
  int64_t nfine;
  const double* src;         // degree-q sources
  const float* src32;
  const double* sstr;        // [6][nsource] degree-q strengths (dens_up)
  const float* sstr32;
  int64_t nsource;
  const float* fpos32lo;     // low parts for the double-float sums
  const float* fstr32lo;
  const float* src32lo;
  const float* sstr32lo;
  int has_f, has_u;
  double* out;
};

// MODE 0: FP64, 1: FP32 compensated, 2: double-float
template <int KIND, int MODE>
__global__ void __launch_bounds__(256) k_near_direct(NearArgs A) {
  constexpr bool F32 = MODE == 1;
  const int pr = blockIdx.x;
  const int64_t t = A.pair_t[pr];
  const int j = A.pair_j[pr];
  const DropDev D = A.drops[j];
  // chunk blockIdx.y of gridDim.y of both grids' nodes (partial sums meet in the atomics)
  const int64_t fn_all = A.fine_n[j];
  const int64_t f0 = fn_all * blockIdx.y / gridDim.y, f1 = fn_all * (blockIdx.y + 1) / gridDim.y;
  const int64_t s0 = (int64_t)D.ns * blockIdx.y / gridDim.y, s1 = (int64_t)D.ns * (blockIdx.y + 1) / gridDim.y;
  const int64_t fo = A.fine_off[j] + f0, fn = f1 - f0;
  const int64_t so = D.src_off + s0, sn = s1 - s0;
  double x0[3], nv[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    x0[c] = A.tgt[c * A.ntarget + t];
    nv[c] = A.tgt[(3 + c) * A.ntarget + t];
  }
  double af[3], au[3];
  if (F32) {
    const double cj[3] = {D.cx, D.cy, D.cz};
    float th[3], tl[3], n32[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = x0[c] - cj[c];
      th[c] = (float)d;
      tl[c] = (float)(d - (double)th[c]);
      n32[c] = (float)nv[c];
    }
    near_sum32<KIND>(A.fpos32 + fo, A.nfine, A.fstr32 + fo, A.nfine, fn, th, tl, n32, A.has_f, A.has_u, af);
    near_sum32<KIND>(A.src32 + so, A.nsource, A.sstr32 + so, A.nsource, sn, th, tl, n32,
                     A.has_f, A.has_u, au);
  } else if (MODE == 2) {
    // the target offset and normal as double-float, converted once per block (FP64 pipe)
    __shared__ float2 tv[6];
    if (threadIdx.x < 6) {
      const double cj[3] = {D.cx, D.cy, D.cz};
      const int c = threadIdx.x % 3;
      const dfl::df v = dfl::from_double(threadIdx.x < 3 ? x0[c] - cj[c] : nv[c]);
      tv[threadIdx.x] = make_float2(v.hi, v.lo);
    }
    __syncthreads();
    dfl::df T[3], nd[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T[c] = dfl::df{tv[c].x, tv[c].y};
      nd[c] = dfl::df{tv[3 + c].x, tv[3 + c].y};
    }
    near_sum_df<KIND>(A.fpos32 + fo, A.fpos32lo + fo, A.nfine, A.fstr32 + fo, A.fstr32lo + fo, A.nfine, fn, T, nd,
                      A.has_f, A.has_u, af);
    near_sum_df<KIND>(A.src32 + so, A.src32lo + so, A.nsource, A.sstr32 + so, A.sstr32lo + so, A.nsource, sn, T,
                      nd, A.has_f, A.has_u, au);
  } else {
    near_sum64<KIND>(A.fpos + fo, A.nfine, A.fstr + fo, A.nfine, fn, x0, nv, A.has_f, A.has_u, af);
    near_sum64<KIND>(A.src + so, A.nsource, A.sstr + so, A.nsource, sn, x0, nv, A.has_f,
                     A.has_u, au);
  }
  const int nc = KIND == 2 ? 3 : 1;
  for (int c = 0; c < nc; ++c) {
    const double v = block_sum_near(af[c] - au[c]);
    if (threadIdx.x == 0) {
      const double val = 0.07957747154594766788 * v;
      if (KIND != 2) {
        atomicAdd(A.out + t, val);
      } else {
        const DropDev Di = A.drops[A.tgt_drop[t]];
        atomicAdd(A.out + 3 * Di.tgt_off + (int64_t)c * Di.nt + (t - Di.tgt_off), val);
      }
    }
  }
}

// FP32 near correction, tiled: a CTA takes a group of near targets of one source drop j (one
// target per thread) and a chunk of the concatenated node list [drop j's upsampled nodes, then
// its degree-q nodes with the strengths negated]; nodes are staged through shared memory in
// tiles and read as broadcasts (as in the all-pairs kernels), sums compensated by two-sum, each
// chunk's result added to the target's output with an FP64 atomic.
template <int KIND>
__global__ void __launch_bounds__(kNearGroup)
k_near_tiled32(NearArgs A, const int4* __restrict__ groups) {
  constexpr int NC = KIND == 2 ? 3 : 1;
  constexpr int TILE = 256;
  __shared__ float4 sp[TILE];                  // x y z (relative to drop j's centre), strength 0
  __shared__ float4 sq[KIND == 2 ? TILE : 1];  // strengths 1..4
  __shared__ float4 sr[KIND == 2 ? TILE : 1];  // strength 5, normal
  const int4 g = groups[blockIdx.x];
  const int j = g.z;
  const DropDev D = A.drops[j];
  const int64_t fo = A.fine_off[j], fn = A.fine_n[j];
  const int64_t ntot = fn + D.ns;
  const int64_t c0 = ntot * blockIdx.y / gridDim.y, c1 = ntot * (blockIdx.y + 1) / gridDim.y;
  const bool act = (int)threadIdx.x < g.y;
  const int64_t t = A.pair_t[g.x + (act ? threadIdx.x : 0)];
  float th[3], tl[3], nv[3];
  {
    const double cj[3] = {D.cx, D.cy, D.cz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = A.tgt[c * A.ntarget + t] - cj[c];
      th[c] = (float)d;
      tl[c] = (float)(d - (double)th[c]);
      nv[c] = (float)A.tgt[(3 + c) * A.ntarget + t];
    }
  }
  float hi[NC], lo[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) hi[c] = lo[c] = 0.f;
  for (int64_t base = c0; base < c1; base += TILE) {
    const int cnt = (int)min((int64_t)TILE, c1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int64_t v = base + e;
      const bool fine = v < fn;
      const float* pos = fine ? A.fpos32 + fo + v : A.src32 + D.src_off + (v - fn);
      const float* str = fine ? A.fstr32 + fo + v : A.sstr32 + D.src_off + (v - fn);
      const int64_t ps = fine ? A.nfine : A.nsource;
      const float sg = fine ? 1.f : -1.f;
      if (KIND != 2) {
        sp[e] = make_float4(pos[0], pos[ps], pos[2 * ps], sg * str[0]);
      } else {
        const float f0 = A.has_f ? sg * str[0] : 0.f, f1 = A.has_f ? sg * str[ps] : 0.f, f2 = A.has_f ? sg * str[2 * ps] : 0.f;
        const float u0 = A.has_u ? sg * str[3 * ps] : 0.f, u1 = A.has_u ? sg * str[4 * ps] : 0.f,
                    u2 = A.has_u ? sg * str[5 * ps] : 0.f;
        sp[e] = make_float4(pos[0], pos[ps], pos[2 * ps], f0);
        sq[e] = make_float4(f1, f2, u0, u1);
        sr[e] = make_float4(u2, pos[3 * ps], pos[4 * ps], pos[5 * ps]);
      }
    }
    __syncthreads();
    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
#pragma unroll 4
    for (int e = 0; e < cnt; ++e) {
      const float4 P = sp[e];
      const float dx = (th[0] - P.x) + tl[0];
      const float dy = (th[1] - P.y) + tl[1];
      const float dz = (th[2] - P.z) + tl[2];
      const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
      if (KIND == 1) {
        acc[0] = fmaf(P.w, ri, acc[0]);
      } else if (KIND == 0) {
        const float dn = fmaf(dx, nv[0], fmaf(dy, nv[1], dz * nv[2]));
        acc[0] = fmaf(P.w * ri * ri * ri, dn, acc[0]);
      } else {
        const float4 Q = sq[e], R = sr[e];
        const float ri2 = ri * ri, ri3 = ri2 * ri;
        const float hf = fmaf(dx, P.w, fmaf(dy, Q.x, dz * Q.y));
        const float hu = fmaf(dx, Q.z, fmaf(dy, Q.w, dz * R.x));
        const float hn = fmaf(dx, R.y, fmaf(dy, R.z, dz * R.w));
        const float tt = ri3 * fmaf(hu * hn, ri2, hf);
        acc[0] = fmaf(P.w, ri, fmaf(dx, tt, acc[0]));
        acc[1] = fmaf(Q.x, ri, fmaf(dy, tt, acc[1]));
        acc[2] = fmaf(Q.y, ri, fmaf(dz, tt, acc[2]));
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) two_sum_f(hi[c], lo[c], acc[c]);
  }
  if (!act) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double val = 0.07957747154594766788 * ((double)hi[c] + (double)lo[c]);
    if (KIND != 2) {
      atomicAdd(A.out + t, val);
    } else {
      const DropDev Di = A.drops[A.tgt_drop[t]];
      atomicAdd(A.out + 3 * Di.tgt_off + (int64_t)c * Di.nt + (t - Di.tgt_off), val);
    }
  }
}

// Double-float near correction, tiled like k_near_tiled32 (FP64-class accuracy on the FP32 pipe);
// the per-source terms are those of the double-float all-pairs kernel.
template <int KIND>
__global__ void __launch_bounds__(kNearGroup)
k_near_tiled_df(NearArgs A, const int4* __restrict__ groups) {
  constexpr int NC = KIND == 2 ? 3 : 1;
  constexpr int NV = KIND == 2 ? 6 : 2;
  constexpr int TILE = 128;
  __shared__ float4 sh[NV][TILE];
  __shared__ float2 tv[kNearGroup][6];   // per target: offset from drop j's centre, normal
  const int4 g = groups[blockIdx.x];
  const int j = g.z;
  const DropDev D = A.drops[j];
  const int64_t fo = A.fine_off[j], fn = A.fine_n[j];
  const int64_t ntot = fn + D.ns;
  const int64_t c0 = ntot * blockIdx.y / gridDim.y, c1 = ntot * (blockIdx.y + 1) / gridDim.y;
  const bool act = (int)threadIdx.x < g.y;
  const int64_t t = A.pair_t[g.x + (act ? threadIdx.x : 0)];
  {
    const double cj[3] = {D.cx, D.cy, D.cz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const dfl::df a = dfl::from_double(A.tgt[c * A.ntarget + t] - cj[c]);
      const dfl::df n = dfl::from_double(A.tgt[(3 + c) * A.ntarget + t]);
      tv[threadIdx.x][c] = make_float2(a.hi, a.lo);
      tv[threadIdx.x][3 + c] = make_float2(n.hi, n.lo);
    }
  }
  dfl::df T[3], N0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T[c] = dfl::df{tv[threadIdx.x][c].x, tv[threadIdx.x][c].y};
    N0[c] = dfl::df{tv[threadIdx.x][3 + c].x, tv[threadIdx.x][3 + c].y};
  }
  dfl::acc acc[3];
  for (int64_t base = c0; base < c1; base += TILE) {
    const int cnt = (int)min((int64_t)TILE, c1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
      const int64_t v = base + e;
      const bool fine = v < fn;
      const int64_t o = fine ? fo + v : D.src_off + (v - fn);
      const float* ph = fine ? A.fpos32 : A.src32;
      const float* pl = fine ? A.fpos32lo : A.src32lo;
      const float* qh = fine ? A.fstr32 : A.sstr32;
      const float* ql = fine ? A.fstr32lo : A.sstr32lo;
      const int64_t ps = fine ? A.nfine : A.nsource;
      const float sg = fine ? 1.f : -1.f;
      sh[0][e] = make_float4(ph[o], ph[ps + o], ph[2 * ps + o], pl[o]);
      if constexpr (KIND != 2) {
        sh[1][e] = make_float4(pl[ps + o], pl[2 * ps + o], sg * qh[o], sg * ql[o]);
      } else {
        float fv[6], uv[6];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          fv[2 * c] = A.has_f ? sg * qh[c * ps + o] : 0.f;
          fv[2 * c + 1] = A.has_f ? sg * ql[c * ps + o] : 0.f;
          uv[2 * c] = A.has_u ? sg * qh[(3 + c) * ps + o] : 0.f;
          uv[2 * c + 1] = A.has_u ? sg * ql[(3 + c) * ps + o] : 0.f;
        }
        sh[1][e] = make_float4(pl[ps + o], pl[2 * ps + o], fv[0], fv[1]);
        sh[2][e] = make_float4(fv[2], fv[3], fv[4], fv[5]);
        sh[3][e] = make_float4(uv[0], uv[1], uv[2], uv[3]);
        sh[4][e] = make_float4(uv[4], uv[5], ph[3 * ps + o], pl[3 * ps + o]);
        sh[5][e] = make_float4(ph[4 * ps + o], pl[4 * ps + o], ph[5 * ps + o], pl[5 * ps + o]);
      }
    }
    __syncthreads();
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int e = 0; e < cnt; ++e) {
      if constexpr (KIND != 2)
        df_term<KIND>(T, N0, sh[0][e], sh[1][e], z4, z4, z4, z4, acc);
      else
        df_term<KIND>(T, N0, sh[0][e], sh[1][e], sh[2][e], sh[3][e], sh[4][e], sh[5][e], acc);
    }
  }
  if (!act) return;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const double val = 0.07957747154594766788 * dfl::to_double(acc[c].value());
    if (KIND != 2) {
      atomicAdd(A.out + t, val);
    } else {
      const DropDev Di = A.drops[A.tgt_drop[t]];
      atomicAdd(A.out + 3 * Di.tgt_off + (int64_t)c * Di.nt + (t - Di.tgt_off), val);
    }
  }
}

int grow(shbim_ctx* ctx, void** p, size_t* cap, size_t bytes, const char* what) {
  if (bytes <= *cap) return SHBIM_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, std::string("cudaMalloc ") + what);
  *cap = bytes;
  return SHBIM_OK;
}

}  // namespace

int build_near(shbim_ctx* ctx, const double* xcoef, cudaStream_t s) {
  auto& N = ctx->near;
  N.npairs = 0;
  N.min_dist = N.min_ratio = INFINITY;
  if (!N.enabled || ctx->n_drops < 2) return SHBIM_OK;
  const int nd = ctx->n_drops;
  int rc;
  // per-drop area, radius and near limit 6 h_j
  // [3 nd] stats the detection reads, then [2 nd] (area, radius) from the device
  if ((rc = grow(ctx, (void**)&N.stats, &N.stats_cap, sizeof(double) * 5 * nd, "near stats"))) return rc;
  double* tmp2 = N.stats + 3 * nd;
  k_drop_stats<<<nd, 256, 0, s>>>(ctx->drops_dev, ctx->geo.src, ctx->nsource, tmp2);
  SHBIM_CHECK_LAUNCH(ctx, "k_drop_stats");
  std::vector<double> st2(2 * nd), st3(3 * nd);
  SHBIM_CUDA(ctx, cudaMemcpyAsync(st2.data(), tmp2, sizeof(double) * 2 * nd, cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  for (int j = 0; j < nd; ++j) {
    st3[3 * j] = st2[2 * j];
    st3[3 * j + 1] = st2[2 * j + 1];
    st3[3 * j + 2] = kNearFactor * std::sqrt(st2[2 * j] / ctx->drops[j].ns);
  }
  SHBIM_CUDA(ctx, cudaMemcpyAsync(N.stats, st3.data(), sizeof(double) * 3 * nd, cudaMemcpyHostToDevice, s));
  // detection
  const int cap = (int)std::min<int64_t>(ctx->ntarget * 2 + 1024, 1 << 26);
  if ((rc = grow(ctx, (void**)&N.det_t, &N.det_t_cap, sizeof(int64_t) * cap, "near pairs")) ||
      (rc = grow(ctx, (void**)&N.det_j, &N.det_j_cap, sizeof(int) * (cap + 1), "near pairs")))
    return rc;
  int* count = N.det_j + cap;
  SHBIM_CUDA(ctx, cudaMemsetAsync(count, 0, sizeof(int), s));
  k_near_detect<<<nb(ctx->ntarget * 32), 256, 0, s>>>(ctx->geo.tgt, ctx->ntarget, ctx->geo.tgt_drop, ctx->drops_dev, nd,
                                                 ctx->geo.src32, ctx->nsource, N.stats, count, N.det_t, N.det_j, cap);
  SHBIM_CHECK_LAUNCH(ctx, "k_near_detect");
  int cnt = 0;
  SHBIM_CUDA(ctx, cudaMemcpyAsync(&cnt, count, sizeof(int), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  if (cnt > cap) return fail(ctx, SHBIM_ERR_NOMEM, "too many near pairs");
  if (cnt == 0) return SHBIM_OK;
  std::vector<int64_t> ht(cnt);
  std::vector<int> hj(cnt);
  SHBIM_CUDA(ctx, cudaMemcpy(ht.data(), N.det_t, sizeof(int64_t) * cnt, cudaMemcpyDeviceToHost));
  SHBIM_CUDA(ctx, cudaMemcpy(hj.data(), N.det_j, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
  // deterministic order: by source drop, then target
  std::vector<int> ord(cnt);
  for (int k = 0; k < cnt; ++k) ord[k] = k;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return hj[a] != hj[b] ? hj[a] < hj[b] : ht[a] < ht[b]; });
  std::vector<int64_t> pt(cnt);
  std::vector<int> pj(cnt);
  for (int k = 0; k < cnt; ++k) {
    pt[k] = ht[ord[k]];
    pj[k] = hj[ord[k]];
  }
  if ((rc = grow(ctx, (void**)&N.pair_t, &N.pair_t_cap, sizeof(int64_t) * cnt, "near pairs")) ||
      (rc = grow(ctx, (void**)&N.pair_j, &N.pair_j_cap, sizeof(int) * cnt, "near pairs")))
    return rc;
  SHBIM_CUDA(ctx, cudaMemcpy(N.pair_t, pt.data(), sizeof(int64_t) * cnt, cudaMemcpyHostToDevice));
  SHBIM_CUDA(ctx, cudaMemcpy(N.pair_j, pj.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice));
  N.npairs = cnt;
  {
    // runs of pairs with the same source drop, cut into groups of at most kNearGroup targets
    std::vector<int4> g;
    for (int k = 0; k < cnt;) {
      int e = k;
      while (e < cnt && pj[e] == pj[k] && e - k < kNearGroup) ++e;
      g.push_back(make_int4(k, e - k, pj[k], 0));
      k = e;
    }
    if ((rc = grow(ctx, (void**)&N.groups, &N.groups_cap, sizeof(int4) * g.size(), "near groups"))) return rc;
    SHBIM_CUDA(ctx, cudaMemcpy(N.groups, g.data(), sizeof(int4) * g.size(), cudaMemcpyHostToDevice));
    N.ngroups = (int)g.size();
  }
  // upsampled geometry of every drop that has near targets
  N.fine_off_h.assign(nd, -1);
  N.fine_n_h.assign(nd, 0);
  int64_t nfine = 0;
  for (int k = 0; k < cnt; ++k) {
    const int j = pj[k];
    if (N.fine_off_h[j] >= 0) continue;
    N.fine_off_h[j] = nfine;
    N.fine_n_h[j] = npts(ctx->drops[j].tab->fine.q);
    nfine += N.fine_n_h[j];
  }
  N.nfine = nfine;
  if ((rc = grow(ctx, (void**)&N.fgeo, &N.fgeo_cap, sizeof(double) * 7 * nfine, "fine geometry")) ||
      (rc = grow(ctx, (void**)&N.fgeo32, &N.fgeo32_cap, sizeof(float) * 7 * nfine, "fine geometry")) ||
      (rc = grow(ctx, (void**)&N.fstr, &N.fstr_cap, sizeof(double) * 6 * nfine, "fine strengths")) ||
      (rc = grow(ctx, (void**)&N.fstr32, &N.fstr32_cap, sizeof(float) * 6 * nfine, "fine strengths")) ||
      (rc = grow(ctx, (void**)&N.fgeo32lo, &N.fgeo32lo_cap, sizeof(float) * 7 * nfine, "fine geometry low parts")) ||
      (rc = grow(ctx, (void**)&N.fstr32lo, &N.fstr32lo_cap, sizeof(float) * 6 * nfine, "fine strengths low parts")) ||
      (rc = grow(ctx, (void**)&N.foff_dev, &N.foff_cap, sizeof(int64_t) * 2 * nd, "fine offsets")))
    return rc;
  {
    std::vector<int64_t> both(2 * nd);
    for (int j = 0; j < nd; ++j) {
      both[j] = N.fine_off_h[j];
      both[nd + j] = N.fine_n_h[j];
    }
    SHBIM_CUDA(ctx, cudaMemcpy(N.foff_dev, both.data(), sizeof(int64_t) * 2 * nd, cudaMemcpyHostToDevice));
  }
  // near drops grouped by degree for the per-application upsampled strengths
  for (auto& g : N.groups_d) {
    cudaFree(g.idx);
    cudaFree(g.coef);
    cudaFree(g.fine);
  }
  N.groups_d.clear();
  for (int j = 0; j < nd; ++j) {
    if (N.fine_off_h[j] < 0) continue;
    bool seen = false;
    for (const auto& g : N.groups_d) seen = seen || g.tab == ctx->drops[j].tab;
    if (seen) continue;
    std::vector<int> idx;
    std::vector<int64_t> co, fo;
    for (int k = j; k < nd; ++k)
      if (N.fine_off_h[k] >= 0 && ctx->drops[k].tab == ctx->drops[j].tab) {
        idx.push_back(k);
        co.push_back(ctx->drops[k].coef_off);
        fo.push_back(N.fine_off_h[k]);
      }
    N.groups_d.push_back(shbim_ctx::Near::DegGroup{});
    auto& g = N.groups_d.back();
    g.tab = ctx->drops[j].tab;
    g.n = (int)idx.size();
    if (cudaMalloc(&g.idx, idx.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&g.coef, co.size() * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&g.fine, fo.size() * sizeof(int64_t)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "near degree groups");
    SHBIM_CUDA(ctx, cudaMemcpy(g.idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
    SHBIM_CUDA(ctx, cudaMemcpy(g.coef, co.data(), co.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    SHBIM_CUDA(ctx, cudaMemcpy(g.fine, fo.data(), fo.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  }
  int64_t maxn = 0;
  for (int j = 0; j < nd; ++j) maxn = std::max(maxn, N.fine_n_h[j]);
  double* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(double) * 9 * maxn) != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "fine scratch");
  for (int j = 0; j < nd && rc == SHBIM_OK; ++j) {
    if (N.fine_off_h[j] < 0) continue;
    const Drop& d = ctx->drops[j];
    const GridTables& fine = d.tab->fine;
    const int64_t n = N.fine_n_h[j];
    rc = sht_synth(ctx, fine, 3, xcoef + 3 * d.coef_off, d.nc, 7, tmp, 3 * n, n, nullptr, nullptr, s);
    if (rc == SHBIM_OK)
      rc = geometry_kernel32(ctx, tmp, n, 3, fine, N.fgeo, N.fgeo32, nfine, N.fine_off_h[j], d.centre, s,
                             N.fgeo32lo);
  }
  if (rc == SHBIM_OK) {
    // smallest target-to-surface distance over the near pairs (sampled on the upsampled grids)
    unsigned* mins = reinterpret_cast<unsigned*>(tmp);
    const unsigned init[2] = {0x7f7fffffu, 0x7f7fffffu};
    cudaMemcpyAsync(mins, init, sizeof(init), cudaMemcpyHostToDevice, s);
    k_near_min_dist<<<nb((int64_t)cnt * 32), 256, 0, s>>>(ctx->geo.tgt, ctx->ntarget, N.pair_t, N.pair_j, cnt,
                                                         ctx->drops_dev, nd, N.fgeo32, nfine, N.foff_dev, N.stats,
                                                         mins);
    ctx->launches++;
    unsigned h[2] = {0u, 0u};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, mins, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      rc = cuda_fail(ctx, e, "k_near_min_dist");
    } else {
      float d2, r2;
      std::memcpy(&d2, &h[0], sizeof(float));
      std::memcpy(&r2, &h[1], sizeof(float));
      N.min_dist = std::sqrt((double)d2);
      N.min_ratio = std::sqrt((double)r2);
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(tmp);
  return rc;
}

namespace {

int launch_direct(shbim_ctx* ctx, int kind, bool has_f, bool has_u, double* out, cudaStream_t s) {
  auto& N = ctx->near;
  NearArgs A{N.pair_t, N.pair_j, N.foff_dev, N.foff_dev + ctx->n_drops, ctx->drops_dev, ctx->geo.tgt_drop,
             ctx->geo.tgt, ctx->ntarget, N.fgeo, N.fgeo32, N.fstr, N.fstr32, N.nfine, ctx->geo.src,
             ctx->geo.src32, ctx->dens_up, ctx->dens_up32, ctx->nsource, N.fgeo32lo, N.fstr32lo,
             ctx->geo.src32lo, ctx->dens_up32lo, has_f ? 1 : 0, has_u ? 1 : 0, out};
  const int mode = ctx->opts.precision == SHBIM_PREC_FP32_COMP ? 1 : (ctx->opts.precision == SHBIM_PREC_DF64 ? 2 : 0);
  // enough CTAs for ~8 per SM: each near pair's sums are split into chunks of both grids
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(32, (8ll * nsm + N.npairs - 1) / N.npairs));
  const dim3 g((unsigned)N.npairs, (unsigned)chunks);
  if (mode != 0) {
    // FP32 and double-float: tiled over groups of targets sharing a source drop
    // chunks of at least 512 nodes, enough CTAs for ~8 per SM
    int64_t nmax = 0;
    for (int j = 0; j < ctx->n_drops; ++j)
      if (N.fine_off_h[j] >= 0) nmax = std::max<int64_t>(nmax, N.fine_n_h[j] + ctx->drops[j].ns);
    const int gc = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::max<int64_t>(1, nmax / 512), (8ll * nsm + N.ngroups - 1) / N.ngroups));
    const dim3 gg((unsigned)N.ngroups, (unsigned)gc);
    if (mode == 1) {
      if (kind == 0) k_near_tiled32<0><<<gg, kNearGroup, 0, s>>>(A, N.groups);
      else if (kind == 1) k_near_tiled32<1><<<gg, kNearGroup, 0, s>>>(A, N.groups);
      else k_near_tiled32<2><<<gg, kNearGroup, 0, s>>>(A, N.groups);
    } else {
      if (kind == 0) k_near_tiled_df<0><<<gg, kNearGroup, 0, s>>>(A, N.groups);
      else if (kind == 1) k_near_tiled_df<1><<<gg, kNearGroup, 0, s>>>(A, N.groups);
      else k_near_tiled_df<2><<<gg, kNearGroup, 0, s>>>(A, N.groups);
    }
    SHBIM_CHECK_LAUNCH(ctx, "k_near_tiled");
    return SHBIM_OK;
  }
  if (kind == 0) {
    if (mode == 1) k_near_direct<0, 1><<<g, 256, 0, s>>>(A);
    else if (mode == 2) k_near_direct<0, 2><<<g, 256, 0, s>>>(A);
    else k_near_direct<0, 0><<<g, 256, 0, s>>>(A);
  } else if (kind == 1) {
    if (mode == 1) k_near_direct<1, 1><<<g, 256, 0, s>>>(A);
    else if (mode == 2) k_near_direct<1, 2><<<g, 256, 0, s>>>(A);
    else k_near_direct<1, 0><<<g, 256, 0, s>>>(A);
  } else {
    if (mode == 1) k_near_direct<2, 1><<<g, 256, 0, s>>>(A);
    else if (mode == 2) k_near_direct<2, 2><<<g, 256, 0, s>>>(A);
    else k_near_direct<2, 0><<<g, 256, 0, s>>>(A);
  }
  SHBIM_CHECK_LAUNCH(ctx, "k_near_direct");
  return SHBIM_OK;
}

}  // namespace

int apply_near_laplace(shbim_ctx* ctx, int which, const double* dens, double* out, cudaStream_t s,
                       cudaEvent_t before_sums) {
  auto& N = ctx->near;
  if (N.npairs == 0) return SHBIM_OK;
  const bool f32 = ctx->opts.precision != SHBIM_PREC_FP64;
  const bool lo = ctx->opts.precision == SHBIM_PREC_DF64;
  for (const auto& g : N.groups_d) {
    const DropList L{g.idx, g.coef, g.fine};
    int rc = sht_synth_drops(ctx, g.tab->fine, g.n, 1, dens, ncoef(g.tab->p), N.fstr, 0, 0, N.fgeo + 6 * N.nfine, 1.0,
                             nullptr, f32 ? N.fstr32 : nullptr, s, lo ? N.fstr32lo : nullptr, &L);
    if (rc) return rc;
  }
  if (before_sums) SHBIM_CUDA(ctx, cudaStreamWaitEvent(s, before_sums, 0));
  return launch_direct(ctx, which == SHBIM_LAPLACE_SL ? 1 : 0, false, false, out, s);
}

int apply_near_stokes(shbim_ctx* ctx, const double* f, const double* u, double* out, cudaStream_t s,
                      cudaEvent_t before_sums) {
  auto& N = ctx->near;
  if (N.npairs == 0) return SHBIM_OK;
  const bool f32 = ctx->opts.precision != SHBIM_PREC_FP64;
  const bool lo = ctx->opts.precision == SHBIM_PREC_DF64;
  for (const auto& g : N.groups_d) {
    const DropList L{g.idx, g.coef, g.fine};
    const int nc = ncoef(g.tab->p);
    const double* w = N.fgeo + 6 * N.nfine;
    int rc;
    if (f && (rc = sht_synth_drops(ctx, g.tab->fine, g.n, 3, f, nc, N.fstr, N.nfine, 0, w, 1.0, nullptr,
                                   f32 ? N.fstr32 : nullptr, s, lo ? N.fstr32lo : nullptr, &L)))
      return rc;
    // strength -6 (lambda_j - 1) u per drop
    if (u && (rc = sht_synth_drops(ctx, g.tab->fine, g.n, 3, u, nc, N.fstr + 3 * N.nfine, N.nfine, 0, w, -6.0,
                                   ctx->lamm1_dev, f32 ? N.fstr32 + 3 * N.nfine : nullptr, s,
                                   lo ? N.fstr32lo + 3 * N.nfine : nullptr, &L)))
      return rc;
  }
  if (before_sums) SHBIM_CUDA(ctx, cudaStreamWaitEvent(s, before_sums, 0));
  return launch_direct(ctx, 2, f != nullptr, u != nullptr, out, s);
}

}  // namespace shbim

extern "C" int shbim_set_near(shbim_ctx* ctx, int on) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->near.enabled = on != 0;
  if (!ctx->near.enabled) ctx->near.npairs = 0;
  return SHBIM_OK;
}

extern "C" int shbim_near_pairs(shbim_ctx* ctx) { return ctx ? ctx->near.npairs : -1; }

extern "C" int shbim_near_min_distance(shbim_ctx* ctx, double* dist_host, double* ratio_host) {
  if (!ctx) return SHBIM_ERR_ARG;
  if (dist_host) *dist_host = ctx->near.min_dist;
  if (ratio_host) *ratio_host = ctx->near.min_ratio;
  return SHBIM_OK;
}
