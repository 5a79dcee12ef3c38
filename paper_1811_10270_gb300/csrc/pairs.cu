// Tiled all-pairs sums of the regular rule (Eq. reg_quadrature) between different drops:
// Laplace single layer and target-normal double layer (Eqs. E_n, dl_op_laplace), Stokeslet and
// stresslet (Eqs. GandT, op_stokes). Same-drop pairs are excluded: those targets get the
// singular self rows instead.
//
// Work decomposition: the target list is cut into tiles of 512 targets of one drop; a CTA owns
// 128 threads x TPT targets of a tile (register blocking, TPT = 1, 2 or 4, so a tile takes 4/TPT
// CTAs) and one split of the other drops' sources; sources are staged through shared memory in
// tiles of 256 and read as warp-wide broadcasts. Each split writes its own partial sums; a second
// kernel adds the splits in a fixed order (deterministic). TPT, the split count and the launch
// form (a CTA per unit, or persistent CTAs on an atomic work counter) are chosen per kernel kind
// and drop layout by timing the candidates on the first FP32 launch (autotune).
//
// Double-float path (FP64-class accuracy on the FP32 pipe): every source coordinate, normal and
// strength is the pair (FP32 copy, FP32 low part of the FP64 value), the target offset from the
// source drop's centre likewise; differences, r^2, 1/r (Newton from the FP32 seed), products and
// the running sums are double-float (~2^-44 relative per operation; error-free transformations
// of Knuth and Dekker). On this GPU that is several times faster than FP64 arithmetic.
//
// FP32 path: sources are stored relative to their drop centre in FP32; for every (target,
// source drop) the target offset x0 - c_j is formed in FP64 and kept as an unevaluated FP32
// sum hi + lo, so xh = (hi - xs) + lo carries an error of order eps * r rather than
// eps * |x0 - c_j| (drops 0.1 apart stay accurate). Each source tile is summed in FP32 and
// added to a (hi, lo) accumulator with the two-sum of Knuth (compensated accumulation).
#include <algorithm>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "pair_df.cuh"
#include "pair_dq.cuh"

namespace shbim {

namespace {

constexpr int kTile = 256;
constexpr int kThreads = 128;
constexpr int kMaxTPT = 4;                         // largest register blocking
constexpr int kTileTargets = kThreads * kMaxTPT;   // targets per tile of the tile list

// Stokes kinds: both terms (STO), the Stokeslet on f alone (STS: right-hand sides) and the stresslet on u
// alone (STD: the GMRES operator); the single-term kinds skip the other term's arithmetic
enum Kind { LDL = 0, LSL = 1, STO = 2, STS = 3, STD = 4 };
__host__ __device__ constexpr bool stokes_kind(int k) { return k >= STO; }

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float a) {
  const float s = hi + a;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (a - bp);
  hi = s;
  lo += e;
}

// virtual source index v in [0, nsource - ns_i) skips drop i's own sources
struct SrcRange {
  int64_t a, b;
};

__device__ __forceinline__ SrcRange drop_range(const DropDev& Di, const DropDev& Dj, int i, int j,
                                               int64_t v0, int64_t v1) {
  const int64_t shift = (j > i) ? Di.ns : 0;
  const int64_t vs = Dj.src_off - shift;
  const int64_t ve = vs + Dj.ns;
  SrcRange r;
  r.a = max(v0, vs) + shift;
  r.b = min(v1, ve) + shift;
  return r;
}

// bx = tile * (kMaxTPT / TPT) + sub-tile; returns false for a sub-tile past the tile's last
// target (the whole CTA then skips it, before any barrier)
template <int TPT>
__device__ __forceinline__ bool sub_tile(const PairTile* __restrict__ tiles, PairTile& t, int bx) {
  constexpr int SUB = kMaxTPT / TPT;
  const PairTile tile = tiles[bx / SUB];
  const int off = (int)(bx % SUB) * kThreads * TPT;
  t.drop = tile.drop;
  t.t0 = tile.t0 + off;
  t.nt = tile.nt - off;
  return t.nt > 0;
}

// One work unit of the FP32 sums: sub-tile bx of the tile list, source split by. Returns at once
// (uniformly for the CTA) for an empty sub-tile.
template <int KIND, int kTPT>
__device__ __forceinline__ void pairs32_unit(int bx, int by, const PairTile* __restrict__ tiles,
                                             const DropDev* __restrict__ drops, int n_drops,
                                             const double* __restrict__ tgt, int64_t ntarget,
                                             const float* __restrict__ src32, int64_t nsource,
                                             const float* __restrict__ dens32, int nsplit, int has_f, int has_u,
                                             double* __restrict__ part, float4* __restrict__ sh0,
                                             float4* __restrict__ sh1, float4* __restrict__ sh2) {
  constexpr int NC = stokes_kind(KIND) ? 3 : 1;
  PairTile tile;
  if (!sub_tile<kTPT>(tiles, tile, bx)) return;
  const int i = tile.drop;
  const DropDev Di = drops[i];
  const int64_t other = nsource - Di.ns;
  const int64_t chunk = (other + nsplit - 1) / nsplit;
  const int64_t v0 = (int64_t)by * chunk;
  const int64_t v1 = min(other, v0 + chunk);

  int64_t tg[kTPT];
  bool ok[kTPT];
  double X0[kTPT][3];
  float N0[kTPT][3];
#pragma unroll
  for (int k = 0; k < kTPT; ++k) {
    tg[k] = tile.t0 + threadIdx.x + k * kThreads;
    ok[k] = tg[k] < (int64_t)tile.t0 + tile.nt;
    const int64_t t = ok[k] ? tg[k] : tile.t0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X0[k][c] = tgt[c * ntarget + t];
      N0[k][c] = (float)tgt[(3 + c) * ntarget + t];
    }
  }
  float hi[kTPT][NC], lo[kTPT][NC];
#pragma unroll
  for (int k = 0; k < kTPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) hi[k][c] = lo[k][c] = 0.f;

  for (int j = 0; j < n_drops; ++j) {
    if (j == i) continue;
    const DropDev Dj = drops[j];
    const SrcRange rg = drop_range(Di, Dj, i, j, v0, v1);
    if (rg.a >= rg.b) continue;
    float th[kTPT][3], tl[kTPT][3];
    const double cj[3] = {Dj.cx, Dj.cy, Dj.cz};
#pragma unroll
    for (int k = 0; k < kTPT; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double d = X0[k][c] - cj[c];
        const float h = (float)d;
        th[k][c] = h;
        tl[k][c] = (float)(d - (double)h);
      }
    for (int64_t base = rg.a; base < rg.b; base += kTile) {
      const int cnt = (int)min((int64_t)kTile, rg.b - base);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += kThreads) {
        const int64_t sI = base + e;
        const float x = src32[sI], y = src32[nsource + sI], z = src32[2 * nsource + sI];
        if (!stokes_kind(KIND)) {
          sh0[e] = make_float4(x, y, z, dens32[sI]);
        } else {
          const float fx = has_f ? dens32[sI] : 0.f;
          const float fy = has_f ? dens32[nsource + sI] : 0.f;
          const float fz = has_f ? dens32[2 * nsource + sI] : 0.f;
          const float ux = has_u ? dens32[3 * nsource + sI] : 0.f;
          const float uy = has_u ? dens32[4 * nsource + sI] : 0.f;
          const float uz = has_u ? dens32[5 * nsource + sI] : 0.f;
          sh0[e] = make_float4(x, y, z, fx);
          sh1[e] = make_float4(fy, fz, ux, uy);
          sh2[e] = make_float4(uz, src32[3 * nsource + sI], src32[4 * nsource + sI],
                               src32[5 * nsource + sI]);
        }
      }
      __syncthreads();
      float acc[kTPT][NC];
#pragma unroll
      for (int k = 0; k < kTPT; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[k][c] = 0.f;
#pragma unroll 4
      for (int e = 0; e < cnt; ++e) {
        const float4 A = sh0[e];
        if (!stokes_kind(KIND)) {
#pragma unroll
          for (int k = 0; k < kTPT; ++k) {
            const float dx = (th[k][0] - A.x) + tl[k][0];
            const float dy = (th[k][1] - A.y) + tl[k][1];
            const float dz = (th[k][2] - A.z) + tl[k][2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrtf(r2);
            if (KIND == LSL) {
              acc[k][0] = fmaf(A.w, ri, acc[k][0]);
            } else {
              const float ri3 = ri * ri * ri;
              const float dn = fmaf(dx, N0[k][0], fmaf(dy, N0[k][1], dz * N0[k][2]));
              acc[k][0] = fmaf(A.w * ri3, dn, acc[k][0]);
            }
          }
        } else {
          const float4 B = sh1[e];
          const float4 C = sh2[e];
#pragma unroll
          for (int k = 0; k < kTPT; ++k) {
            const float dx = (th[k][0] - A.x) + tl[k][0];
            const float dy = (th[k][1] - A.y) + tl[k][1];
            const float dz = (th[k][2] - A.z) + tl[k][2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrtf(r2);
            const float ri2 = ri * ri;
            const float ri3 = ri2 * ri;
            if (KIND == STD) {
              const float hu = fmaf(dx, B.z, fmaf(dy, B.w, dz * C.x));
              const float hn = fmaf(dx, C.y, fmaf(dy, C.z, dz * C.w));
              const float t = (hu * hn) * (ri3 * ri2);
              acc[k][0] = fmaf(dx, t, acc[k][0]);
              acc[k][1] = fmaf(dy, t, acc[k][1]);
              acc[k][2] = fmaf(dz, t, acc[k][2]);
            } else {
              const float hf = fmaf(dx, A.w, fmaf(dy, B.x, dz * B.y));
              float t;
              if (KIND == STS) {
                t = ri3 * hf;
              } else {
                const float hu = fmaf(dx, B.z, fmaf(dy, B.w, dz * C.x));
                const float hn = fmaf(dx, C.y, fmaf(dy, C.z, dz * C.w));
                t = ri3 * fmaf(hu * hn, ri2, hf);
              }
              acc[k][0] = fmaf(A.w, ri, fmaf(dx, t, acc[k][0]));
              acc[k][1] = fmaf(B.x, ri, fmaf(dy, t, acc[k][1]));
              acc[k][2] = fmaf(B.y, ri, fmaf(dz, t, acc[k][2]));
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kTPT; ++k)
#pragma unroll
        for (int c = 0; c < NC; ++c) two_sum_acc(hi[k][c], lo[k][c], acc[k][c]);
    }
  }
  double* P = part + (int64_t)by * NC * ntarget;
#pragma unroll
  for (int k = 0; k < kTPT; ++k) {
    if (!ok[k]) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double v = 0.07957747154594766788 * ((double)hi[k][c] + (double)lo[k][c]);
      const int64_t o = (NC == 1) ? tg[k] : 3 * Di.tgt_off + (int64_t)c * Di.nt + (tg[k] - Di.tgt_off);
      P[o] = v;
    }
  }
}

// one CTA per work unit (grid = sub-tiles x splits)
template <int KIND, int kTPT>
__global__ void __launch_bounds__(kThreads)
k_pairs32(const PairTile* __restrict__ tiles, const DropDev* __restrict__ drops, int n_drops,
          const double* __restrict__ tgt, int64_t ntarget, const float* __restrict__ src32,
          int64_t nsource, const float* __restrict__ dens32, int nsplit, int has_f, int has_u,
          double* __restrict__ part) {
  __shared__ float4 sh0[kTile];
  __shared__ float4 sh1[stokes_kind(KIND) ? kTile : 1];
  __shared__ float4 sh2[stokes_kind(KIND) ? kTile : 1];
  pairs32_unit<KIND, kTPT>(blockIdx.x, blockIdx.y, tiles, drops, n_drops, tgt, ntarget, src32, nsource, dens32,
                           nsplit, has_f, has_u, part, sh0, sh1, sh2);
}

// Persistent form: resident CTAs take work units from an atomic counter, in the order of the tile
// list (sorted by cost, largest first), splits of a sub-tile consecutively. The last CTA to
// finish puts the counter back to zero for the next launch on the stream. No CTA waits on another.
template <int KIND, int kTPT>
__global__ void __launch_bounds__(kThreads)
k_pairs32_queue(const PairTile* __restrict__ tiles, const DropDev* __restrict__ drops, int n_drops,
                const double* __restrict__ tgt, int64_t ntarget, const float* __restrict__ src32,
                int64_t nsource, const float* __restrict__ dens32, int nsplit, int has_f, int has_u,
                double* __restrict__ part, int nunits, int* __restrict__ queue) {
  __shared__ float4 sh0[kTile];
  __shared__ float4 sh1[stokes_kind(KIND) ? kTile : 1];
  __shared__ float4 sh2[stokes_kind(KIND) ? kTile : 1];
  __shared__ int s_unit;
  for (;;) {
    __syncthreads();   // every thread is done with the previous unit's shared tiles and index
    if (threadIdx.x == 0) s_unit = atomicAdd(queue, 1);
    __syncthreads();
    const int u = s_unit;
    if (u >= nunits) break;
    pairs32_unit<KIND, kTPT>(u / nsplit, u - (u / nsplit) * nsplit, tiles, drops, n_drops, tgt, ntarget, src32,
                             nsource, dens32, nsplit, has_f, has_u, part, sh0, sh1, sh2);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
      queue[0] = 0;
      queue[1] = 0;
      __threadfence();
    }
  }
}

template <int KIND>
__global__ void __launch_bounds__(kThreads)
k_pairs_df(const PairTile* __restrict__ tiles, const DropDev* __restrict__ drops, int n_drops,
           const double* __restrict__ tgt, int64_t ntarget, const float* __restrict__ src32,
           const float* __restrict__ src32lo, int64_t nsource, const float* __restrict__ dens32,
           const float* __restrict__ dens32lo, int nsplit, int has_f, int has_u, double* __restrict__ part) {
  using dfl::df;
  constexpr int NC = stokes_kind(KIND) ? 3 : 1;
  constexpr int NV = stokes_kind(KIND) ? 6 : 2;   // float4 per staged source
  __shared__ float4 sh[NV][kTile];
  PairTile tile;
  if (!sub_tile<1>(tiles, tile, blockIdx.x)) return;
  const int i = tile.drop;
  const DropDev Di = drops[i];
  const int64_t other = nsource - Di.ns;
  const int64_t chunk = (other + nsplit - 1) / nsplit;
  const int64_t v0 = (int64_t)blockIdx.y * chunk;
  const int64_t v1 = min(other, v0 + chunk);
  const int64_t tg = tile.t0 + threadIdx.x;
  const bool ok = (int)threadIdx.x < tile.nt;
  const int64_t t = ok ? tg : tile.t0;
  double X0[3];
  df N0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X0[c] = tgt[c * ntarget + t];
    N0[c] = dfl::from_double(tgt[(3 + c) * ntarget + t]);
  }
  dfl::acc A[NC];
  for (int j = 0; j < n_drops; ++j) {
    if (j == i) continue;
    const DropDev Dj = drops[j];
    const SrcRange rg = drop_range(Di, Dj, i, j, v0, v1);
    if (rg.a >= rg.b) continue;
    const df T[3] = {dfl::from_double(X0[0] - Dj.cx), dfl::from_double(X0[1] - Dj.cy),
                     dfl::from_double(X0[2] - Dj.cz)};
    for (int64_t base = rg.a; base < rg.b; base += kTile) {
      const int cnt = (int)min((int64_t)kTile, rg.b - base);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += kThreads) {
        const int64_t sI = base + e;
        const float xh = src32[sI], yh = src32[nsource + sI], zh = src32[2 * nsource + sI];
        const float xl = src32lo[sI], yl = src32lo[nsource + sI], zl = src32lo[2 * nsource + sI];
        if (!stokes_kind(KIND)) {
          sh[0][e] = make_float4(xh, yh, zh, xl);
          sh[1][e] = make_float4(yl, zl, dens32[sI], dens32lo[sI]);
        } else {
          float fv[6], uv[6];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            fv[2 * c] = has_f ? dens32[c * nsource + sI] : 0.f;
            fv[2 * c + 1] = has_f ? dens32lo[c * nsource + sI] : 0.f;
            uv[2 * c] = has_u ? dens32[(3 + c) * nsource + sI] : 0.f;
            uv[2 * c + 1] = has_u ? dens32lo[(3 + c) * nsource + sI] : 0.f;
          }
          sh[0][e] = make_float4(xh, yh, zh, xl);
          sh[1][e] = make_float4(yl, zl, fv[0], fv[1]);
          sh[2][e] = make_float4(fv[2], fv[3], fv[4], fv[5]);
          sh[3][e] = make_float4(uv[0], uv[1], uv[2], uv[3]);
          sh[4][e] = make_float4(uv[4], uv[5], src32[3 * nsource + sI], src32lo[3 * nsource + sI]);
          sh[5][e] = make_float4(src32[4 * nsource + sI], src32lo[4 * nsource + sI], src32[5 * nsource + sI],
                                 src32lo[5 * nsource + sI]);
        }
      }
      __syncthreads();
      for (int e = 0; e < cnt; ++e) {
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr (!stokes_kind(KIND))
          df_term<KIND>(T, N0, sh[0][e], sh[1][e], z4, z4, z4, z4, A);
        else
          df_term<KIND>(T, N0, sh[0][e], sh[1][e], sh[2][e], sh[3][e], sh[4][e], sh[5][e], A);
      }
    }
  }
  if (!ok) return;
  double* P = part + (int64_t)blockIdx.y * NC * ntarget;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t o = (NC == 1) ? tg : 3 * Di.tgt_off + (int64_t)c * Di.nt + (tg - Di.tgt_off);
    P[o] = 0.07957747154594766788 * dfl::to_double(A[c].value());
  }
}

// FP64-class sums, per source drop either on quantised positions (pair_dq.cuh) or in general
// double-float (pair_df.cuh): dq_far[i * n_drops + j] != 0 selects the quantised form for targets of drop
// i against sources of drop j. Its positions are exact to ~2^-(Q+25) absolute (the FP32 remainder below
// the quantum 2^-Q), which is double-float accuracy relative to r only for pairs at least ~2^(19-Q)
// apart: the host sets the flag for drop pairs whose surfaces are that far apart. The choice is uniform
// for a CTA (its targets are on one drop). Quantised copy srcq: [xq yq zq][xl yl zl], each [nsource];
// qs = 2^Q, qi = 2^-Q.
template <int KIND>
__global__ void __launch_bounds__(kThreads)
k_pairs_dq(const PairTile* __restrict__ tiles, const DropDev* __restrict__ drops, int n_drops,
           const double* __restrict__ tgt, int64_t ntarget, const float* __restrict__ srcq,
           const float* __restrict__ src32, const float* __restrict__ src32lo, int64_t nsource,
           const float* __restrict__ dens32, const float* __restrict__ dens32lo, int nsplit, int has_f, int has_u,
           double qs, double qi, const unsigned char* __restrict__ dq_far, double* __restrict__ part) {
  using dfl::df;
  constexpr int NC = stokes_kind(KIND) ? 3 : 1;
  constexpr int NV = stokes_kind(KIND) ? 6 : 2;   // float4 per staged source
  __shared__ float4 sh[NV][kTile];
  PairTile tile;
  if (!sub_tile<1>(tiles, tile, blockIdx.x)) return;
  const int i = tile.drop;
  const DropDev Di = drops[i];
  const int64_t other = nsource - Di.ns;
  const int64_t chunk = (other + nsplit - 1) / nsplit;
  const int64_t v0 = (int64_t)blockIdx.y * chunk;
  const int64_t v1 = min(other, v0 + chunk);
  const int64_t tg = tile.t0 + threadIdx.x;
  const bool ok = (int)threadIdx.x < tile.nt;
  const int64_t t = ok ? tg : tile.t0;
  double X0[3];
  df N0[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    X0[c] = tgt[c * ntarget + t];
    N0[c] = dfl::from_double(tgt[(3 + c) * ntarget + t]);
  }
  dfl::acc A[NC];
  for (int j = 0; j < n_drops; ++j) {
    if (j == i) continue;
    const DropDev Dj = drops[j];
    const SrcRange rg = drop_range(Di, Dj, i, j, v0, v1);
    if (rg.a >= rg.b) continue;
    const bool far = dq_far[(int64_t)i * n_drops + j] != 0;
    const double cj[3] = {Dj.cx, Dj.cy, Dj.cz};
    float Th[3], Tl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v = X0[c] - cj[c];
      const double h = far ? rint(v * qs) * qi : (double)(float)v;
      Th[c] = (float)h;
      Tl[c] = (float)(v - h);
    }
    const float* phi = far ? srcq : src32;
    const float* plo = far ? srcq + 3 * nsource : src32lo;
    for (int64_t base = rg.a; base < rg.b; base += kTile) {
      const int cnt = (int)min((int64_t)kTile, rg.b - base);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += kThreads) {
        const int64_t sI = base + e;
        const float xh = phi[sI], yh = phi[nsource + sI], zh = phi[2 * nsource + sI];
        const float xl = plo[sI], yl = plo[nsource + sI], zl = plo[2 * nsource + sI];
        if (!stokes_kind(KIND)) {
          sh[0][e] = make_float4(xh, yh, zh, xl);
          sh[1][e] = make_float4(yl, zl, dens32[sI], dens32lo[sI]);
        } else {
          float fv[6], uv[6];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            fv[2 * c] = has_f ? dens32[c * nsource + sI] : 0.f;
            fv[2 * c + 1] = has_f ? dens32lo[c * nsource + sI] : 0.f;
            uv[2 * c] = has_u ? dens32[(3 + c) * nsource + sI] : 0.f;
            uv[2 * c + 1] = has_u ? dens32lo[(3 + c) * nsource + sI] : 0.f;
          }
          sh[0][e] = make_float4(xh, yh, zh, xl);
          sh[1][e] = make_float4(yl, zl, fv[0], fv[1]);
          sh[2][e] = make_float4(fv[2], fv[3], fv[4], fv[5]);
          sh[3][e] = make_float4(uv[0], uv[1], uv[2], uv[3]);
          sh[4][e] = make_float4(uv[4], uv[5], src32[3 * nsource + sI], src32lo[3 * nsource + sI]);
          sh[5][e] = make_float4(src32[4 * nsource + sI], src32lo[4 * nsource + sI], src32[5 * nsource + sI],
                                 src32lo[5 * nsource + sI]);
        }
      }
      __syncthreads();
      const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (far) {
        for (int e = 0; e < cnt; ++e) {
          if constexpr (!stokes_kind(KIND))
            dq_term<KIND>(Th, Tl, N0, sh[0][e], sh[1][e], z4, z4, z4, z4, A);
          else
            dq_term<KIND>(Th, Tl, N0, sh[0][e], sh[1][e], sh[2][e], sh[3][e], sh[4][e], sh[5][e], A);
        }
      } else {
        const df T[3] = {df{Th[0], Tl[0]}, df{Th[1], Tl[1]}, df{Th[2], Tl[2]}};
        for (int e = 0; e < cnt; ++e) {
          if constexpr (!stokes_kind(KIND))
            df_term<KIND>(T, N0, sh[0][e], sh[1][e], z4, z4, z4, z4, A);
          else
            df_term<KIND>(T, N0, sh[0][e], sh[1][e], sh[2][e], sh[3][e], sh[4][e], sh[5][e], A);
        }
      }
    }
  }
  if (!ok) return;
  double* P = part + (int64_t)blockIdx.y * NC * ntarget;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int64_t o = (NC == 1) ? tg : 3 * Di.tgt_off + (int64_t)c * Di.nt + (tg - Di.tgt_off);
    P[o] = 0.07957747154594766788 * dfl::to_double(A[c].value());
  }
}

template <int KIND, int kTPT>
__global__ void __launch_bounds__(kThreads)
k_pairs64(const PairTile* __restrict__ tiles, const DropDev* __restrict__ drops, int n_drops,
          const double* __restrict__ tgt, int64_t ntarget, const double* __restrict__ src,
          int64_t nsource, const double* __restrict__ dens, int nsplit, int has_f, int has_u,
          double* __restrict__ part) {
  constexpr int NC = stokes_kind(KIND) ? 3 : 1;
  constexpr int NF = stokes_kind(KIND) ? 12 : 4;
  __shared__ double sh[NF][kTile];
  PairTile tile;
  if (!sub_tile<kTPT>(tiles, tile, blockIdx.x)) return;
  const int i = tile.drop;
  const DropDev Di = drops[i];
  const int64_t other = nsource - Di.ns;
  const int64_t chunk = (other + nsplit - 1) / nsplit;
  const int64_t v0 = (int64_t)blockIdx.y * chunk;
  const int64_t v1 = min(other, v0 + chunk);
  int64_t tg[kTPT];
  bool ok[kTPT];
  double X0[kTPT][3], N0[kTPT][3], acc[kTPT][NC];
#pragma unroll
  for (int k = 0; k < kTPT; ++k) {
    tg[k] = tile.t0 + threadIdx.x + k * kThreads;
    ok[k] = tg[k] < (int64_t)tile.t0 + tile.nt;
    const int64_t t = ok[k] ? tg[k] : tile.t0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X0[k][c] = tgt[c * ntarget + t];
      N0[k][c] = tgt[(3 + c) * ntarget + t];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[k][c] = 0.0;
  }
  for (int j = 0; j < n_drops; ++j) {
    if (j == i) continue;
    const DropDev Dj = drops[j];
    const SrcRange rg = drop_range(Di, Dj, i, j, v0, v1);
    if (rg.a >= rg.b) continue;
    for (int64_t base = rg.a; base < rg.b; base += kTile) {
      const int cnt = (int)min((int64_t)kTile, rg.b - base);
      __syncthreads();
      for (int e = threadIdx.x; e < cnt; e += kThreads) {
        const int64_t sI = base + e;
        sh[0][e] = src[sI];
        sh[1][e] = src[nsource + sI];
        sh[2][e] = src[2 * nsource + sI];
        if (!stokes_kind(KIND)) {
          sh[3][e] = dens[sI];
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            sh[3 + c][e] = has_f ? dens[c * nsource + sI] : 0.0;
            sh[6 + c][e] = has_u ? dens[(3 + c) * nsource + sI] : 0.0;
            sh[9 + c][e] = src[(3 + c) * nsource + sI];
          }
        }
      }
      __syncthreads();
      for (int e = 0; e < cnt; ++e) {
        const double sx = sh[0][e], sy = sh[1][e], sz = sh[2][e];
#pragma unroll
        for (int k = 0; k < kTPT; ++k) {
          const double dx = X0[k][0] - sx, dy = X0[k][1] - sy, dz = X0[k][2] - sz;
          const double r2 = dx * dx + dy * dy + dz * dz;
          const double ri = rsqrt(r2);
          if (KIND == LSL) {
            acc[k][0] = fma(sh[3][e], ri, acc[k][0]);
          } else if (KIND == LDL) {
            const double dn = dx * N0[k][0] + dy * N0[k][1] + dz * N0[k][2];
            acc[k][0] = fma(sh[3][e] * ri * ri * ri, dn, acc[k][0]);
          } else {
            const double ri2 = ri * ri, ri3 = ri2 * ri;
            const double fx = sh[3][e], fy = sh[4][e], fz = sh[5][e];
            const double hf = KIND == STD ? 0.0 : dx * fx + dy * fy + dz * fz;
            const double hu = KIND == STS ? 0.0 : dx * sh[6][e] + dy * sh[7][e] + dz * sh[8][e];
            const double hn = KIND == STS ? 0.0 : dx * sh[9][e] + dy * sh[10][e] + dz * sh[11][e];
            const double t = ri3 * (hf + hu * hn * ri2);
            if (KIND == STD) {
              acc[k][0] += dx * t;
              acc[k][1] += dy * t;
              acc[k][2] += dz * t;
            } else {
              acc[k][0] += fx * ri + dx * t;
              acc[k][1] += fy * ri + dy * t;
              acc[k][2] += fz * ri + dz * t;
            }
          }
        }
      }
    }
  }
  double* P = part + (int64_t)blockIdx.y * NC * ntarget;
#pragma unroll
  for (int k = 0; k < kTPT; ++k) {
    if (!ok[k]) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t o = (NC == 1) ? tg[k] : 3 * Di.tgt_off + (int64_t)c * Di.nt + (tg[k] - Di.tgt_off);
      P[o] = 0.07957747154594766788 * acc[k][c];
    }
  }
}

__global__ void k_reduce_parts(const double* __restrict__ part, int nsplit, int64_t n,
                               double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * n + e];
  out[e] += s;
}

// resident CTAs of the persistent pair kernel on this device
template <int KIND, int TPT>
int queue_grid() {
  static int g = 0;
  if (!g) {
    int dev = 0, nsm = 152, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pairs32_queue<KIND, TPT>, kThreads, 0) != cudaSuccess)
      per = 1;
    g = std::max(1, per) * nsm;
  }
  return g;
}

template <int KIND, int TPT>
void launch_shape(shbim_ctx* ctx, bool has_f, bool has_u, int splits, bool queue, cudaStream_t s) {
  dim3 grid((unsigned)(ctx->tiles.size() * (kMaxTPT / TPT)), splits);
  if (queue && ctx->opts.precision == SHBIM_PREC_FP32_COMP) {
    const int nunits = (int)(grid.x * grid.y);
    const int g = std::min(nunits, queue_grid<KIND, TPT>());
    k_pairs32_queue<KIND, TPT><<<g, kThreads, 0, s>>>(ctx->tiles_dev, ctx->drops_dev, ctx->n_drops, ctx->geo.tgt,
                                                       ctx->ntarget, ctx->geo.src32, ctx->nsource, ctx->dens_up32,
                                                       splits, has_f, has_u, ctx->part, nunits, ctx->pair_queue);
    return;
  }
  if (ctx->opts.precision == SHBIM_PREC_DF64 && ctx->dq_pairs && ctx->dq_scale > 0.0) {
    k_pairs_dq<KIND><<<dim3((unsigned)(ctx->tiles.size() * kMaxTPT), splits), kThreads, 0, s>>>(
        ctx->tiles_dev, ctx->drops_dev, ctx->n_drops, ctx->geo.tgt, ctx->ntarget, ctx->geo.srcq, ctx->geo.src32,
        ctx->geo.src32lo, ctx->nsource, ctx->dens_up32, ctx->dens_up32lo, splits, has_f, has_u, ctx->dq_scale,
        1.0 / ctx->dq_scale, ctx->dq_far, ctx->part);
  } else if (ctx->opts.precision == SHBIM_PREC_DF64) {
    k_pairs_df<KIND><<<dim3((unsigned)(ctx->tiles.size() * kMaxTPT), splits), kThreads, 0, s>>>(
        ctx->tiles_dev, ctx->drops_dev, ctx->n_drops, ctx->geo.tgt, ctx->ntarget, ctx->geo.src32,
        ctx->geo.src32lo, ctx->nsource, ctx->dens_up32, ctx->dens_up32lo, splits, has_f, has_u, ctx->part);
  } else if (ctx->opts.precision == SHBIM_PREC_FP32_COMP) {
    k_pairs32<KIND, TPT><<<grid, kThreads, 0, s>>>(ctx->tiles_dev, ctx->drops_dev, ctx->n_drops, ctx->geo.tgt,
                                                   ctx->ntarget, ctx->geo.src32, ctx->nsource, ctx->dens_up32,
                                                   splits, has_f, has_u, ctx->part);
  } else {
    k_pairs64<KIND, TPT><<<grid, kThreads, 0, s>>>(ctx->tiles_dev, ctx->drops_dev, ctx->n_drops, ctx->geo.tgt,
                                                   ctx->ntarget, ctx->geo.src, ctx->nsource, ctx->dens_up,
                                                   splits, has_f, has_u, ctx->part);
  }
}

template <int KIND>
void launch_raw(shbim_ctx* ctx, bool has_f, bool has_u, int tpt, int splits, bool queue, cudaStream_t s) {
  if (tpt == 4) launch_shape<KIND, 4>(ctx, has_f, has_u, splits, queue, s);
  else if (tpt == 2) launch_shape<KIND, 2>(ctx, has_f, has_u, splits, queue, s);
  else launch_shape<KIND, 1>(ctx, has_f, has_u, splits, queue, s);
}

// Choose the register blocking (targets per thread), the source-split count and the launch form
// (one CTA per work unit, or resident CTAs taking units from an atomic counter) of one FP32 kernel
// kind for this drop layout: every TPT in {1, 2, 4} with split counts in powers of two around the
// layout's default (times 1/4 ... 4, at most the partial-buffer capacity), in both forms, is
// launched twice and the second launch timed with CUDA events; the fastest is kept.
template <int KIND>
int autotune(shbim_ctx* ctx, bool has_f, bool has_u, cudaStream_t s) {
  auto& C = ctx->pair_cfg[KIND];
  C.tuned = true;
  if (ctx->timing || ctx->opts.precision != SHBIM_PREC_FP32_COMP) return SHBIM_OK;
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return SHBIM_OK;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "autotune event");
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return cuda_fail(ctx, cudaGetLastError(), "autotune event");
  }
  const int lo = std::max(1, ctx->pair_splits / 4), hi = std::min(ctx->split_max, 4 * ctx->pair_splits);
  int best_t = C.tpt, best_s = C.splits;
  bool best_q = C.queue;
  float best_ms = 1e30f;
  int sp0 = 1;
  while (2 * sp0 <= lo) sp0 *= 2;
  for (int q = 0; q < 2; ++q)
    for (int tpt = 1; tpt <= kMaxTPT; tpt *= 2) {
      for (int sp = sp0; sp <= hi; sp *= 2) {
        launch_raw<KIND>(ctx, has_f, has_u, tpt, sp, q != 0, s);  // warm
        cudaEventRecord(a, s);
        launch_raw<KIND>(ctx, has_f, has_u, tpt, sp, q != 0, s);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ctx->launches += 2;
        if (ms < best_ms) {
          best_ms = ms;
          best_t = tpt;
          best_s = sp;
          best_q = q != 0;
        }
      }
    }
  C.tpt = best_t;
  C.splits = best_s;
  C.queue = best_q;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SHBIM_OK : cuda_fail(ctx, e, "pair kernel autotune");
}

// Source splits of the FP64-class kernel: its CTAs are long (one target per thread, ~100-200 FP32
// instructions per pair), so a grid of a few waves loses much of its last wave. The smallest split count
// (at most the partial buffer's) that gives at least six waves of resident CTAs (occupancy query) is
// taken, or the largest allowed if none does; chosen once per layout and kind.
template <int KIND>
int fp64class_splits(shbim_ctx* ctx) {
  auto& C = ctx->pair_cfg[KIND];
  if (C.fp64class_splits > 0) return C.fp64class_splits;
  int dev = 0, nsm = 152, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool quant = ctx->dq_pairs && ctx->dq_scale > 0.0;
  const cudaError_t e = quant ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pairs_dq<KIND>, kThreads, 0)
                              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pairs_df<KIND>, kThreads, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    per = 1;
  }
  const int64_t resident = (int64_t)std::max(1, per) * nsm;
  const int64_t units = (int64_t)ctx->tiles.size() * kMaxTPT;
  int s = std::max(1, ctx->split_max);
  for (int k = 1; k <= ctx->split_max; ++k)
    if (units * k >= 6 * resident) {
      s = k;
      break;
    }
  C.fp64class_splits = std::max(s, std::min(ctx->pair_splits, ctx->split_max));
  return C.fp64class_splits;
}

template <int KIND>
int launch_pairs(shbim_ctx* ctx, bool has_f, bool has_u, double* out, cudaStream_t s, cudaEvent_t before_reduce) {
  constexpr int NC = stokes_kind(KIND) ? 3 : 1;
  if (ctx->n_drops < 2 || ctx->tiles.empty()) {
    if (before_reduce) SHBIM_CUDA(ctx, cudaStreamWaitEvent(s, before_reduce, 0));
    return SHBIM_OK;
  }
  auto& C = ctx->pair_cfg[KIND];
  if (!C.tuned) {
    int rc = autotune<KIND>(ctx, has_f, has_u, s);
    if (rc) return rc;
  }
  // the FP64 kernels keep the layout's default shape; the FP64-class kernel (4 CTAs per tile, one target
  // per thread) takes the split count fp64class_splits chooses for its occupancy
  const bool fp32 = ctx->opts.precision == SHBIM_PREC_FP32_COMP;
  const bool df = ctx->opts.precision == SHBIM_PREC_DF64;
  const int tpt = fp32 ? C.tpt : (df ? 1 : 2);
  const int splits = fp32 ? C.splits : (df ? fp64class_splits<KIND>(ctx) : ctx->pair_splits);
  launch_raw<KIND>(ctx, has_f, has_u, tpt, splits, fp32 && C.queue, s);
  SHBIM_CHECK_LAUNCH(ctx, "k_pairs");
  if (before_reduce) SHBIM_CUDA(ctx, cudaStreamWaitEvent(s, before_reduce, 0));
  const int64_t n = NC * ctx->ntarget;
  k_reduce_parts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(ctx->part, splits, n, out);
  SHBIM_CHECK_LAUNCH(ctx, "k_reduce_parts");
  return SHBIM_OK;
}

// Largest |x - c| (Euclidean) over the sources of every drop: one CTA row per drop; the maximum goes to
// out[drop] as the bit pattern of a non-negative float (integer order = float order), rounded up.
__global__ void k_src_extent(const double* __restrict__ src, int64_t nsource, const DropDev* __restrict__ drops,
                             unsigned* __restrict__ out) {
  const DropDev D = drops[blockIdx.y];
  float m = 0.0f;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < D.ns; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sI = D.src_off + e;
    const double dx = src[sI] - D.cx, dy = src[nsource + sI] - D.cy, dz = src[2 * nsource + sI] - D.cz;
    m = fmaxf(m, __double2float_ru(sqrt(dx * dx + dy * dy + dz * dz)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + blockIdx.y, __float_as_uint(m));
}

// v = x - c split as the multiple vq of qi = 2^-Q nearest to v and the FP32 remainder vl = v - vq
__global__ void k_quantize_src(const double* __restrict__ src, int64_t nsource, const DropDev* __restrict__ drops,
                               double qs, double qi, float* __restrict__ srcq) {
  const DropDev D = drops[blockIdx.y];
  const double c[3] = {D.cx, D.cy, D.cz};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < D.ns; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sI = D.src_off + e;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double v = src[k * nsource + sI] - c[k];
      const double h = rint(v * qs) * qi;
      srcq[k * nsource + sI] = (float)h;
      srcq[(3 + k) * nsource + sI] = (float)(v - h);
    }
  }
}

}  // namespace

int pairs_laplace(shbim_ctx* ctx, int which, double* out, cudaStream_t s, cudaEvent_t before_reduce) {
  return which == SHBIM_LAPLACE_SL ? launch_pairs<LSL>(ctx, false, false, out, s, before_reduce)
                                   : launch_pairs<LDL>(ctx, false, false, out, s, before_reduce);
}

int pairs_stokes(shbim_ctx* ctx, bool has_f, bool has_u, double* out, cudaStream_t s, cudaEvent_t before_reduce) {
  if (has_f && has_u) return launch_pairs<STO>(ctx, true, true, out, s, before_reduce);
  if (has_f) return launch_pairs<STS>(ctx, true, false, out, s, before_reduce);
  return launch_pairs<STD>(ctx, false, true, out, s, before_reduce);
}

int pairs_tile_targets() { return kTileTargets; }

// Quantum of the FP64-class pair sums for the current geometry (pair_dq.cuh) and the drop pairs that
// use it. With ext_j the largest |x - c_j| of drop j's nodes, B = max over pairs of drops of
// |c_i - c_j| (per component) + 1.01 ext_i + ext_j bounds every target offset |x0 - c_j|, every source
// offset and every difference of the two (targets lie on the degree-p grids of the same surfaces: 1 %
// is allowed for them). With Q = 23 - ceil(log2 B), B <= 2^(23-Q), so every quantised offset and every
// difference of two is an integer multiple of 2^-Q below 2^24 quanta: exact in FP32. The FP32
// remainders below the quantum are good to ~2^-(Q+23) absolute, ~2^-42 relative to r for r >= 2^(19-Q):
// the quantised form is used for drop pairs whose surfaces are at least that far apart,
// |c_i - c_j| - 1.01 ext_i - ext_j >= 2^(19-Q); closer pairs keep the general double-float form.
int build_quantized_sources(shbim_ctx* ctx, cudaStream_t s) {
  ctx->dq_scale = 0.0;
  const int nd = ctx->n_drops;
  if (nd < 2 || !ctx->geo.srcq) return SHBIM_OK;
  if (ctx->dq_cap < nd) {
    cudaFree(ctx->dq_ext_dev);
    cudaFree(ctx->dq_far);
    ctx->dq_ext_dev = nullptr;
    ctx->dq_far = nullptr;
    if (cudaMalloc(&ctx->dq_ext_dev, (size_t)nd * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&ctx->dq_far, (size_t)nd * nd) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc quantisation tables");
    ctx->dq_cap = nd;
  }
  int maxns = 0;
  for (const auto& d : ctx->drops) maxns = std::max(maxns, d.ns);
  const dim3 grid((unsigned)std::min(64, (maxns + 255) / 256), (unsigned)nd);
  SHBIM_CUDA(ctx, cudaMemsetAsync(ctx->dq_ext_dev, 0, (size_t)nd * sizeof(unsigned), s));
  k_src_extent<<<grid, 256, 0, s>>>(ctx->geo.src, ctx->nsource, ctx->drops_dev, ctx->dq_ext_dev);
  SHBIM_CHECK_LAUNCH(ctx, "k_src_extent");
  std::vector<unsigned> bits(nd);
  SHBIM_CUDA(ctx, cudaMemcpyAsync(bits.data(), ctx->dq_ext_dev, (size_t)nd * sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  SHBIM_CUDA(ctx, cudaStreamSynchronize(s));
  std::vector<double> ext(nd);
  for (int i = 0; i < nd; ++i) {
    float e;
    std::memcpy(&e, &bits[i], sizeof(e));
    ext[i] = (double)e;
  }
  double B = 0.0;
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < nd; ++j) {
      if (i == j) continue;
      double dc = 0.0;
      for (int k = 0; k < 3; ++k) dc = std::max(dc, std::fabs(ctx->drops[i].centre[k] - ctx->drops[j].centre[k]));
      B = std::max(B, dc + 1.01 * ext[i] + ext[j]);
    }
  if (!std::isfinite(B) || !(B > 0.0)) return fail(ctx, SHBIM_ERR_NONFINITE, "non-finite drop extent");
  const int Q = 23 - (int)std::ceil(std::log2(B));
  const double gap_min = std::ldexp(1.0, 19 - Q);
  std::vector<unsigned char> far((size_t)nd * nd, 0);
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j < nd; ++j) {
      if (i == j) continue;
      double d2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double dc = ctx->drops[i].centre[k] - ctx->drops[j].centre[k];
        d2 += dc * dc;
      }
      far[(size_t)i * nd + j] = std::sqrt(d2) - 1.01 * ext[i] - ext[j] >= gap_min ? 1 : 0;
    }
  SHBIM_CUDA(ctx, cudaMemcpy(ctx->dq_far, far.data(), far.size(), cudaMemcpyHostToDevice));
  ctx->dq_scale = std::ldexp(1.0, Q);
  k_quantize_src<<<grid, 256, 0, s>>>(ctx->geo.src, ctx->nsource, ctx->drops_dev, ctx->dq_scale,
                                      std::ldexp(1.0, -Q), ctx->geo.srcq);
  SHBIM_CHECK_LAUNCH(ctx, "k_quantize_src");
  ctx->launches += 2;
  return SHBIM_OK;
}


// Operations of one kernel term in the method's formulas (add or multiply 1, fused multiply-add 2,
// reciprocal square root 1), d = x0 - x: d 3, r^2 = d.d 5, 1/r 1, then
//   single layer   s (1/r) accumulated 2                                          -> 11
//   double layer   1/r^3 2, d.n0 5, s/r^3 1, times d.n0 accumulated 2             -> 19
//   Stokeslet      1/r^2 1, 1/r^3 1, d.f 5, t = d.f/r^3 1, per component f/r + d t accumulated 4 -> 29
//   stresslet      1/r^2 1, 1/r^5 2, d.u 5, d.n 5, t = (d.u)(d.n)/r^5 2, per component d t accumulated 2 -> 30
//   both           1/r^2 1, 1/r^3 1, d.f, d.u, d.n 15, t 4, per component 4       -> 42
// (the 1/(4 pi) and the stresslet's -6 (lambda - 1) are applied per target or folded into strengths)
double pairs_work(const shbim_ctx* ctx, int kind) {
  static const double kFlops[5] = {19.0, 11.0, 42.0, 29.0, 30.0};
  return kind >= 0 && kind < 5 ? kFlops[kind] * (double)ctx->cross_pairs : 0.0;
}

}  // namespace shbim
