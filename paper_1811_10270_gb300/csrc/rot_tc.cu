// Pole rotation of the singular-row build (Section 3.1) on the fifth-generation tensor cores, with
// FP64-class accuracy: the two products with the quarter-turn block Dq_n of every degree n are
// GEMMs of (vectors x 2n+1) by a fixed (2n+1) x (2n+1) table, split into exact bfloat16 digit
// products (tc.cuh); the z rotations between them act on the double-float values in shared memory.
//   forward (ADJ = false): out = Dq^T Dz(-theta) Dq Dz(-phi) in   (position coefficients)
//   adjoint (ADJ = true):  out = Dz(phi) Dq^T Dz(theta) Dq in     (rows, FP32 planes)
// theta, phi are the base-grid angles of each vector's target; Dz(a) turns the pair of real
// coefficients (n, m), (n, -m) by the angle m a.
//
// Work decomposition: persistent CTAs (one per SM, 256 threads, all 512 tensor-memory columns:
// six accumulators of up to 80 columns) loop over items (128 vectors, one degree), largest degree
// first. Per item: the rows' degree block is read into shared memory as double-float; for each of
// the two products the rows get a power-of-two scale, per K step of 16 their digit planes and the
// table's pre-laid-out planes (one bulk copy) fill one of two stages and one thread issues the 21
// MMAs; the epilogue combines the six accumulators in double-float back into shared memory, where
// the z rotation follows. Every wait is bounded; a timeout sets the error flag and the CTA stops.
// Degrees with 2n+1 <= 80 (p <= 39) only: larger blocks use the FP32-pipe kernel.
#include <algorithm>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "tc.cuh"

namespace shbim {

namespace {

using dfl::df;
using namespace tc;

constexpr int kThreads = 256;
constexpr int kNmax = 80;                                  // largest padded block (N and K)
constexpr int kPlaneA = kMT * kKS;                          // bf16 per row-digit plane
constexpr int kPlaneBmax = kNmax * kKS;                     // bf16 per table-digit plane
constexpr int kStageBytes = kDig * (kPlaneA + kPlaneBmax) * 2;
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ df lds(const float2* p, int i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void sts(float2* p, int i, df v) { p[i] = make_float2(v.hi, v.lo); }

__host__ __device__ inline int padded(int w) { return w <= 16 ? 16 : (w + 15) / 16 * 16; }

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, 1)
k_rotate_tc(const float2* __restrict__ vin, int64_t in_stride, int nc, int p, int t_begin, int ct, int ncomp,
            const float2* __restrict__ cs_theta, const float2* __restrict__ cs_phi, const uint4* __restrict__ tdig,
            const int* __restrict__ toff, float2* __restrict__ vout, float* __restrict__ rows_lap,
            float* __restrict__ rows_sto, int nt_drop, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t bbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int rowexp[kMT];
  __shared__ int rowlat[kMT], rowlon[kMT];
  const int WS = 2 * p + 1;   // row stride of the value block (odd: conflict-free column access)
  float2* sX = reinterpret_cast<float2*>(smem + 2 * kStageBytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nlon = 2 * p + 2;
  const int64_t nvec = (int64_t)ct * ncomp;
  const int64_t tiles_v = (nvec + kMT - 1) / kMT;
  const int64_t total = tiles_v * (p + 1);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&bbar[0], 1);
    mbar_init(&bbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base;
  uint32_t phase[2] = {0u, 0u}, bphase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool abort_all = false;
  const int r_loc = tid & (kMT - 1), half = tid >> 7;

  // z rotation of every row's degree-n block, in place: angle index from the row's target
  auto dz = [&](int n, bool theta, bool neg) {
    const int li = theta ? rowlat[r_loc] : rowlon[r_loc];
    if (li < 0) return;
    const float2* cs = (theta ? cs_theta : cs_phi) + (int64_t)li * 2 * (p + 1);
    float2* x = sX + r_loc * WS;
    for (int m = 1 + half; m <= n; m += 2) {
      const float2 c2 = cs[m], s2 = cs[p + 1 + m];
      const df ca{c2.x, c2.y};
      const df sa = neg ? df{-s2.x, -s2.y} : df{s2.x, s2.y};
      const df a = lds(x, n + m), b = lds(x, n - m);
      sts(x, n + m, dfl::sub(dfl::mul(ca, a), dfl::mul(sa, b)));
      sts(x, n - m, dfl::add(dfl::mul(sa, a), dfl::mul(ca, b)));
    }
  };

  for (int64_t item = blockIdx.x; item < total && !abort_all; item += gridDim.x) {
    const int n = p - (int)(item / tiles_v);
    const int64_t tv = item - (int64_t)(p - n) * tiles_v;
    const int w = 2 * n + 1;
    const int Np = padded(w);
    const int ksteps = Np / kKS;
    const uint32_t idesc = idesc_bf16(Np);
    // rows of the item: vector v = (chunk-local target b, component c)
    if (tid < kMT) {
      const int64_t v = tv * kMT + tid;
      if (v < nvec) {
        const int tl = t_begin + (int)(v / ncomp);
        rowlat[tid] = tl / nlon;
        rowlon[tid] = tl - (tl / nlon) * nlon;
      } else {
        rowlat[tid] = rowlon[tid] = -1;
      }
    }
    // the degree block of every row (warp per row, lanes along the block: coalesced)
    for (int r = warp; r < kMT; r += kThreads / 32) {
      const int64_t v = tv * kMT + r;
      if (v < nvec) {
        const int64_t b = v / ncomp, c = v - b * ncomp;
        const float2* src = vin + b * in_stride + c * nc + (int64_t)n * n;
        for (int k = lane; k < w; k += 32) sX[r * WS + k] = src[k];
      } else {
        for (int k = lane; k < w; k += 32) sX[r * WS + k] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    if (!ADJ) {
      dz(n, false, true);
      __syncthreads();
    }
    for (int g = 0; g < 2 && !abort_all; ++g) {
      // per-row power-of-two scale, max |hi| < 2^e: warp w scans rows 16 w .. 16 w + 15
      for (int rr = 0; rr < kMT / (kThreads / 32); ++rr) {
        const int rl = warp * (kMT / (kThreads / 32)) + rr;
        float mx = 0.f;
        for (int k = lane; k < w; k += 32) mx = fmaxf(mx, fabsf(sX[rl * WS + k].x));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
          int e = 0;
          frexpf(mx, &e);
          rowexp[rl] = max(e, -120);
        }
      }
      __syncthreads();
      const int e_r = rowexp[r_loc];
      const float2* xrow = sX + r_loc * WS;
      const uint4* tab = tdig + toff[g * (p + 1) + n];
      const uint32_t bbytes = (uint32_t)(kDig * Np * kKS * 2);
      for (int ks = 0; ks < ksteps; ++ks) {
        const int st = ks & 1;
        if (pending[st]) {
          const bool ok = mbar_wait(&mbar[st], phase[st]);
          phase[st] ^= 1u;
          pending[st] = false;
          if (__syncthreads_or(!ok)) {
            abort_all = true;
            break;
          }
        }
        uint8_t* base = smem + st * kStageBytes;
        if (tid == 0) bulk_load(base + kDig * kPlaneA * 2, tab + (int64_t)ks * (bbytes / 16), bbytes, &bbar[st]);
        {
          const float sc = __int_as_float((127 + 7 - e_r) << 23);   // 2^(7 - e), exact
          float d[kDig][8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int k = ks * kKS + half * 8 + i;
            const float2 v = k < w ? xrow[k] : make_float2(0.f, 0.f);
            float yh = v.x * sc, yl = v.y * sc;
#pragma unroll
            for (int j = kDig - 1; j >= 0; --j) {
              const float dj = rintf(yh);
              d[j][i] = dj;
              const df r = dfl::two_sum(dfl::sub_rn(yh, dj), yl);
              yh = r.hi * 128.f;
              yl = r.lo * 128.f;
            }
          }
          const int off = canon16(r_loc, half * 8) * 2;
#pragma unroll
          for (int j = 0; j < kDig; ++j) {
            uint4 q;
            q.x = pack_bf16f(d[j][0], d[j][1]);
            q.y = pack_bf16f(d[j][2], d[j][3]);
            q.z = pack_bf16f(d[j][4], d[j][5]);
            q.w = pack_bf16f(d[j][6], d[j][7]);
            *reinterpret_cast<uint4*>(base + j * kPlaneA * 2 + off) = q;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;\n");
        __syncthreads();
        if (tid == 0) {
          if (!mbar_wait(&bbar[st], bphase[st])) atomicExch(err, 1);
          asm volatile("tcgen05.fence::after_thread_sync;\n");
          const uint32_t a0 = smem_u32(base), b0 = smem_u32(base + kDig * kPlaneA * 2);
#pragma unroll
          for (int ja = 0; ja < kDig; ++ja)
#pragma unroll
            for (int jb = 0; jb < kDig; ++jb) {
              if (ja + jb < kDig - 1) continue;
              const int dgl = ja + jb - (kDig - 1);
              const uint32_t acc = (ks > 0 || jb != kDig - 1) ? 1u : 0u;
              mma_bf16(tmem + (uint32_t)(dgl * Np), desc_k16(a0 + ja * kPlaneA * 2),
                       desc_k16(b0 + jb * Np * kKS * 2), idesc, acc);
            }
          mma_commit(&mbar[st]);
        }
        bphase[st] ^= 1u;
        pending[st] = true;
      }
      if (abort_all) break;
      bool ok = true;
      for (int st = 0; st < 2; ++st)
        if (pending[st]) {
          ok = ok && mbar_wait(&mbar[st], phase[st]);
          phase[st] ^= 1u;
          pending[st] = false;
        }
      if (__syncthreads_or(!ok)) {
        abort_all = true;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      // epilogue: warp w reads lanes 32 (w % 4) .. +31; column blocks of 16 split between w and w+4
      {
        const int lq = warp & 3, wh = warp >> 2;
        const int rl = 32 * lq + lane;
        const int ee = rowexp[rl];
        for (int cb = wh; cb < Np / 16; cb += 2) {
          uint32_t a[kDig][16];
#pragma unroll
          for (int dg = 0; dg < kDig; ++dg)
            tmem_ld16(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dg * Np + cb * 16), a[dg]);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            df r{__uint_as_float(a[kDig - 1][j]), 0.f};
            float wt = 1.f;
#pragma unroll
            for (int dg = kDig - 2; dg >= 0; --dg) {
              wt *= 0.0078125f;   // 2^-7
              r = dfl::add_f(r, __uint_as_float(a[dg][j]) * wt);
            }
            const int o = cb * 16 + j;
            if (o < w) sX[rl * WS + o] = make_float2(ldexpf(r.hi, ee - 13), ldexpf(r.lo, ee - 13));
          }
        }
      }
      // the next products overwrite the accumulators only after every read
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      if (g == 0) {
        dz(n, true, !ADJ);
        __syncthreads();
      } else if (ADJ) {
        dz(n, false, false);
        __syncthreads();
      }
    }
    if (abort_all) break;
    // store (warp per row, lanes along the block)
    for (int r = warp; r < kMT; r += kThreads / 32) {
      const int64_t v = tv * kMT + r;
      if (v >= nvec) continue;
      const int64_t b = v / ncomp;
      const int c = (int)(v - b * ncomp);
      if (!ADJ) {
        float2* dst = vout + (b * ncomp + c) * nc + (int64_t)n * n;
        for (int k = lane; k < w; k += 32) dst[k] = sX[r * WS + k];
      } else {
        const int64_t tl = t_begin + b;
        float* dst = c < kNumLap ? rows_lap + (tl * kNumLap + c) * nc : rows_sto + (tl * kNumSto + (c - kNumLap)) * nc;
        const int64_t plane = (int64_t)nt_drop * (c < kNumLap ? kNumLap : kNumSto) * nc;
        for (int k = lane; k < w; k += 32) {
          const float2 x = sX[r * WS + k];
          dst[n * n + k] = x.x;
          dst[plane + n * n + k] = x.y;
        }
      }
    }
    __syncthreads();
  }
  if (abort_all) {
    for (int st = 0; st < 2; ++st)
      if (pending[st]) mbar_wait(&mbar[st], phase[st]);
    if (tid == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

int rot_tc_smem(int p) { return 2 * kStageBytes + kMT * (2 * p + 1) * (int)sizeof(float2); }

}  // namespace

bool rot_tc_fits(int p) { return padded(2 * p + 1) <= kNmax && rot_tc_smem(p) + 4096 <= 227 * 1024; }

// Digit planes of Dq_n (g = 0, B[m][k] = Dq_n[m][k]) and its transpose (g = 1) for every degree:
// [g][n][K step][digit][Np x 16, K-major canonical], offsets in 16-byte units per (g, n).
int rot_tc_digits(shbim_ctx* ctx, int p, const std::vector<double>& D, DegreeTables& T) {
  if (!rot_tc_fits(p)) return SHBIM_OK;
  std::vector<int> off(2 * (p + 1));
  size_t total = 0;
  for (int g = 0; g < 2; ++g)
    for (int n = 0; n <= p; ++n) {
      off[g * (p + 1) + n] = (int)(total / 8);   // uint16 -> 16-byte units
      const int Np = padded(2 * n + 1);
      total += (size_t)(Np / kKS) * kDig * Np * kKS;
    }
  std::vector<uint16_t> h(total, 0);
  for (int g = 0; g < 2; ++g)
    for (int n = 0; n <= p; ++n) {
      const int w = 2 * n + 1, Np = padded(w), o = T.dq_off[n];
      uint16_t* dst = h.data() + (size_t)off[g * (p + 1) + n] * 8;
      for (int ks = 0; ks < Np / kKS; ++ks)
        for (int m = 0; m < Np; ++m)
          for (int kk = 0; kk < kKS; ++kk) {
            const int k = ks * kKS + kk;
            double v = 0.0;
            if (m < w && k < w) v = g == 0 ? D[o + (size_t)m * w + k] : D[o + (size_t)k * w + m];
            int dg[kDig];
            digits_host(v, 1, dg);   // |Dq| <= 1 < 2^1
            for (int j = 0; j < kDig; ++j)
              dst[((size_t)ks * kDig + j) * Np * kKS + canon16(m, kk)] = bf16_int(dg[j]);
          }
    }
  if (cudaMalloc(&T.rot_digits, h.size() * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&T.rot_toff, off.size() * sizeof(int)) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc rotation digit table");
  if (cudaMemcpy(T.rot_digits, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.rot_toff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_CUDA, "cudaMemcpy rotation digit table");
  return SHBIM_OK;
}

int rotate_tc(shbim_ctx* ctx, const DegreeTables& T, bool adjoint, const float2* vin, int64_t in_stride, int nc,
              int t_begin, int ct, int ncomp, float2* vout, float* rows_lap, float* rows_sto, int nt_drop,
              cudaStream_t s) {
  if (ct <= 0) return SHBIM_OK;
  if (!T.rot_digits) return fail(ctx, SHBIM_ERR_ARG, "rotation digit table missing");
  if (!ctx->tc_err) {
    if (cudaMalloc(&ctx->tc_err, sizeof(int)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc tensor-core error flag");
    SHBIM_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s));
  }
  const int p = T.p;
  const int smem = rot_tc_smem(p);
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t items = (((int64_t)ct * ncomp + kMT - 1) / kMT) * (p + 1);
  const unsigned grid = (unsigned)std::min<int64_t>(items, nsm);
  const uint4* tdig = reinterpret_cast<const uint4*>(T.rot_digits);
  if (adjoint) {
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rotate_tc<true><<<grid, kThreads, smem, s>>>(vin, in_stride, nc, p, t_begin, ct, ncomp, T.cs_theta_df,
                                                   T.cs_phi_df, tdig, T.rot_toff, vout, rows_lap, rows_sto, nt_drop,
                                                   ctx->tc_err);
  } else {
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rotate_tc<false><<<grid, kThreads, smem, s>>>(vin, in_stride, nc, p, t_begin, ct, ncomp, T.cs_theta_df,
                                                    T.cs_phi_df, tdig, T.rot_toff, vout, rows_lap, rows_sto, nt_drop,
                                                    ctx->tc_err);
  }
  SHBIM_CHECK_LAUNCH(ctx, "k_rotate_tc");
  return SHBIM_OK;
}

}  // namespace shbim
