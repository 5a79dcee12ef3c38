// Fourier stage of the analysis of the singular-row weights (Section 3.1) on the fifth-generation
// tensor cores, with FP64-class accuracy.
//
// F[r][o] = sum_k W[r][k] T[o][k], T[o][k] = cos(m phi_k) (o = m <= p) or sin(m phi_k)
// (o = p+1+m), phi_k = 2 pi k / (2q+2): a GEMM with the row count of a chunk of weights
// (targets x 14 components x latitudes) and a fixed table. Every double-float value is split,
// after scaling by a power of two per row (per table for T), into six integer digits exactly
// representable in bfloat16: X ~ x 2^42 = sum_j d_j 128^j, balanced base 2^7 (|d_j| <= 72) with the
// top digit d_5 the rest (|d_5| <= 128; tc.cuh). The 21 digit products with
// j_a + j_b >= 5 are tensor-core GEMMs (tcgen05.mma kind::f16, bf16 x bf16 -> f32); products of
// equal j_a + j_b share one accumulator, and every accumulator sums integers below 2^24, so the
// FP32 accumulation in tensor memory is exact. The epilogue combines the six accumulators into a
// double-float. The neglected products (j_a + j_b < 5) and the rounding of the digits bound the
// error by ~2^-42 of sum_k |W[r][k]| (Ozaki-style error-free splitting of a matrix product).
//
// Work decomposition: persistent CTAs (one per SM, 256 threads; the six accumulators of an
// 80-column tile take 480 of the SM's 512 tensor-memory columns) loop over tiles of 128 rows x 80
// outputs. Per K step of 16 longitudes the threads write the rows' digit planes into one of two
// shared-memory stages (two threads per row, eight values each), copy the table's pre-laid-out
// digit planes, and one thread issues the 21 MMAs and commits them to the stage's mbarrier; the
// other stage is filled meanwhile. Every wait is bounded; a timeout sets the error flag and the
// kernel stops issuing work.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "tc.cuh"

namespace shbim {

namespace {

using namespace tc;

constexpr int kNT = 80;                       // outputs per tile (MMA N)
constexpr int kThreadsTC = 256;
constexpr int kPlaneA = kMT * kKS;            // bf16 per row-digit plane (4096 B)
constexpr int kPlaneB = kNT * kKS;            // bf16 per table-digit plane (2560 B)
constexpr int kStageBytes = kDig * (kPlaneA + kPlaneB) * 2;
constexpr uint32_t kTmemCols = 512;

__global__ void __launch_bounds__(kThreadsTC, 1)
k_dft_tc(const float2* __restrict__ W, int64_t rows, int nlon, int nout, const uint4* __restrict__ tdig,
         int ntiles_n, int ksteps, float2* __restrict__ F, int* __restrict__ err) {
  // dynamic shared memory: [two MMA stages][the current 128-row tile of W, rows contiguous]
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t tbar;
  __shared__ __align__(8) uint64_t bbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int rowexp[kMT];
  const float2* tileb = reinterpret_cast<const float2*>(smem + 2 * kStageBytes);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t tiles_m = (rows + kMT - 1) / kMT;
  const int64_t total = tiles_m * ntiles_n;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&tbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&bbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&bbar[1])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  // the first tile's rows: one bulk (TMA) copy of contiguous memory
  auto issue_tile = [&](int64_t tile) {
    const int64_t r0 = (tile / ntiles_n) * kMT;
    const int64_t nr = min((int64_t)kMT, rows - r0);
    bulk_load(smem + 2 * kStageBytes, W + r0 * nlon, (uint32_t)(nr * nlon * sizeof(float2)), &tbar);
  };
  if (tid == 0 && (int64_t)blockIdx.x < total) issue_tile(blockIdx.x);
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNT >> 3) << 17) | ((uint32_t)(kMT >> 4) << 24);
  uint32_t phase[2] = {0u, 0u}, tphase = 0u, bphase[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool tile_pending = (int64_t)blockIdx.x < total;
  bool abort_all = false;
  const int r_loc = tid & (kMT - 1), half = tid >> 7;
  for (int64_t tile = blockIdx.x; tile < total && !abort_all; tile += gridDim.x) {
    const int64_t tm = tile / ntiles_n;
    const int tn = (int)(tile - tm * ntiles_n);
    {
      const bool ok = mbar_wait(&tbar, tphase);
      tphase ^= 1u;
      tile_pending = false;
      if (__syncthreads_or(!ok)) {
        abort_all = true;
        break;
      }
    }
    // per-row power-of-two scale, max |hi| < 2^e: warp w scans rows 16 w .. 16 w + 15 (four rows'
    // reductions interleaved)
#pragma unroll 4
    for (int rr = 0; rr < kMT / (kThreadsTC / 32); ++rr) {
      const int rl = warp * (kMT / (kThreadsTC / 32)) + rr;
      float mx = 0.f;
      if (tm * kMT + rl < rows)
        for (int k = tid & 31; k < nlon; k += 32) mx = fmaxf(mx, fabsf(tileb[rl * nlon + k].x));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if ((tid & 31) == 0) {
        int e = 0;
        frexpf(mx, &e);
        rowexp[rl] = max(e, -120);   // keeps 2^(7 - e) a normal float; smaller rows scale the same
      }
    }
    __syncthreads();
    const int e_r = rowexp[r_loc];
    const bool rv = tm * kMT + r_loc < rows;
    const float2* wrow = tileb + r_loc * nlon;
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
      // table digits of this (n tile, K step): a bulk copy of the pre-laid-out planes, in flight
      // while the row digits are formed
      if (tid == 0)
        bulk_load(base + kDig * kPlaneA * 2, tdig + ((int64_t)tn * ksteps + ks) * (kDig * kPlaneB / 8),
                  (uint32_t)(kDig * kPlaneB * 2), &bbar[st]);
      // row digits, top down in FP32: y = x 2^(7 - e); d = rint(y.hi); y = (y - d) 128 with the
      // residual kept exactly as a double-float; d_5 (|d_5| <= 128) .. d_0 (|d_j| <= 64)
      {
        const float sc = __int_as_float((127 + 7 - e_r) << 23);   // 2^(7 - e), exact
        float d[kDig][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = ks * kKS + half * 8 + i;
          const float2 v = (rv && k < nlon) ? wrow[k] : make_float2(0.f, 0.f);
          float dd[kDig];
          digits6(v.x * sc, v.y * sc, dd);
#pragma unroll
          for (int j = 0; j < kDig; ++j) d[j][i] = dd[j];
        }
        const int off = canon16(r_loc, half * 8) * 2;   // bytes; 16-byte aligned
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
        // the table planes have landed (bounded; on expiry the products are skipped and the
        // caller sees the error flag)
        if (!mbar_wait(&bbar[st], bphase[st])) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t a0 = smem_u32(base), b0 = smem_u32(base + kDig * kPlaneA * 2);
#pragma unroll
        for (int ja = 0; ja < kDig; ++ja)
#pragma unroll
          for (int jb = 0; jb < kDig; ++jb) {
            if (ja + jb < kDig - 1) continue;
            const int dgl = ja + jb - (kDig - 1);
            // the first product of each diagonal (j_b = 5 in this loop order) in the first K step
            // overwrites the accumulator
            const uint32_t acc = (ks > 0 || jb != kDig - 1) ? 1u : 0u;
            const uint64_t da = desc_k16(a0 + ja * kPlaneA * 2);
            const uint64_t db = desc_k16(b0 + jb * kPlaneB * 2);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(dgl * kNT)),
                "l"(da), "l"(db), "r"(idesc), "r"(acc));
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(&mbar[st])));
      }
      bphase[st] ^= 1u;
      pending[st] = true;
    }
    if (abort_all) break;
    // every thread is done with this tile's rows: the next tile's copy overlaps the epilogue
    __syncthreads();
    if (tile + gridDim.x < total) {
      tile_pending = true;
      if (tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;\n");
        issue_tile(tile + gridDim.x);
      }
    }
    // all products of the tile complete
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
    const int lq = warp & 3, wh = warp >> 2;
    const int rl = 32 * lq + (tid & 31);
    const int64_t rowe = tm * kMT + rl;
    const int ee = rowexp[rl];
    for (int cb = wh; cb < kNT / 16; cb += 2) {
      uint32_t a[kDig][16];
#pragma unroll
      for (int dg = 0; dg < kDig; ++dg) {
        const uint32_t addr = tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dg * kNT + cb * 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(a[dg][0]), "=r"(a[dg][1]), "=r"(a[dg][2]), "=r"(a[dg][3]), "=r"(a[dg][4]), "=r"(a[dg][5]),
              "=r"(a[dg][6]), "=r"(a[dg][7]), "=r"(a[dg][8]), "=r"(a[dg][9]), "=r"(a[dg][10]), "=r"(a[dg][11]),
              "=r"(a[dg][12]), "=r"(a[dg][13]), "=r"(a[dg][14]), "=r"(a[dg][15])
            : "r"(addr));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const dfl::df r = combine6(__uint_as_float(a[5][j]), __uint_as_float(a[4][j]), __uint_as_float(a[3][j]),
                                   __uint_as_float(a[2][j]), __uint_as_float(a[1][j]), __uint_as_float(a[0][j]));
        const int o = tn * kNT + cb * 16 + j;
        if (rowe < rows && o < nout) F[rowe * nout + o] = scale2(r, ee - 13);
      }
    }
    // the next tile's first products overwrite the accumulators only after every read
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
  }
  if (abort_all) {
    // let products and copies still in flight finish (bounded) before resources are released
    for (int st = 0; st < 2; ++st)
      if (pending[st]) mbar_wait(&mbar[st], phase[st]);
    if (tile_pending) mbar_wait(&tbar, tphase);
    if (tid == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

int dft_tc_smem(int p) { return 2 * kStageBytes + kMT * 4 * (p + 1) * (int)sizeof(float2); }

bool dft_tc_fits(int p) { return dft_tc_smem(p) + 4096 <= 227 * 1024; }

int dft_tc_digits(shbim_ctx* ctx, int p, DegreeTables& T) {
  const int nlon = 4 * (p + 1), nout = 2 * (p + 1);
  const int ntiles = (nout + kNT - 1) / kNT, ksteps = (nlon + kKS - 1) / kKS;
  std::vector<uint16_t> h((size_t)ntiles * ksteps * kDig * kPlaneB, 0);
  for (int tn = 0; tn < ntiles; ++tn)
    for (int ks = 0; ks < ksteps; ++ks)
      for (int n = 0; n < kNT; ++n)
        for (int kk = 0; kk < kKS; ++kk) {
          const int o = tn * kNT + n, k = ks * kKS + kk;
          double v = 0.0;
          if (o < nout && k < nlon) {
            const int m = o % (p + 1);
            const double a = 2.0 * kPi * (double)((int64_t)m * k % nlon) / nlon;
            v = o <= p ? std::cos(a) : std::sin(a);
          }
          int d[kDig];
          digits_host(v, 1, d);   // |T| <= 1 < 2^1
          for (int j = 0; j < kDig; ++j)
            h[(((size_t)tn * ksteps + ks) * kDig + j) * kPlaneB + canon16(n, kk)] = bf16_int(d[j]);
        }
  cudaError_t e = cudaMalloc(&T.dft_digits, h.size() * sizeof(uint16_t));
  if (e != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc DFT digit table");
  e = cudaMemcpy(T.dft_digits, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy DFT digit table");
  T.dft_ntiles = ntiles;
  T.dft_ksteps = ksteps;
  return SHBIM_OK;
}

int analysis_fourier_tc(shbim_ctx* ctx, const DegreeTables& T, const float2* W, int64_t rows, float2* F,
                        cudaStream_t s) {
  if (rows <= 0) return SHBIM_OK;
  if (!ctx->tc_err) {
    if (cudaMalloc(&ctx->tc_err, sizeof(int)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc tensor-core error flag");
    SHBIM_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s));
  }
  const int p = T.p, nlon = 4 * (p + 1), nout = 2 * (p + 1);
  const int smem = dft_tc_smem(p);
  SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_dft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tiles = ((rows + kMT - 1) / kMT) * T.dft_ntiles;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
  k_dft_tc<<<grid, kThreadsTC, smem, s>>>(W, rows, nlon, nout, reinterpret_cast<const uint4*>(T.dft_digits),
                                          T.dft_ntiles, T.dft_ksteps, F, ctx->tc_err);
  SHBIM_CHECK_LAUNCH(ctx, "k_dft_tc");
  return SHBIM_OK;
}

}  // namespace shbim
