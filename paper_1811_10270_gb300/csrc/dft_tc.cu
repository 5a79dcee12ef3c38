// Fourier stage of the analysis of the singular-row weights (Section 2.1) on the fifth-generation
// tensor cores, with FP64-class accuracy.
//
// F[r][o] = sum_k W[r][k] T[o][k], T[o][k] = cos(m phi_k) (o = m <= p) or sin(m phi_k)
// (stored row-major, or order-major F[o][r] for the tensor-core Legendre stage)
// (o = p+1+m), phi_k = 2 pi k / (2q+2): a GEMM with the row count of a chunk of weights
// (targets x 14 components x latitudes) and a fixed table. Every double-float value is split,
// after scaling by a power of two per row (per table for T), into six integer digits exactly
// representable in bfloat16: X ~ x 2^42 = sum_j d_j 128^j, balanced base 2^7 (|d_j| <= 72) with the
// top digit d_5 the rest (|d_5| <= 128; tc.cuh). The 21 digit products with
// j_a + j_b >= 5 are tensor-core GEMMs (tcgen05.mma kind::f16, bf16 x bf16 -> f32); products of
// equal j_a + j_b share one accumulator, and every accumulator sums integers below 2^24, so the
// FP32 accumulation in tensor memory is exact. The epilogue combines the six accumulators into a
// double-float. The neglected products (j_a + j_b < 5) and the rounding of the digits bound the
// error by ~2^-40 of sum_k |W[r][k] T[o][k]| (Ozaki-style error-free splitting of a matrix product;
// 2^-40.0 at worst in the host test of the degree-32 table).
//
// Work decomposition: persistent CTAs (one per SM, 16 producer warps + one MMA warp; the six
// accumulators of the 80-output tile take 480 of the SM's 512 tensor-memory columns) loop over
// tiles of 128 rows. The table's pre-laid-out digit planes (all K steps, up to 150 KB) are copied
// into shared memory once per CTA; the next tile's rows are prefetched into L2. Per tile the rows'
// scales come with the rows (or four threads per row find them), then per K step of 16 longitudes
// each producer thread turns four values (read from global memory two steps ahead) into digit
// planes in one of two shared-memory stages, and one thread of the MMA warp issues the 21 digit
// products as 9 MMAs (one row digit against up to three table digits, N <= 240) and commits them to
// the stage's mbarrier; the other stage is filled meanwhile. Every wait is bounded; a timeout sets
// the error flag and the kernel stops issuing work. Degrees with 2p + 2 <= 80 (p <= 39).
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
// K = 2q + 2 = 4(p + 1) longitudes, at most 2 kNT (2p + 2 <= kNT)
static_assert(diag_sums_exact(2 * kNT), "Fourier stage: digit sums must stay exact in FP32");
constexpr int kProducers = 512;                // digit-writing and epilogue threads (16 warps)
constexpr int kThreadsTC = kProducers + 32;    // + one warp that issues the MMAs
constexpr int kPlaneA = kMT * kKS;            // bf16 per row-digit plane (4096 B)
constexpr int kPlaneB = kNT * kKS;            // bf16 per table-digit plane (2560 B)
constexpr uint32_t kTmemCols = 512;

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(kThreadsTC, 1)
k_dft_tc(const float2* __restrict__ W, int64_t rows, int nlon, int nout, const uint4* __restrict__ tdig,
         int ksteps, const int* __restrict__ rexp, float2* __restrict__ F, int omajor, int* __restrict__ err,
         uint64_t wlim) {
  // dynamic shared memory: [the table's digit planes for every K step, resident][two stages of row
  // digit planes]
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[2];    // stage written by the 256 producers
  __shared__ __align__(8) uint64_t empty[2];   // stage's products done (tcgen05.commit)
  __shared__ __align__(8) uint64_t tbar;
  __shared__ uint32_t tmem_base;
  __shared__ int rowexp[kMT];
  __shared__ float rowmax[4][kMT];
  uint8_t* sB = smem;
  uint8_t* sA = smem + (size_t)ksteps * kDig * kPlaneB * 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool producer = tid < kProducers;
  const int64_t total = (rows + kMT - 1) / kMT;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    mbar_init(&full[0], kProducers);
    mbar_init(&full[1], kProducers);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(&tbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  // the whole table (one bulk copy), waited for once
  const uint32_t tbytes = (uint32_t)ksteps * kDig * kPlaneB * 2;
  if (tid == 0 && (int64_t)blockIdx.x < total) bulk_load(sB, tdig, tbytes, &tbar);
  bool table_ok = true;
  if ((int64_t)blockIdx.x < total) table_ok = mbar_wait(&tbar, 0, wlim);
  const uint32_t tmem = tmem_base;
  // uses of each stage so far (the same count in every thread): fill u waits for the products of
  // fill u - 1 (parity (u - 1) & 1 of `empty`), the MMA warp waits for fill u (parity u & 1 of `full`)
  uint32_t uses[2] = {0u, 0u};
  bool abort_all = __syncthreads_or(!table_ok);
  const int r_loc = tid & (kMT - 1), qt = (tid >> 7) & 3;   // row of the tile, quarter of a K step
  for (int64_t tm = blockIdx.x; tm < total && !abort_all; tm += gridDim.x) {
    const int64_t row = tm * kMT + r_loc;
    const bool rv = producer && row < rows;
    const float2* wrow = W + (rv ? row : 0) * nlon;
    // four values per K step (two per 16-byte load; nlon is a multiple of 4, so a pair lies wholly
    // inside or wholly past the row), read two steps ahead; the first two steps are requested
    // before the row scales arrive
    auto load_step = [&](int ks, float4 (&v)[2]) {
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2) {
        const int k = ks * kKS + qt * 4 + 2 * i2;
        v[i2] = (rv && ks < ksteps && k < nlon) ? *reinterpret_cast<const float4*>(wrow + k)
                                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    float4 q0[2], q1[2];
    load_step(0, q0);
    load_step(1, q1);
    // the next tile's rows start moving from HBM into L2 now
    if (tid == kProducers && tm + gridDim.x < total) {
      const int64_t r1 = (tm + gridDim.x) * kMT;
      const int64_t bytes = min((int64_t)kMT, rows - r1) * nlon * (int64_t)sizeof(float2);
      for (int64_t off = 0; off < bytes; off += 32768)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(reinterpret_cast<const char*>(W + r1 * nlon) + off),
                     "r"((uint32_t)min((int64_t)32768, bytes - off)));
    }
    // per-row power-of-two scale, max |hi| < 2^e: given by the producer of W, or four threads per
    // row scanning every fourth pair of its values each
    if (rexp) {
      if (tid < kMT) rowexp[tid] = tm * kMT + tid < rows ? rexp[tm * kMT + tid] : 0;
    } else if (producer) {
      float mx = 0.f;
      if (rv) {
#pragma unroll 4
        for (int k = 2 * qt; k < nlon; k += 8) {
          const float4 v = *reinterpret_cast<const float4*>(wrow + k);
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
        }
      }
      rowmax[qt][r_loc] = mx;
    }
    __syncthreads();
    if (!rexp && tid < kMT) {
      int e = 0;
      frexpf(fmaxf(fmaxf(rowmax[0][tid], rowmax[1][tid]), fmaxf(rowmax[2][tid], rowmax[3][tid])), &e);
      rowexp[tid] = max(e, -120);   // keeps 2^(7 - e) a normal float; smaller rows scale the same
    }
    __syncthreads();
    bool bad = false;
    if (producer) {
      const float sc = __int_as_float((127 + 7 - rowexp[r_loc]) << 23);   // 2^(7 - e), exact
      for (int ks = 0; ks < ksteps && !bad; ++ks) {
        const int st = ks & 1;
        float4 cur[2];
#pragma unroll
        for (int i2 = 0; i2 < 2; ++i2) {
          cur[i2] = q0[i2];
          q0[i2] = q1[i2];
        }
        load_step(ks + 2, q1);
        if (uses[st] > 0 && !mbar_wait(&empty[st], (uses[st] - 1) & 1, wlim)) {
          bad = true;
          break;
        }
        uint8_t* base = sA + st * (kDig * kPlaneA * 2);
        float d[kDig][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 v4 = cur[i >> 1];
          const float vh = (i & 1) ? v4.z : v4.x, vl = (i & 1) ? v4.w : v4.y;
          float dd[kDig];
          digits6(vh * sc, vl * sc, dd);
#pragma unroll
          for (int j = 0; j < kDig; ++j) d[j][i] = dd[j];
        }
        const int off = canon16(r_loc, qt * 4) * 2;   // bytes; 8-byte aligned
#pragma unroll
        for (int j = 0; j < kDig; ++j) {
          uint2 q;
          q.x = pack_bf16f(d[j][0], d[j][1]);
          q.y = pack_bf16f(d[j][2], d[j][3]);
          *reinterpret_cast<uint2*>(base + j * kPlaneA * 2 + off) = q;
        }
        // the writes become visible to the tensor cores' (async-proxy) reads, then the stage is
        // reported full
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(&full[st]);
        ++uses[st];
      }
    } else if (tid == kProducers) {
      for (int ks = 0; ks < ksteps; ++ks) {
        const int st = ks & 1;
        if (!mbar_wait(&full[st], uses[st] & 1, wlim)) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t a0 = smem_u32(sA + st * (kDig * kPlaneA * 2)), b0 = smem_u32(sB + (size_t)ks * kDig * kPlaneB * 2);
        // A digit j_a times up to three consecutive table digits j_b .. j_b + g - 1 in one MMA of
        // N = 80 g: the table's digit planes lie one after the other like the rows of one operand,
        // and their products go to the consecutive accumulators j_a + j_b - 5 .. + g - 1. The two
        // products of j_a = 5 come first and, in the first K step, overwrite all six accumulators.
#pragma unroll
        for (int ja = kDig - 1; ja >= 0; --ja)
#pragma unroll
          for (int jb0 = kDig - 1 - ja; jb0 < kDig; jb0 += 3) {
            const int g = min(3, kDig - jb0);
            const int dgl = ja + jb0 - (kDig - 1);
            const uint32_t acc = (ks > 0 || ja != kDig - 1) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(dgl * kNT), desc_k16(a0 + ja * kPlaneA * 2), desc_k16(b0 + jb0 * kPlaneB * 2),
                     idesc_bf16(kNT * g), acc);
          }
        mma_commit(&empty[st]);
        ++uses[st];
      }
    } else {
      for (int ks = 0; ks < ksteps; ++ks) ++uses[ks & 1];
    }
    if (__syncthreads_or(bad)) {
      abort_all = true;
      break;
    }
    // all products of the tile complete: the last commit covers every earlier product
    {
      const int st = (ksteps - 1) & 1;
      if (__syncthreads_or(!mbar_wait(&empty[st], (uses[st] - 1) & 1, wlim))) {
        abort_all = true;
        break;
      }
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // epilogue: warp w (< 16) reads lanes 32 (w % 4) .. +31; column blocks of 8 split among w, w+4,
    // w+8 and w+12
    if (producer) {
      const int lq = warp & 3, wq = warp >> 2;
      const int rl = 32 * lq + (tid & 31);
      const int64_t rowe = tm * kMT + rl;
      const int ee = rowexp[rl];
      for (int cb = wq; cb < (nout + 7) / 8; cb += 4) {
        uint32_t a[kDig][8];
#pragma unroll
        for (int dg = 0; dg < kDig; ++dg)
          tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dg * kNT + cb * 8), a[dg]);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = cb * 8 + j;
          if (rowe < rows && o < nout) {
            const dfl::df r = combine6(__uint_as_float(a[5][j]), __uint_as_float(a[4][j]), __uint_as_float(a[3][j]),
                                       __uint_as_float(a[2][j]), __uint_as_float(a[1][j]), __uint_as_float(a[0][j]));
            F[omajor ? (int64_t)o * rows + rowe : rowe * nout + o] = scale2(r, ee - 13);
          }
        }
      }
    }
    // the next tile's first products overwrite the accumulators only after every read
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
  }
  // let products and copies still in flight finish (bounded) before resources are released
  if (abort_all) {
    for (int st = 0; st < 2; ++st)
      if (uses[st] > 0) mbar_wait(&empty[st], (uses[st] - 1) & 1, kDrainNs);
    if (!table_ok && tid == 0) mbar_wait(&tbar, 0, kDrainNs);
    if (tid == 0) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace

int dft_tc_ksteps(int p) { return (4 * (p + 1) + kKS - 1) / kKS; }

int dft_tc_smem(int p) { return (dft_tc_ksteps(p) * kPlaneB + 2 * kPlaneA) * kDig * 2; }

// one 80-output tile (2p + 2 <= 80) with the table resident beside two row stages
bool dft_tc_fits(int p) { return 2 * (p + 1) <= kNT && dft_tc_smem(p) + 4096 <= 227 * 1024; }

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

int analysis_fourier_tc(shbim_ctx* ctx, const DegreeTables& T, const float2* W, int64_t rows, const int* rexp,
                        float2* F, cudaStream_t s, bool omajor) {
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
  if (!dft_tc_fits(p) || T.dft_ntiles != 1 || T.dft_ksteps != dft_tc_ksteps(p))
    return fail(ctx, SHBIM_ERR_ARG, "tensor-core Fourier stage: degree out of range");
  const int64_t tiles = (rows + kMT - 1) / kMT;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
  k_dft_tc<<<grid, kThreadsTC, smem, s>>>(W, rows, nlon, nout, reinterpret_cast<const uint4*>(T.dft_digits),
                                          T.dft_ksteps, rexp, F, omajor ? 1 : 0, ctx->tc_err,
                                          ctx->wait_ns);
  SHBIM_CHECK_LAUNCH(ctx, "k_dft_tc");
  return SHBIM_OK;
}

}  // namespace shbim
