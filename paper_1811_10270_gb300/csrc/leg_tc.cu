// Legendre stage of the analysis of the singular-row weights (Section 2.1) on the fifth-generation
// tensor cores, with FP64-class accuracy:
//   v[item][n^2 + n +- m] = s_m sum_j F[(cs, m)][item][j] Pbar_n^m(t_j),   s_0 = 1, s_m = sqrt(2),
// the cosine part (cs = 0) giving order +m and the sine part (cs = 1) order -m. For one (cs, m) it
// is a GEMM of the items' latitude rows (the Fourier stage's output, order-major) by the fixed
// table Pbar_n^m(t_j), n = m .. p; both are split into six bfloat16 digits (tc.cuh), the table per
// row n after its own power-of-two scale.
//
// Work decomposition: persistent CTAs (one per SM, eight producer warps and one MMA warp, as in
// the Fourier stage) take contiguous ranges of work items (cs, m, 128 items) ordered by m, so the
// table of one m (at most 5 K steps x 6 digits x 48 x 16 bfloat16, 46 KB) is loaded once per CTA
// and order. Per item: the next item's rows are prefetched into L2, two threads per row find the
// row's scale, the rows are read two K steps ahead; per K step of 16 latitudes the producers
// write the rows' digit planes into one of two stages and the MMA warp issues the 21
// MMAs; the epilogue combines the six accumulators and scatters the outputs into the coefficient
// rows. Every wait is bounded; a timeout sets the error flag and the CTA stops. p <= 39.
#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"
#include "tc.cuh"

namespace shbim {

namespace {

using dfl::df;
using namespace tc;

constexpr int kProducers = 256;
constexpr int kThreads = kProducers + 32;
constexpr int kNmax = 48;                      // largest padded table height (p + 1 <= 40)
constexpr int kKmax = 80;                      // latitudes q + 1 = 2p + 2 <= 80
static_assert(diag_sums_exact(kKmax), "Legendre stage: digit sums must stay exact in FP32");
constexpr int kPlaneA = kMT * kKS;
constexpr int kPlaneBmax = kNmax * kKS;
constexpr uint32_t kTmemCols = 512;

__host__ __device__ inline int padded16(int w) { return w <= 16 ? 16 : (w + 15) / 16 * 16; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// work item it -> (m, cs, tile); the sine part of m = 0 does not exist
struct LegItems {
  int p, tiles;
  int64_t total;
  __host__ __device__ LegItems(int p_, int64_t nitems) : p(p_) {
    tiles = (int)((nitems + kMT - 1) / kMT);
    total = (int64_t)(2 * (p + 1) - 1) * tiles;
  }
  __device__ void decode(int64_t it, int& m, int& cs, int& tile) const {
    const int u = (int)(it / tiles);   // 0: (m 0, cos); 2m - 1, 2m: (m, cos), (m, sin)
    tile = (int)(it - (int64_t)u * tiles);
    m = (u + 1) >> 1;
    cs = (u == 0) ? 0 : ((u - 1) & 1);
  }
};

__global__ void __launch_bounds__(kThreads, 1)
k_leg_tc(const float2* __restrict__ FT, int64_t nitems, int p, const uint4* __restrict__ tdig,
         const int* __restrict__ toff, const signed char* __restrict__ texp, float2* __restrict__ coef,
         int64_t coef_stride, int* __restrict__ err, uint64_t wlim) {
  // dynamic shared memory: [the current order's table planes][two stages of row digit planes]
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[2];
  __shared__ __align__(8) uint64_t empty[2];
  __shared__ __align__(8) uint64_t tbar;
  __shared__ uint32_t tmem_base;
  __shared__ int rowexp[kMT];
  __shared__ float rowmax[2][kMT];
  __shared__ int colexp[kNmax];
  const int K = 2 * p + 2;                       // latitudes of the degree 2p + 1 grid
  const int ksteps = (K + kKS - 1) / kKS;
  const int P1 = p + 1;
  uint8_t* sB = smem;
  uint8_t* sA = smem + (size_t)ksteps * kDig * kPlaneBmax * 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const bool producer = tid < kProducers;
  const LegItems I(p, nitems);
  const int64_t per = (I.total + gridDim.x - 1) / gridDim.x;
  const int64_t it0 = (int64_t)blockIdx.x * per, it1 = min(I.total, it0 + per);
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
  const uint32_t tmem = tmem_base;
  uint32_t uses[2] = {0u, 0u};
  uint32_t tphase = 0u;
  bool tpend = false;        // a table copy issued and not yet waited for (MMA thread)
  int cur_m = -1;
  bool abort_all = false;
  const int r_loc = tid & (kMT - 1), half = (tid >> 7) & 1;
  const int64_t nrowsF = nitems * K;             // rows of one (cs, m) slice of F
  for (int64_t it = it0; it < it1 && !abort_all; ++it) {
    int m, cs, tile;
    I.decode(it, m, cs, tile);
    const int Nm = P1 - m, Np = padded16(Nm);
    const uint32_t idesc = idesc_bf16(Np);
    const int64_t item = (int64_t)tile * kMT + r_loc;
    const bool rv = producer && item < nitems;
    const float2* arow = FT + ((int64_t)(cs * P1 + m) * nrowsF + (rv ? item : 0) * K);
    // a new order: its table (after every product of the previous one has completed, which the
    // previous item's epilogue waited for) and its row exponents
    if (m != cur_m) {
      if (tid == kProducers) {
        const uint32_t bytes = (uint32_t)(ksteps * kDig * Np * kKS * 2);
        bulk_load(sB, tdig + toff[m], bytes, &tbar);
        tpend = true;
      }
      if (tid < Nm) colexp[tid] = texp[m * P1 + tid];
      cur_m = m;
    }
    // the next item's rows start moving into L2; this item's first two K steps are requested
    if (tid == kProducers && it + 1 < it1) {
      int m2, cs2, tile2;
      I.decode(it + 1, m2, cs2, tile2);
      const float2* nrow = FT + ((int64_t)(cs2 * P1 + m2) * nrowsF + (int64_t)tile2 * kMT * K);
      const int64_t bytes = min((int64_t)kMT, nitems - (int64_t)tile2 * kMT) * K * (int64_t)sizeof(float2);
      for (int64_t off = 0; off < bytes; off += 32768)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(reinterpret_cast<const char*>(nrow) + off),
                     "r"((uint32_t)min((int64_t)32768, bytes - off)));
    }
    auto load_step = [&](int ks, float2 (&v)[8]) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = ks * kKS + half * 8 + i;
        v[i] = (rv && ks < ksteps && k < K) ? arow[k] : make_float2(0.f, 0.f);
      }
    };
    float2 q0[8], q1[8];
    load_step(0, q0);
    load_step(1, q1);
    // per-row power-of-two scale, max |hi| < 2^e: two threads per row, each an even-length part
    // (K is even; both parts start at an even index, so every 16-byte load is aligned)
    if (producer) {
      float mx = 0.f;
      if (rv) {
        const int split = (K >> 1) & ~1;
        const int k0 = half ? split : 0, k1 = half ? K : split;
        for (int k = k0; k < k1; k += 2) {
          const float4 v = *reinterpret_cast<const float4*>(arow + k);
          mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
        }
      }
      rowmax[half][r_loc] = mx;
    }
    __syncthreads();
    if (tid < kMT) {
      int e = 0;
      frexpf(fmaxf(rowmax[0][tid], rowmax[1][tid]), &e);
      rowexp[tid] = max(e, -120);
    }
    __syncthreads();
    bool bad = false;
    if (producer) {
      const float sc = __int_as_float((127 + 7 - rowexp[r_loc]) << 23);
      for (int ks = 0; ks < ksteps && !bad; ++ks) {
        const int st = ks & 1;
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          v[i] = q0[i];
          q0[i] = q1[i];
        }
        load_step(ks + 2, q1);
        if (uses[st] > 0 && !mbar_wait(&empty[st], (uses[st] - 1) & 1, wlim)) {
          bad = true;
          break;
        }
        uint8_t* base = sA + st * (kDig * kPlaneA * 2);
        float d[kDig][8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          float dd[kDig];
          digits6(v[i].x * sc, v[i].y * sc, dd);
#pragma unroll
          for (int j = 0; j < kDig; ++j) d[j][i] = dd[j];
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
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive(&full[st]);
        ++uses[st];
      }
    } else if (tid == kProducers) {
      if (tpend) {
        if (!mbar_wait(&tbar, tphase, wlim)) bad = true;
        tphase ^= 1u;
        tpend = false;
      }
      for (int ks = 0; ks < ksteps && !bad; ++ks) {
        const int st = ks & 1;
        if (!mbar_wait(&full[st], uses[st] & 1, wlim)) {
          bad = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t a0 = smem_u32(sA + st * (kDig * kPlaneA * 2)), b0 = smem_u32(sB + (size_t)ks * kDig * Np * kKS * 2);
#pragma unroll
        for (int ja = 0; ja < kDig; ++ja)
#pragma unroll
          for (int jb = 0; jb < kDig; ++jb) {
            if (ja + jb < kDig - 1) continue;
            const int dgl = ja + jb - (kDig - 1);
            const uint32_t acc = (ks > 0 || jb != kDig - 1) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(dgl * Np), desc_k16(a0 + ja * kPlaneA * 2), desc_k16(b0 + jb * Np * kKS * 2),
                     idesc, acc);
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
    {
      const int st = (ksteps - 1) & 1;
      if (__syncthreads_or(!mbar_wait(&empty[st], (uses[st] - 1) & 1, wlim))) {
        abort_all = true;
        break;
      }
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // epilogue: warp w (< 8) reads lanes 32 (w % 4) .. +31; column blocks of 16 split between w and w+4
    if (producer) {
      const int lq = warp & 3, wh = warp >> 2;
      const int rl = 32 * lq + (tid & 31);
      const int64_t ie = (int64_t)tile * kMT + rl;
      const int ee = rowexp[rl];
      const df s2 = m == 0 ? df{1.f, 0.f} : df{1.41421353816986084f, 2.4203234971764687e-08f};   // sqrt 2
      float2* crow = coef + (ie < nitems ? ie : 0) * coef_stride;
      for (int cb = wh; cb < Np / 16; cb += 2) {
        uint32_t a[kDig][16];
#pragma unroll
        for (int dg = 0; dg < kDig; ++dg)
          tmem_ld16(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dg * Np + cb * 16), a[dg]);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int nn = cb * 16 + j;   // n - m
          if (ie < nitems && nn < Nm) {
            const df r = combine6(__uint_as_float(a[5][j]), __uint_as_float(a[4][j]), __uint_as_float(a[3][j]),
                                  __uint_as_float(a[2][j]), __uint_as_float(a[1][j]), __uint_as_float(a[0][j]));
            const float2 v = scale2(r, ee + colexp[nn] - 14);
            const df o = dfl::mul(df{v.x, v.y}, s2);
            const int n = m + nn;
            crow[n * n + n + (cs ? -m : m)] = make_float2(o.hi, o.lo);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
  }
  if (abort_all) {
    for (int st = 0; st < 2; ++st)
      if (uses[st] > 0) mbar_wait(&empty[st], (uses[st] - 1) & 1, kDrainNs);
    if (tid == 0) atomicExch(err, 1);
  }
  if (tpend && tid == kProducers) mbar_wait(&tbar, tphase, kDrainNs);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

int leg_tc_smem(int p) {
  const int ksteps = (2 * p + 2 + kKS - 1) / kKS;
  return (ksteps * kPlaneBmax + 2 * kPlaneA) * kDig * 2;
}

}  // namespace

bool leg_tc_fits(int p) { return p + 1 <= kNmax && 2 * p + 2 <= kKmax && leg_tc_smem(p) + 4096 <= 227 * 1024; }

// Digit planes of Pbar_n^m(t_j) (degree 2p+1 grid latitudes j, n = m .. p) per order m:
// [m][K step][digit][Np x 16, K-major canonical], row n - m split after its own scale 2^-e.
int leg_tc_digits(shbim_ctx* ctx, int p, const std::vector<double>& alf0, DegreeTables& T) {
  if (!leg_tc_fits(p)) return SHBIM_OK;
  const int P1 = p + 1, K = 2 * p + 2, ksteps = (K + kKS - 1) / kKS;
  const int nt = P1 * (p + 2) / 2;
  std::vector<int> off(P1);
  size_t total = 0;
  for (int m = 0; m <= p; ++m) {
    off[m] = (int)(total / 8);
    const int Np = padded16(P1 - m);
    total += (size_t)ksteps * kDig * Np * kKS;
  }
  std::vector<uint16_t> h(total, 0);
  std::vector<signed char> ex((size_t)P1 * P1, 0);
  for (int m = 0; m <= p; ++m) {
    const int Nm = P1 - m, Np = padded16(Nm);
    const int tro = m * (p + 1) - m * (m - 1) / 2;
    std::vector<int> em(Np, 0);
    for (int nn = 0; nn < Nm; ++nn) {
      double mx = 0.0;
      for (int j = 0; j < K; ++j) mx = std::max(mx, std::fabs(alf0[(size_t)j * nt + tro + nn]));
      int e = 0;
      std::frexp(mx, &e);
      em[nn] = std::max(e, -60);
      ex[(size_t)m * P1 + nn] = (signed char)em[nn];
    }
    uint16_t* dst = h.data() + (size_t)off[m] * 8;
    for (int ks = 0; ks < ksteps; ++ks)
      for (int nn = 0; nn < Np; ++nn)
        for (int kk = 0; kk < kKS; ++kk) {
          const int j = ks * kKS + kk;
          const double v = (nn < Nm && j < K) ? alf0[(size_t)j * nt + tro + nn] : 0.0;
          int dg[kDig];
          digits_host(v, em[nn], dg);
          for (int jd = 0; jd < kDig; ++jd) dst[((size_t)ks * kDig + jd) * Np * kKS + canon16(nn, kk)] = bf16_int(dg[jd]);
        }
  }
  if (cudaMalloc(&T.leg_digits, h.size() * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&T.leg_toff, off.size() * sizeof(int)) != cudaSuccess || cudaMalloc(&T.leg_exp, ex.size()) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc Legendre digit table");
  if (cudaMemcpy(T.leg_digits, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.leg_toff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.leg_exp, ex.data(), ex.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_CUDA, "cudaMemcpy Legendre digit table");
  return SHBIM_OK;
}

int analysis_legendre_tc(shbim_ctx* ctx, const DegreeTables& T, const float2* FT, int64_t nitems, float2* coef,
                         int64_t coef_stride, cudaStream_t s) {
  if (nitems <= 0) return SHBIM_OK;
  if (!T.leg_digits) return fail(ctx, SHBIM_ERR_ARG, "Legendre digit table missing");
  if (!ctx->tc_err) {
    if (cudaMalloc(&ctx->tc_err, sizeof(int)) != cudaSuccess)
      return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc tensor-core error flag");
    SHBIM_CUDA(ctx, cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), s));
  }
  const int p = T.p;
  const int smem = leg_tc_smem(p);
  SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_leg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const LegItems I(p, nitems);
  const unsigned grid = (unsigned)std::min<int64_t>(I.total, nsm);
  k_leg_tc<<<grid, kThreads, smem, s>>>(FT, nitems, p, reinterpret_cast<const uint4*>(T.leg_digits), T.leg_toff,
                                        T.leg_exp, coef, coef_stride, ctx->tc_err, ctx->wait_ns);
  SHBIM_CHECK_LAUNCH(ctx, "k_leg_tc");
  return SHBIM_OK;
}

}  // namespace shbim
