// Pole rotation of the singular-row build (Section 2.1) on the fifth-generation tensor cores, with
// FP64-class accuracy.
//   forward (ADJ = false): out = Dq^T Dz(-theta) Dq Dz(-phi) in   (position coefficients)
//   adjoint (ADJ = true):  out = Dz(phi) Dq^T Dz(theta) Dq in     (rows, FP32 planes)
// theta, phi are the base-grid angles of each vector's target; Dz(a) turns the pair of real
// coefficients (n, m), (n, -m) by the angle m a; Dq is the real-basis block of the quarter turn
// Rx(pi/2). Every target of one latitude shares M(+-theta) = Dq^T Dz(+-theta) Dq, so the middle
// three factors are one fixed (2n+1) x (2n+1) matrix per (latitude, degree, direction), formed in
// FP64 on the host: the rotation of the vectors of one latitude is a GEMM by that table, split into
// exact bfloat16 digit products (tc.cuh), followed (adjoint) or preceded (forward) by Dz(phi) on
// the double-float values in shared memory.
//
// Work decomposition: persistent CTAs (one per SM, 512 threads, all 512 tensor-memory columns:
// six accumulators of up to 80 columns) loop over items (up to 128 vectors of one latitude, one
// degree), largest degree first. Per item: the rows' degree block and their targets' phi tables are
// copied asynchronously into shared memory; the rows get a power-of-two scale; per K step of 16
// their digit planes and the table's pre-laid-out planes (bulk copies, prefetched a step ahead)
// fill one of two stages and one thread issues the 21 digit products as 9 MMAs (one row digit
// against up to three table digits, N <= 240); the epilogue combines the six
// accumulators in double-float. Every wait is bounded; a timeout sets the error flag and the CTA
// stops. Degree blocks with 2n+1 <= 80 (n <= 39) only: for drops of higher degree (whose shared memory
// still fits, p <= 48) the degrees above 39 use the FP32-pipe kernel (singular_df.cu).
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

constexpr int kThreads = 512;
constexpr int kNmax = 80;                                  // largest padded block (N and K)
static_assert(diag_sums_exact(kNmax), "rotations: digit sums must stay exact in FP32");
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

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// most targets one item's 128 vectors can touch, with ncomp components per target
__host__ __device__ inline int max_targets(int ncomp) { return kMT / ncomp + 2; }

// The items of one launch: latitudes lat0 .. lat0 + L - 1 of the chunk, T tiles of 128 vectors per
// latitude, degrees nmax .. 0 (nmax <= p: the higher degrees of a drop whose blocks exceed kNmax are
// rotated by the double-float kernel).
struct Items {
  int p, nmax, nlon, ncomp, t_begin, ct, lat0, L, T;
  int64_t total;
  __host__ __device__ Items(int p_, int nmax_, int ncomp_, int t_begin_, int ct_)
      : p(p_), nmax(nmax_), nlon(2 * p_ + 2), ncomp(ncomp_), t_begin(t_begin_), ct(ct_) {
    lat0 = t_begin / nlon;
    L = (t_begin + ct - 1) / nlon - lat0 + 1;
    T = (nlon * ncomp + kMT - 1) / kMT;
    total = (int64_t)(nmax + 1) * L * T;
  }
  // degree, latitude and chunk-local vector range [va, vb) of an item (empty if va >= vb)
  __device__ void decode(int64_t it, int& n, int& lat, int& va, int& vb) const {
    const int64_t per_n = (int64_t)L * T;
    n = nmax - (int)(it / per_n);
    const int rem = (int)(it - (int64_t)(nmax - n) * per_n);
    lat = lat0 + rem / T;
    const int tile = rem - (rem / T) * T;
    const int ta = max(t_begin, lat * nlon) - t_begin, tb = min(t_begin + ct, (lat + 1) * nlon) - t_begin;
    va = ta * ncomp + tile * kMT;
    vb = min(tb * ncomp, va + kMT);
  }
  // the first non-empty item at or after `it` in steps of `stride` (total if none)
  __device__ int64_t next(int64_t it, int64_t stride) const {
    for (; it < total; it += stride) {
      int n, lat, va, vb;
      decode(it, n, lat, va, vb);
      if (va < vb) return it;
    }
    return total;
  }
};

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, 1)
k_rotate_tc(const float2* __restrict__ vin, int64_t in_stride, int nc, int p, int nmax, int t_begin, int ct, int ncomp,
            const float2* __restrict__ cs_phi, const uint4* __restrict__ tdig, const int* __restrict__ toff,
            const signed char* __restrict__ texp, float2* __restrict__ vout, float* __restrict__ rows_lap,
            float* __restrict__ rows_sto, int nt_drop, int* __restrict__ err, uint64_t wlim) {
  // dynamic shared memory: [two MMA stages][value block 128 x (2p+1)][(cos, sin)(m phi) of the
  // item's targets, 2 (p+1) each]
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t bbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int rowexp[kMT];
  __shared__ int rowtgt[kMT];
  __shared__ int colexp[kNmax];
  const int WS = 2 * p + 1;   // row stride of the value block (odd: conflict-free column access)
  const int CS = 2 * (p + 1); // one angle table
  float2* sX = reinterpret_cast<float2*>(smem + 2 * kStageBytes);
  float2* sCS = sX + kMT * WS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Items I(p, nmax, ncomp, t_begin, ct);
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
  bool pending[2] = {false, false};   // MMAs committed on the stage and not yet waited for
  bool bpend[2] = {false, false};     // table copy issued into the stage and not yet waited for
  bool abort_all = false;
  const int r_loc = tid & (kMT - 1), qt = tid >> 7;   // row of the tile, quarter of a K step
  // table planes of (latitude, degree), K step ks, into stage st (thread 0)
  auto issue_b = [&](int lat, int n, int ks, int st) {
    const int Np = padded(2 * n + 1);
    const uint32_t bytes = (uint32_t)(kDig * Np * kKS * 2);
    const int64_t o = toff[((ADJ ? 1 : 0) * (p + 1) + lat) * (p + 1) + n];
    bulk_load(smem + st * kStageBytes + kDig * kPlaneA * 2, tdig + o + (int64_t)ks * (bytes / 16), bytes, &bbar[st]);
  };
  // the first two K steps' table planes of item `it` (both stages free)
  auto prefetch = [&](int64_t it) {
    int n, lat, va, vb;
    I.decode(it, n, lat, va, vb);
    const bool two = padded(2 * n + 1) > kKS;
    if (tid == 0) {
      issue_b(lat, n, 0, 0);
      if (two) issue_b(lat, n, 1, 1);
    }
    bpend[0] = true;
    bpend[1] = two;
  };
  // Dz(+-phi) on every row's degree-n block, in place, with the row's target's table
  auto dz = [&](int n, bool neg) {
    const int rt = rowtgt[r_loc];
    if (rt < 0) return;
    const float2* cs = sCS + rt * CS;
    float2* x = sX + r_loc * WS;
    for (int m = 1 + qt; m <= n; m += 4) {
      const float2 c2 = cs[m], s2 = cs[p + 1 + m];
      const df ca{c2.x, c2.y};
      const df sa = neg ? df{-s2.x, -s2.y} : df{s2.x, s2.y};
      const df a = lds(x, n + m), b = lds(x, n - m);
      sts(x, n + m, dfl::sub(dfl::mul(ca, a), dfl::mul(sa, b)));
      sts(x, n - m, dfl::add(dfl::mul(sa, a), dfl::mul(ca, b)));
    }
  };

  int64_t item = I.next(blockIdx.x, gridDim.x);
  if (item < I.total) prefetch(item);
  while (item < I.total && !abort_all) {
    int n, lat, va, vb;
    I.decode(item, n, lat, va, vb);
    const int w = 2 * n + 1;
    const int Np = padded(w);
    const int ksteps = Np / kKS;
    const int b_lo = va / ncomp;
    const int nb = (vb - 1) / ncomp - b_lo + 1;
    // rows of the item (vector v = chunk-local target b, component c), their targets' phi tables
    // and degree blocks: asynchronous copies, one wait
    if (tid < kMT) {
      const int v = va + tid;
      rowtgt[tid] = v < vb ? v / ncomp - b_lo : -1;
    }
    if (tid < w) colexp[tid] = texp[((int64_t)(ADJ ? 1 : 0) * (p + 1) + lat) * (p + 1) * (p + 1) + n * n + tid];
    for (int e = tid; e < nb * (CS / 2); e += kThreads) {
      const int bt = e / (CS / 2), k2 = e - bt * (CS / 2);   // target, 16-byte piece of its table
      const int tl = t_begin + b_lo + bt;
      const float2* src = cs_phi + (int64_t)(tl % I.nlon) * CS;
      cp_async16(sCS + bt * CS + 2 * k2, src + 2 * k2);
    }
    for (int r = warp; r < kMT; r += kThreads / 32) {
      const int v = va + r;
      if (v < vb) {
        const int b = v / ncomp, c = v - b * ncomp;
        const float2* src = vin + (int64_t)b * in_stride + (int64_t)c * nc + (int64_t)n * n;
        for (int k = lane; k < w; k += 32) cp_async8(sX + r * WS + k, src + k);
      } else {
        for (int k = lane; k < w; k += 32) sX[r * WS + k] = make_float2(0.f, 0.f);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    if (!ADJ) {
      dz(n, true);
      __syncthreads();
    }
    // per-row power-of-two scale, max |hi| < 2^e: one thread per row (odd row stride: no bank
    // conflicts)
    if (tid < kMT) {
      float mx = 0.f;
      const float2* xr = sX + tid * WS;
      for (int k = 0; k < w; ++k) mx = fmaxf(mx, fabsf(xr[k].x));
      int e = 0;
      frexpf(mx, &e);
      rowexp[tid] = max(e, -120);
    }
    __syncthreads();
    const int e_r = rowexp[r_loc];
    const float2* xrow = sX + r_loc * WS;
    for (int ks = 0; ks < ksteps; ++ks) {
      const int st = ks & 1;
      if (pending[st]) {
        const bool ok = mbar_wait(&mbar[st], phase[st], wlim);
        phase[st] ^= 1u;
        pending[st] = false;
        if (__syncthreads_or(!ok)) {
          abort_all = true;
          break;
        }
      }
      uint8_t* base = smem + st * kStageBytes;
      {
        const float sc = __int_as_float((127 + 7 - e_r) << 23);   // 2^(7 - e), exact
        float d[kDig][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int k = ks * kKS + qt * 4 + i;
          const float2 v = k < w ? xrow[k] : make_float2(0.f, 0.f);
          float dd[kDig];
          digits6(v.x * sc, v.y * sc, dd);
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
      }
      asm volatile("fence.proxy.async.shared::cta;\n");
      __syncthreads();
      if (tid == 0) {
        // the table planes have landed (bounded; on expiry the products are skipped and the
        // caller sees the error flag)
        if (!mbar_wait(&bbar[st], bphase[st], wlim)) atomicExch(err, 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        const uint32_t a0 = smem_u32(base), b0 = smem_u32(base + kDig * kPlaneA * 2);
        // row digit j_a against up to three consecutive table digits in one MMA of N = Np g (the
        // planes lie one after the other like the rows of one operand; their products go to the
        // consecutive accumulators j_a + j_b - 5 ..); j_a = 5 first, overwriting all six in step 0
#pragma unroll
        for (int ja = kDig - 1; ja >= 0; --ja)
#pragma unroll
          for (int jb0 = kDig - 1 - ja; jb0 < kDig; jb0 += 3) {
            const int g = min(3, kDig - jb0);
            const int dgl = ja + jb0 - (kDig - 1);
            const uint32_t acc = (ks > 0 || ja != kDig - 1) ? 1u : 0u;
            mma_bf16(tmem + (uint32_t)(dgl * Np), desc_k16(a0 + ja * kPlaneA * 2), desc_k16(b0 + jb0 * Np * kKS * 2),
                     idesc_bf16(Np * g), acc);
          }
        mma_commit(&mbar[st]);
        // the table planes of K step ks + 1 go to the other stage once its products are done
        // (step 1's planes were issued with step 0's)
        if (ks >= 1 && ks + 1 < ksteps) {
          mbar_wait(&mbar[st ^ 1], phase[st ^ 1], wlim);
          issue_b(lat, n, ks + 1, st ^ 1);
        }
      }
      bphase[st] ^= 1u;
      bpend[st] = false;
      if (ks >= 1 && ks + 1 < ksteps) bpend[st ^ 1] = true;
      pending[st] = true;
    }
    if (abort_all) break;
    bool ok = true;
    for (int st = 0; st < 2; ++st)
      if (pending[st]) {
        ok = ok && mbar_wait(&mbar[st], phase[st], wlim);
        phase[st] ^= 1u;
        pending[st] = false;
      }
    if (__syncthreads_or(!ok)) {
      abort_all = true;
      break;
    }
    // both stages are free: the next item's first table planes travel during the epilogue
    const int64_t next = I.next(item + gridDim.x, gridDim.x);
    if (next < I.total) prefetch(next);
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    // epilogue: warp w reads lanes 32 (w % 4) .. +31; column blocks of 8 split among w, w+4, w+8, w+12
    {
      const int lq = warp & 3, wq = warp >> 2;
      const int rl = 32 * lq + lane;
      const int ee = rowexp[rl];
      for (int cb = wq; cb < Np / 8; cb += 4) {
        uint32_t a[kDig][8];
#pragma unroll
        for (int dg = 0; dg < kDig; ++dg)
          tmem_ld8(tmem + ((uint32_t)(32 * lq) << 16) + (uint32_t)(dg * Np + cb * 8), a[dg]);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int o = cb * 8 + j;
          if (o < w) {
            const df r = combine6(__uint_as_float(a[5][j]), __uint_as_float(a[4][j]), __uint_as_float(a[3][j]),
                                  __uint_as_float(a[2][j]), __uint_as_float(a[1][j]), __uint_as_float(a[0][j]));
            sX[rl * WS + o] = scale2(r, ee + colexp[o] - 14);
          }
        }
      }
    }
    // the next products overwrite the accumulators only after every read
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (ADJ) {
      dz(n, false);
      __syncthreads();
    }
    // store (warp per row, lanes along the block)
    for (int r = warp; r < kMT; r += kThreads / 32) {
      const int v = va + r;
      if (v >= vb) continue;
      const int b = v / ncomp, c = v - b * ncomp;
      if (!ADJ) {
        float2* dst = vout + ((int64_t)b * ncomp + c) * nc + (int64_t)n * n;
        for (int k = lane; k < w; k += 32) dst[k] = sX[r * WS + k];
      } else {
        const int64_t tl = (int64_t)t_begin + b;
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
    item = next;
  }
  // let products and copies still in flight finish (bounded) before the memory is released
  for (int st = 0; st < 2; ++st) {
    if (pending[st]) mbar_wait(&mbar[st], phase[st], kDrainNs);
    if (bpend[st] && tid == 0) mbar_wait(&bbar[st], bphase[st], kDrainNs);
  }
  if (abort_all && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

int rot_tc_smem(int p, int ncomp) {
  return 2 * kStageBytes + (kMT * (2 * p + 1) + max_targets(ncomp) * 2 * (p + 1)) * (int)sizeof(float2);
}

}  // namespace

// Highest degree the tensor-core rotations take for drops of degree p (blocks up to kNmax), or -1 where
// the shared memory of degree p does not fit (the forward rotation, 3 components per target, needs the
// most angle tables); the degrees above it go to the double-float kernel.
int rot_tc_nmax(int p) {
  if (rot_tc_smem(p, 3) + 4096 > 227 * 1024) return -1;
  int n = p;
  while (n >= 0 && padded(2 * n + 1) > kNmax) --n;
  return n;
}

// Digit planes of M = Dq_n^T Dz(-theta_j) Dq_n (forward, dir 0) and Dq_n^T Dz(theta_j) Dq_n
// (adjoint, dir 1) for every base-grid latitude j and degree n, as the B operand B[m][k] = M[m][k]:
// [dir][j][n][K step][digit][Np x 16, K-major canonical], offsets in 16-byte units per (dir, j, n).
// Row m is split after its own power-of-two scale 2^-e_m (e_m stored per (dir, j, n, m)), so the
// digits keep ~42 bits of every row whatever its size.
int rot_tc_digits(shbim_ctx* ctx, int p, const std::vector<double>& D, const std::vector<double>& theta,
                  DegreeTables& T) {
  const int nmax = rot_tc_nmax(p);
  if (nmax < 0) return SHBIM_OK;
  const int P1 = p + 1;
  std::vector<int64_t> off((size_t)2 * P1 * P1, 0);
  int64_t total = 0;   // uint16 elements
  for (int dir = 0; dir < 2; ++dir)
    for (int j = 0; j < P1; ++j)
      for (int n = 0; n <= nmax; ++n) {
        off[((size_t)dir * P1 + j) * P1 + n] = total / 8;
        const int Np = padded(2 * n + 1);
        total += (int64_t)(Np / kKS) * kDig * Np * kKS;
      }
  if (total / 8 > INT_MAX) return fail(ctx, SHBIM_ERR_ARG, "rotation digit table too large");
  std::vector<uint16_t> h((size_t)total, 0);
  std::vector<signed char> ex((size_t)2 * P1 * P1 * P1, 0);   // [dir][j][(p+1)^2] row exponents
#pragma omp parallel for schedule(dynamic, 1)
  for (int dj = 0; dj < 2 * P1; ++dj) {
    const int dir = dj / P1, j = dj - dir * P1;
    const double a = dir == 0 ? -theta[j] : theta[j];
    std::vector<double> Z, M;
    for (int n = 0; n <= nmax; ++n) {
      const int w = 2 * n + 1, Np = padded(w);
      const double* Dn = &D[T.dq_off[n]];
      // Z = Dz(a) Dq_n: rows (n + m, n - m) turned by m a
      Z.assign(Dn, Dn + (size_t)w * w);
      for (int m = 1; m <= n; ++m) {
        const double c = std::cos(m * a), s = std::sin(m * a);
        for (int k = 0; k < w; ++k) {
          const double x = Dn[(size_t)(n + m) * w + k], y = Dn[(size_t)(n - m) * w + k];
          Z[(size_t)(n + m) * w + k] = c * x - s * y;
          Z[(size_t)(n - m) * w + k] = s * x + c * y;
        }
      }
      // M = Dq_n^T Z
      M.assign((size_t)w * w, 0.0);
      for (int k = 0; k < w; ++k)
        for (int r = 0; r < w; ++r) {
          const double dkr = Dn[(size_t)k * w + r];
          if (dkr == 0.0) continue;
          for (int c2 = 0; c2 < w; ++c2) M[(size_t)r * w + c2] += dkr * Z[(size_t)k * w + c2];
        }
      // a power-of-two scale per row m of M (max_k |M[m][k]| < 2^e_m), undone per output column
      std::vector<int> em(Np, 0);
      for (int m = 0; m < w; ++m) {
        double mx = 0.0;
        for (int k = 0; k < w; ++k) mx = std::max(mx, std::fabs(M[(size_t)m * w + k]));
        int e = 0;
        std::frexp(mx, &e);
        em[m] = std::max(e, -60);
        ex[((size_t)dj * P1) * P1 + (size_t)n * n + m] = (signed char)em[m];
      }
      uint16_t* dst = h.data() + off[(size_t)dj * P1 + n] * 8;
      for (int ks = 0; ks < Np / kKS; ++ks)
        for (int m = 0; m < Np; ++m)
          for (int kk = 0; kk < kKS; ++kk) {
            const int k = ks * kKS + kk;
            const double v = (m < w && k < w) ? M[(size_t)m * w + k] : 0.0;
            int dg[kDig];
            digits_host(v, em[m], dg);
            for (int jd = 0; jd < kDig; ++jd)
              dst[((size_t)ks * kDig + jd) * Np * kKS + canon16(m, kk)] = bf16_int(dg[jd]);
          }
    }
  }
  std::vector<int> off32(off.begin(), off.end());
  if (cudaMalloc(&T.rot_digits, h.size() * sizeof(uint16_t)) != cudaSuccess ||
      cudaMalloc(&T.rot_toff, off32.size() * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&T.rot_exp, ex.size()) != cudaSuccess)
    return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc rotation digit table");
  if (cudaMemcpy(T.rot_digits, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.rot_toff, off32.data(), off32.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(T.rot_exp, ex.data(), ex.size(), cudaMemcpyHostToDevice) != cudaSuccess)
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
  const int nmax = rot_tc_nmax(p);
  if (nmax < 0) return fail(ctx, SHBIM_ERR_ARG, "degree too large for the tensor-core rotations");
  const int smem = rot_tc_smem(p, ncomp);
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const Items I(p, nmax, ncomp, t_begin, ct);
  const unsigned grid = (unsigned)std::min<int64_t>(I.total, nsm);
  const uint4* tdig = reinterpret_cast<const uint4*>(T.rot_digits);
  if (adjoint) {
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rotate_tc<true><<<grid, kThreads, smem, s>>>(vin, in_stride, nc, p, nmax, t_begin, ct, ncomp, T.cs_phi_df, tdig,
                                                   T.rot_toff, T.rot_exp, vout, rows_lap, rows_sto, nt_drop,
                                                   ctx->tc_err, ctx->wait_ns);
  } else {
    SHBIM_CUDA(ctx, cudaFuncSetAttribute(k_rotate_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_rotate_tc<false><<<grid, kThreads, smem, s>>>(vin, in_stride, nc, p, nmax, t_begin, ct, ncomp, T.cs_phi_df, tdig,
                                                    T.rot_toff, T.rot_exp, vout, rows_lap, rows_sto, nt_drop,
                                                   ctx->tc_err, ctx->wait_ns);
  }
  SHBIM_CHECK_LAUNCH(ctx, "k_rotate_tc");
  return SHBIM_OK;
}

}  // namespace shbim
