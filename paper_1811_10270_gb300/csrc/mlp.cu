// Learned GMRES warm start: a multilayer perceptron with bfloat16 weights and FP32
// accumulation, trained and evaluated by the kernels in this file (the paper has no learned
// component; the network only supplies an initial guess that GMRES then judges).
//
// Layers: h_l = tanh(bf16(h_{l-1}) bf16(W_l)^T + b_l), the last one linear; loss
// sum (y - t)^2 / (2 B); backward with the bfloat16 rounding treated as identity; Adam on FP32
// master weights, whose bfloat16 copy feeds the forward products.
//
// All products go through one tensor-core GEMM: C(m, n) = sum_k A(m, k) B(k, n) with A and B
// read through arbitrary strides (so W, W^T, dZ^T need no transposed copies), staged to shared
// memory as bfloat16 and multiplied by the fifth-generation tensor cores (tcgen05.mma, bf16 x bf16
// -> f32 accumulated in tensor memory).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

struct shbim_mlp {
  int L = 0;
  std::vector<int> w;          // widths, L+1
  int max_batch = 0;
  std::vector<float*> W, b, gW, gb, mW, vW, mb, vb;
  std::vector<__nv_bfloat16*> Wh;
  std::vector<float*> H;       // activations [max_batch][w_l], l = 0..L
  float* xin = nullptr;        // [max_batch][w_0] standardised input when an input affine is set
  float* shift = nullptr;      // [w_0] input affine x_n = (x - shift) * scale, applied in FP32
  float* scale = nullptr;
  bool affine = false;
  float* dA = nullptr;         // [max_batch][max width]
  float* dB = nullptr;
  double* loss = nullptr;
  int t = 0;                   // Adam step
};

namespace shbim {
namespace {

// ---------------------------------------------------------------- tcgen05 GEMM
// C(m, n) = act(sum_k A(m, k) B(k, n) + bias(n)) for one 128 x 64 tile of C per CTA (4 warps).
// Per K block of 64: the CTA stages A (128 x 64) and B (64 x 64, as N x K) into shared memory as
// bfloat16 in the no-swizzle K-major canonical layout (8-row x 16-byte core matrices; leading-
// dimension offset = 128 B between core matrices along K, stride offset = 1024 B between 8-row
// groups), one thread issues four tcgen05.mma kind::f16 (M = 128, N = 64, K = 16) accumulating in
// tensor memory and commits them to an mbarrier; every wait is bounded (a timed-out tile is
// written as NaN so the failure is loud). The epilogue reads the accumulator with tcgen05.ld.
constexpr int TM = 128, TN = 64, TK = 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// index of element (row r, k) in a [rows][TK] K-major canonical tile
__device__ __forceinline__ int canon(int r, int k) { return ((r >> 3) * (TK >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;          // leading-dimension byte offset (K)
  d |= (uint64_t)(((TK / 8 * 128) >> 4) & 0x3FFF) << 32;  // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                                // descriptor version; no swizzle
  return d;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(128)
k_gemm_tc(int M, int N, int K, const TA* __restrict__ A, int64_t sam, int64_t sak, const TB* __restrict__ B,
          int64_t sbk, int64_t sbn, float* __restrict__ C, int64_t scm, int64_t scn,
          const float* __restrict__ bias, int act) {
  __shared__ __align__(1024) __nv_bfloat16 sA[TM * TK];
  __shared__ __align__(1024) __nv_bfloat16 sB[TN * TK];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  bool ok = true;
  int phase = 0;
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = tid; e < TM * TK; e += 128) {
      const int mm = e / TK, kk = e - mm * TK;
      const int gm = m0 + mm, gk = k0 + kk;
      const float v = (gm < M && gk < K) ? (float)A[(int64_t)gm * sam + (int64_t)gk * sak] : 0.f;
      sA[canon(mm, kk)] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < TN * TK; e += 128) {
      const int nn = e / TK, kk = e - nn * TK;
      const int gn = n0 + nn, gk = k0 + kk;
      const float v = (gn < N && gk < K) ? (float)B[(int64_t)gk * sbk + (int64_t)gn * sbn] : 0.f;
      sB[canon(nn, kk)] = __float2bfloat16_rn(v);
    }
    asm volatile("fence.proxy.async.shared::cta;\n");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
      for (int ks = 0; ks < TK / 16; ++ks) {
        const uint64_t da = smem_desc(smem_u32(sA) + ks * 256);
        const uint64_t db = smem_desc(smem_u32(sB) + ks * 256);
        const uint32_t acc = (k0 > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(&mbar)));
    }
    // the staged tiles may be overwritten only after the MMAs that read them have completed
    // (bounded by one second of the global timer)
    uint32_t done = 0;
    uint64_t t0 = 0;
    for (int it = 0; !done; ++it) {
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(done)
          : "r"(smem_u32(&mbar)), "r"(phase));
      uint64_t t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (it == 0) t0 = t;
      else if (!done && t - t0 > 1000000000ull) break;
    }
    phase ^= 1;
    // leave the K loop together: a barrier count mismatch would hang the CTA
    if (!__syncthreads_and(done)) {
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n");
  }
  const int row = m0 + 32 * warp + (tid & 31);
  for (int c0 = 0; c0 < TN; c0 += 16) {
    uint32_t v[16];
    if (ok) {
      const uint32_t addr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n");
    }
    if (row < M) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int gn = n0 + c0 + j;
        if (gn < N) {
          float x = ok ? __uint_as_float(v[j]) + (bias ? bias[gn] : 0.f) : __int_as_float(0x7fc00000);
          if (act) x = tanhf(x);
          C[(int64_t)row * scm + (int64_t)gn * scn] = x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN));
}

template <typename TA, typename TB>
int gemm(shbim_mlp*, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk,
         int64_t sbn, float* C, int64_t scm, int64_t scn, const float* bias, int act, cudaStream_t s) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm_tc<TA, TB><<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, scm, scn, bias, act);
  return cudaGetLastError() == cudaSuccess ? SHBIM_OK : SHBIM_ERR_CUDA;
}

__global__ void k_out_grad(const float* __restrict__ y, const float* __restrict__ t, int64_t n, float inv_b,
                           float* __restrict__ d, double* __restrict__ loss) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (e < n) {
    const float r = y[e] - t[e];
    d[e] = r * inv_b;
    l = 0.5 * (double)r * (double)r * inv_b;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

__global__ void k_tanh_grad(float* __restrict__ d, const float* __restrict__ h, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) d[e] *= 1.f - h[e] * h[e];
}

// gb[n] = sum_b d[b][n]  (fixed order)
__global__ void k_colsum(const float* __restrict__ d, int B, int N, float* __restrict__ gb) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += d[(int64_t)b * N + n];
  gb[n] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float c1, float c2, __nv_bfloat16* __restrict__ ph) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float gg = g[e];
  const float mm = 0.9f * m[e] + 0.1f * gg;
  const float vv = 0.999f * v[e] + 0.001f * gg * gg;
  m[e] = mm;
  v[e] = vv;
  const float q = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
  p[e] = q;
  if (ph) ph[e] = __float2bfloat16_rn(q);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = __float2bfloat16_rn(a[e]);
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) b[e] = (float)a[e];
}

__global__ void k_warm(const float* __restrict__ y, const double* __restrict__ rhs, double c, double* __restrict__ x0,
                       int64_t n) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) x0[e] = c * rhs[e] + (double)y[e];
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

// the scalar tail of the warm-start features: E_u (3), E_q, lambda per drop, R, Q, Ca_E
__global__ void k_feature_tail(float* __restrict__ f, double e0, double e1, double e2, double eq,
                               const double* __restrict__ lamm1, int n_drops, double R, double Q, double ca) {
  const int i = threadIdx.x;
  if (i == 0) {
    f[0] = (float)e0;
    f[1] = (float)e1;
    f[2] = (float)e2;
    f[3] = (float)eq;
    f[4 + n_drops] = (float)R;
    f[5 + n_drops] = (float)Q;
    f[6 + n_drops] = (float)ca;
  }
  for (int d = i; d < n_drops; d += blockDim.x) f[4 + d] = (float)(lamm1[d] + 1.0);
}

__global__ void k_guess(const float* __restrict__ y, const double* __restrict__ rhs, double c, double* __restrict__ En0,
                        double* __restrict__ u0, int64_t nc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * nc) return;
  if (e < nc) {
    if (En0) En0[e] = c * rhs[e] + (double)y[e];
  } else if (u0) {
    u0[e - nc] = (double)y[e];
  }
}

__global__ void k_affine(const float* __restrict__ x, const float* __restrict__ shift, const float* __restrict__ scale,
                         int64_t n, int w, float* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) {
    const int c = (int)(e % w);
    out[e] = (x[e] - shift[c]) * scale[c];
  }
}

// network input after the optional FP32 affine
const float* input_of(shbim_mlp* net, int B, const float* x, cudaStream_t s) {
  if (!net->affine) return x;
  const int64_t n = (int64_t)B * net->w[0];
  k_affine<<<nb(n), 256, 0, s>>>(x, net->shift, net->scale, n, net->w[0], net->xin);
  return net->xin;
}

// Inference of a few rows (B <= 4), where a layer is a matrix-vector product bound by reading the
// weights once from HBM: y[b][n] = act(sum_k bf16(x[b][k]) W[n][k] + bias[n]), the same function as
// the tensor-core forward (inputs rounded to bfloat16, products exact in FP32, FP32 sums). The rows
// of x sit in shared memory; two warps per output split K and read W's row coalesced.
constexpr int kGemvRows = 4;
constexpr int kGemvOut = 4;            // outputs per CTA (8 warps)
__global__ void __launch_bounds__(256)
k_gemv_bf16(int B, int N, int K, const float* __restrict__ x, const __nv_bfloat16* __restrict__ W,
            const float* __restrict__ bias, int act, float* __restrict__ y) {
  extern __shared__ float xs[];        // [B][K] bf16-rounded inputs
  __shared__ float part[8][kGemvRows];
  for (int e = threadIdx.x; e < B * K; e += blockDim.x) xs[e] = __bfloat162float(__float2bfloat16_rn(x[e]));
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = blockIdx.x * kGemvOut + (warp >> 1);
  const int half = (K + 1) / 2;
  const int k0 = (warp & 1) * half, k1 = min(K, k0 + half);
  float acc[kGemvRows] = {0.f, 0.f, 0.f, 0.f};
  if (n < N) {
    const __nv_bfloat16* w = W + (int64_t)n * K;
    for (int k = k0 + lane; k < k1; k += 32) {
      const float wv = __bfloat162float(w[k]);
#pragma unroll
      for (int b = 0; b < kGemvRows; ++b)
        if (b < B) acc[b] = fmaf(wv, xs[b * K + k], acc[b]);
    }
  }
#pragma unroll
  for (int b = 0; b < kGemvRows; ++b)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[b] += __shfl_xor_sync(0xffffffffu, acc[b], o);
  if (lane == 0)
#pragma unroll
    for (int b = 0; b < kGemvRows; ++b) part[warp][b] = acc[b];
  __syncthreads();
  if (!(warp & 1) && lane < B && n < N) {
    float v = part[warp][lane] + part[warp + 1][lane] + (bias ? bias[n] : 0.f);
    if (act) v = tanhf(v);
    y[(int64_t)lane * N + n] = v;
  }
}

int forward(shbim_mlp* net, int B, const float* x, cudaStream_t s) {
  const float* in = x;
  for (int l = 0; l < net->L; ++l) {
    const int K = net->w[l], N = net->w[l + 1];
    const size_t smem = (size_t)B * K * sizeof(float);
    if (B <= kGemvRows && smem <= 200 * 1024) {
      if (smem > 48 * 1024 &&
          cudaFuncSetAttribute(k_gemv_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return SHBIM_ERR_CUDA;
      k_gemv_bf16<<<(unsigned)((N + kGemvOut - 1) / kGemvOut), 256, smem, s>>>(B, N, K, in, net->Wh[l], net->b[l],
                                                                              l < net->L - 1 ? 1 : 0, net->H[l + 1]);
      if (cudaGetLastError() != cudaSuccess) return SHBIM_ERR_CUDA;
    } else {
      int rc = gemm<float, __nv_bfloat16>(net, B, N, K, in, K, 1, net->Wh[l], 1, K, net->H[l + 1], N, 1, net->b[l],
                                          l < net->L - 1 ? 1 : 0, s);
      if (rc) return rc;
    }
    in = net->H[l + 1];
  }
  return SHBIM_OK;
}

}  // namespace
}  // namespace shbim

using namespace shbim;

extern "C" {

int shbim_mlp_create(int n_layers, const int32_t* widths, int max_batch, shbim_mlp** out) {
  if (!out || n_layers < 1 || n_layers > 16 || !widths || max_batch < 1) return SHBIM_ERR_ARG;
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || widths[l] > (1 << 20)) return SHBIM_ERR_ARG;
  shbim_mlp* n = new shbim_mlp();
  n->L = n_layers;
  n->w.assign(widths, widths + n_layers + 1);
  n->max_batch = max_batch;
  bool ok = true;
  auto alloc = [&](float** p, size_t cnt) {
    if (cudaMalloc(p, std::max<size_t>(cnt, 1) * sizeof(float)) != cudaSuccess) ok = false;
    else cudaMemset(*p, 0, cnt * sizeof(float));
  };
  int wmax = 0;
  for (int l = 0; l <= n_layers; ++l) wmax = std::max(wmax, widths[l]);
  n->W.resize(n_layers); n->b.resize(n_layers); n->gW.resize(n_layers); n->gb.resize(n_layers);
  n->mW.resize(n_layers); n->vW.resize(n_layers); n->mb.resize(n_layers); n->vb.resize(n_layers);
  n->Wh.resize(n_layers);
  n->H.resize(n_layers + 1);
  for (int l = 0; l < n_layers && ok; ++l) {
    const size_t nw = (size_t)widths[l] * widths[l + 1];
    alloc(&n->W[l], nw); alloc(&n->gW[l], nw); alloc(&n->mW[l], nw); alloc(&n->vW[l], nw);
    alloc(&n->b[l], widths[l + 1]); alloc(&n->gb[l], widths[l + 1]);
    alloc(&n->mb[l], widths[l + 1]); alloc(&n->vb[l], widths[l + 1]);
    if (cudaMalloc(&n->Wh[l], nw * sizeof(__nv_bfloat16)) != cudaSuccess) ok = false;
    else cudaMemset(n->Wh[l], 0, nw * sizeof(__nv_bfloat16));
  }
  for (int l = 0; l <= n_layers && ok; ++l) alloc(&n->H[l], (size_t)max_batch * widths[l]);
  if (ok) alloc(&n->xin, (size_t)max_batch * widths[0]);
  if (ok) alloc(&n->shift, widths[0]);
  if (ok) alloc(&n->scale, widths[0]);
  if (ok) alloc(&n->dA, (size_t)max_batch * wmax);
  if (ok) alloc(&n->dB, (size_t)max_batch * wmax);
  if (ok && cudaMalloc(&n->loss, sizeof(double)) != cudaSuccess) ok = false;
  if (!ok) {
    *out = n;
    return SHBIM_ERR_NOMEM;
  }
  *out = n;
  return SHBIM_OK;
}

int shbim_mlp_destroy(shbim_mlp* n) {
  if (!n) return SHBIM_ERR_ARG;
  cudaDeviceSynchronize();
  for (int l = 0; l < n->L; ++l) {
    cudaFree(n->W[l]); cudaFree(n->gW[l]); cudaFree(n->mW[l]); cudaFree(n->vW[l]);
    cudaFree(n->b[l]); cudaFree(n->gb[l]); cudaFree(n->mb[l]); cudaFree(n->vb[l]); cudaFree(n->Wh[l]);
  }
  for (auto* h : n->H) cudaFree(h);
  cudaFree(n->xin);
  cudaFree(n->shift);
  cudaFree(n->scale);
  cudaFree(n->dA);
  cudaFree(n->dB);
  cudaFree(n->loss);
  delete n;
  return SHBIM_OK;
}

int shbim_mlp_set_layer(shbim_mlp* n, int l, const float* W_host, const float* b_host) {
  if (!n || l < 0 || l >= n->L || !W_host || !b_host) return SHBIM_ERR_ARG;
  const size_t nw = (size_t)n->w[l] * n->w[l + 1];
  if (cudaMemcpy(n->W[l], W_host, nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n->b[l], b_host, n->w[l + 1] * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return SHBIM_ERR_CUDA;
  k_to_bf16<<<nb(nw), 256>>>(n->W[l], n->Wh[l], nw);
  cudaMemset(n->mW[l], 0, nw * sizeof(float));
  cudaMemset(n->vW[l], 0, nw * sizeof(float));
  cudaMemset(n->mb[l], 0, n->w[l + 1] * sizeof(float));
  cudaMemset(n->vb[l], 0, n->w[l + 1] * sizeof(float));
  n->t = 0;
  return cudaDeviceSynchronize() == cudaSuccess ? SHBIM_OK : SHBIM_ERR_CUDA;
}

int shbim_mlp_set_input_affine(shbim_mlp* n, const float* shift_host, const float* scale_host) {
  if (!n) return SHBIM_ERR_ARG;
  if (!shift_host || !scale_host) {
    n->affine = false;
    return SHBIM_OK;
  }
  if (cudaMemcpy(n->shift, shift_host, n->w[0] * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(n->scale, scale_host, n->w[0] * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
    return SHBIM_ERR_CUDA;
  n->affine = true;
  return SHBIM_OK;
}

int shbim_mlp_get_layer(shbim_mlp* n, int l, float* W_host, float* b_host, float* gW_host, float* gb_host) {
  if (!n || l < 0 || l >= n->L) return SHBIM_ERR_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return SHBIM_ERR_CUDA;
  const size_t nw = (size_t)n->w[l] * n->w[l + 1];
  const size_t nbias = n->w[l + 1];
  if ((W_host && cudaMemcpy(W_host, n->W[l], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (b_host && cudaMemcpy(b_host, n->b[l], nbias * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (gW_host && cudaMemcpy(gW_host, n->gW[l], nw * 4, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (gb_host && cudaMemcpy(gb_host, n->gb[l], nbias * 4, cudaMemcpyDeviceToHost) != cudaSuccess))
    return SHBIM_ERR_CUDA;
  return SHBIM_OK;
}

int shbim_mlp_forward(shbim_mlp* n, int batch, const float* x_dev, float* y_dev, void* stream) {
  if (!n || batch < 1 || batch > n->max_batch || !x_dev || !y_dev) return SHBIM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(n, batch, input_of(n, batch, x_dev, s), s);
  if (rc) return rc;
  const size_t ny = (size_t)batch * n->w[n->L];
  return cudaMemcpyAsync(y_dev, n->H[n->L], ny * sizeof(float), cudaMemcpyDeviceToDevice, s) == cudaSuccess
             ? SHBIM_OK : SHBIM_ERR_CUDA;
}

int shbim_mlp_train_step(shbim_mlp* n, int batch, const float* x_dev, const float* t_dev, float lr, int update,
                         double* loss_host, void* stream) {
  if (!n || batch < 1 || batch > n->max_batch || !x_dev || !t_dev) return SHBIM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const float* x_in = input_of(n, batch, x_dev, s);
  int rc = forward(n, batch, x_in, s);
  if (rc) return rc;
  const int L = n->L;
  const int64_t ny = (int64_t)batch * n->w[L];
  cudaMemsetAsync(n->loss, 0, sizeof(double), s);
  k_out_grad<<<nb(ny), 256, 0, s>>>(n->H[L], t_dev, ny, 1.0f / batch, n->dA, n->loss);
  float* d = n->dA;
  float* dn = n->dB;
  for (int l = L - 1; l >= 0; --l) {
    const int K = n->w[l], N = n->w[l + 1];
    if (l < L - 1) k_tanh_grad<<<nb((int64_t)batch * N), 256, 0, s>>>(d, n->H[l + 1], (int64_t)batch * N);
    const float* in = l == 0 ? x_in : n->H[l];
    // gW[N x K] = d^T [N x B] . in [B x K]
    if ((rc = gemm<float, float>(n, N, K, batch, d, 1, N, in, K, 1, n->gW[l], K, 1, nullptr, 0, s))) return rc;
    k_colsum<<<(N + 255) / 256, 256, 0, s>>>(d, batch, N, n->gb[l]);
    if (l > 0) {
      // dn [B x K] = d [B x N] . W [N x K]
      if ((rc = gemm<float, __nv_bfloat16>(n, batch, K, N, d, N, 1, n->Wh[l], K, 1, dn, K, 1, nullptr, 0, s)))
        return rc;
      std::swap(d, dn);
    }
  }
  if (update) {
    n->t += 1;
    const float c1 = 1.f - std::pow(0.9f, (float)n->t), c2 = 1.f - std::pow(0.999f, (float)n->t);
    for (int l = 0; l < L; ++l) {
      const int64_t nw = (int64_t)n->w[l] * n->w[l + 1];
      k_adam<<<nb(nw), 256, 0, s>>>(n->W[l], n->gW[l], n->mW[l], n->vW[l], nw, lr, c1, c2, n->Wh[l]);
      k_adam<<<nb(n->w[l + 1]), 256, 0, s>>>(n->b[l], n->gb[l], n->mb[l], n->vb[l], n->w[l + 1], lr, c1, c2, nullptr);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return SHBIM_ERR_CUDA;
  if (loss_host) {
    if (cudaMemcpyAsync(loss_host, n->loss, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return SHBIM_ERR_CUDA;
  }
  return SHBIM_OK;
}

int shbim_electric_warm_start(shbim_ctx* ctx, shbim_mlp* n, const double* xcoef_dev, const double* rhs_dev,
                              double* x0_dev, void* stream) {
  if (!ctx || !n || !xcoef_dev || !rhs_dev || !x0_dev) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (n->w[0] != 3 * ctx->ncoef || n->w[n->L] != ctx->ncoef)
    return fail(ctx, SHBIM_ERR_ARG, "network widths do not match 3 ncoef inputs and ncoef outputs");
  cudaStream_t s = (cudaStream_t)stream;
  float* feat = n->dA;  // [1][3 ncoef] as the network input
  k_to_f32<<<nb(3 * ctx->ncoef), 256, 0, s>>>(xcoef_dev, feat, 3 * ctx->ncoef);
  SHBIM_CHECK_LAUNCH(ctx, "k_to_f32");
  int rc = forward(n, 1, input_of(n, 1, feat, s), s);
  if (rc) return cuda_fail(ctx, cudaGetLastError(), "mlp forward");
  const double R = ctx->opts.R;
  // spherical baseline E_n = 3R/(R+2) E.n, i.e. 3(R+1)/(R+2) times the right-hand side
  k_warm<<<nb(ctx->ncoef), 256, 0, s>>>(n->H[n->L], rhs_dev, 3.0 * (R + 1.0) / (R + 2.0), x0_dev, ctx->ncoef);
  SHBIM_CHECK_LAUNCH(ctx, "k_warm");
  return SHBIM_OK;
}

int64_t shbim_warm_start_feature_count(shbim_ctx* ctx) {
  if (!ctx || ctx->n_drops == 0) return -1;
  return 4 * ctx->ncoef + 7 + ctx->n_drops;
}

int shbim_warm_start_features(shbim_ctx* ctx, const double* xcoef_dev, const double* gamma_dev,
                              const shbim_phys* phys, float* feat_dev, void* stream) {
  if (!ctx || !xcoef_dev || !gamma_dev || !phys || !feat_dev) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nc = ctx->ncoef;
  k_to_f32<<<nb(3 * nc), 256, 0, s>>>(xcoef_dev, feat_dev, 3 * nc);
  SHBIM_CHECK_LAUNCH(ctx, "k_to_f32");
  k_to_f32<<<nb(nc), 256, 0, s>>>(gamma_dev, feat_dev + 3 * nc, nc);
  SHBIM_CHECK_LAUNCH(ctx, "k_to_f32");
  k_feature_tail<<<1, 128, 0, s>>>(feat_dev + 4 * nc, phys->E_u[0], phys->E_u[1], phys->E_u[2], phys->E_q,
                                   ctx->lamm1_dev, ctx->n_drops, phys->R, phys->Q, phys->Ca_E);
  SHBIM_CHECK_LAUNCH(ctx, "k_feature_tail");
  return SHBIM_OK;
}

int shbim_learned_guess(shbim_ctx* ctx, shbim_mlp* n, const float* feat_dev, const double* rhs_e_dev, double* En0_dev,
                        double* u0_dev, void* stream) {
  if (!ctx || !n || !feat_dev) return SHBIM_ERR_ARG;
  if (ctx->n_drops == 0) return fail(ctx, SHBIM_ERR_ARG, "no drops set");
  if (En0_dev && !rhs_e_dev) return fail(ctx, SHBIM_ERR_ARG, "the electric guess needs the right-hand side");
  if (n->w[0] != shbim_warm_start_feature_count(ctx) || n->w[n->L] != 4 * ctx->ncoef)
    return fail(ctx, SHBIM_ERR_ARG, "network widths do not match the warm-start features and 4 ncoef outputs");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(n, 1, input_of(n, 1, feat_dev, s), s);
  if (rc) return cuda_fail(ctx, cudaGetLastError(), "mlp forward");
  ctx->launches += 2 * n->L;
  const double R = ctx->opts.R;
  k_guess<<<nb(4 * ctx->ncoef), 256, 0, s>>>(n->H[n->L], rhs_e_dev, 3.0 * (R + 1.0) / (R + 2.0), En0_dev, u0_dev,
                                              ctx->ncoef);
  SHBIM_CHECK_LAUNCH(ctx, "k_guess");
  return SHBIM_OK;
}

int shbim_set_warm_start(shbim_ctx* ctx, shbim_mlp* n) {
  if (!ctx) return SHBIM_ERR_ARG;
  ctx->warm_net = n;
  return SHBIM_OK;
}

}  // extern "C"
