// Throughput probes of the SM pipes the hot path runs on: FP32 FMA (the compensated all-pairs
// sums), FP64 FMA (transforms, rotations, singular rows), the MUFU reciprocal square root (one per
// pair), and the warp-level tensor instructions mma.sync m16n8k16 bf16 -> f32 and m8n8k4 f64.
// A measurement utility for the roofline denominators; the paper has no counterpart.
//
// Every thread runs kChains independent dependency chains so that instruction issue, not
// latency, bounds the rate; the chains end in a store per thread so nothing is optimised away.
#include <cuda_bf16.h>

#include "internal.h"
#include "tc.cuh"

namespace shbim {
namespace {

constexpr int kChains = 8;
constexpr int kThreadsProbe = 256;

__global__ void __launch_bounds__(kThreadsProbe) k_probe_ffma(int64_t iters, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  const float m = 0.9999999f, b = 1e-7f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreadsProbe) k_probe_dfma(int64_t iters, float* __restrict__ sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  const double m = 0.9999999, b = 1e-7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(kThreadsProbe) k_probe_rsqrt(int64_t iters, float* __restrict__ sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = 1.0f + 1e-3f * (threadIdx.x + c);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = rsqrtf(a[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D = A B + D with fragments held in registers (values are irrelevant to the rate)
__global__ void __launch_bounds__(kThreadsProbe) k_probe_hmma(int64_t iters, float* __restrict__ sink) {
  const uint32_t a0 = 0x3f803f80u + threadIdx.x, a1 = 0x3f003f00u, a2 = 0x3e803e80u, a3 = 0x3f403f40u;
  const uint32_t b0 = 0x3f803f80u, b1 = 0x3e003e00u + threadIdx.x;
  float d[kChains][4];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) d[c][r] = 0.f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};\n"
          : "+f"(d[c][0]), "+f"(d[c][1]), "+f"(d[c][2]), "+f"(d[c][3])
          : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreadsProbe) k_probe_dmma(int64_t iters, float* __restrict__ sink) {
  const double a = 1.0 + 1e-6 * threadIdx.x, b = 0.5;
  double d[kChains][2];
#pragma unroll
  for (int c = 0; c < kChains; ++c) d[c][0] = d[c][1] = 0.0;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(d[c][0]), "+d"(d[c][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += d[c][0] + d[c][1];
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

}  // namespace
}  // namespace shbim

using namespace shbim;

extern "C" int shbim_probe_peak(int kind, int64_t iters, double* ops_per_s_host, double* ms_host, void* stream) {
  if (!ops_per_s_host || iters < 1 || kind < 0 || kind > SHBIM_PROBE_DMMA_F64) return SHBIM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SHBIM_ERR_CUDA;
  const int blocks = nsm * 4;
  const int64_t threads = (int64_t)blocks * kThreadsProbe;
  float* sink = nullptr;
  if (cudaMalloc(&sink, threads * sizeof(float)) != cudaSuccess) return SHBIM_ERR_NOMEM;
  // operations per thread per outer iteration
  double per = 0.0;
  auto launch = [&](int64_t it) {
    switch (kind) {
      case SHBIM_PROBE_FFMA: k_probe_ffma<<<blocks, kThreadsProbe, 0, s>>>(it, sink); per = 2.0 * 8 * kChains; break;
      case SHBIM_PROBE_DFMA: k_probe_dfma<<<blocks, kThreadsProbe, 0, s>>>(it, sink); per = 2.0 * 8 * kChains; break;
      case SHBIM_PROBE_RSQRT: k_probe_rsqrt<<<blocks, kThreadsProbe, 0, s>>>(it, sink); per = 8.0 * kChains; break;
      case SHBIM_PROBE_HMMA_BF16:
        // one warp instruction = 2 * 16 * 8 * 16 flops, shared by its 32 threads
        k_probe_hmma<<<blocks, kThreadsProbe, 0, s>>>(it, sink); per = 2.0 * 16 * 8 * 16 * kChains / 32.0; break;
      default:
        k_probe_dmma<<<blocks, kThreadsProbe, 0, s>>>(it, sink); per = 2.0 * 8 * 8 * 4 * kChains / 32.0; break;
    }
  };
  cudaEvent_t a = nullptr, b = nullptr;
  int rc = SHBIM_OK;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) rc = SHBIM_ERR_CUDA;
  if (!rc) {
    launch(std::max<int64_t>(1, iters / 10));  // warm-up (clocks, instruction cache)
    cudaEventRecord(a, s);
    launch(iters);
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = SHBIM_ERR_CUDA;
  }
  if (!rc) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    *ops_per_s_host = per * (double)iters * (double)threads / (ms / 1e3);
    if (ms_host) *ms_host = ms;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(sink);
  return rc;
}

namespace shbim {
namespace {

// one thread waits on a fresh mbarrier (expected arrivals: 1) with the bounded wait of the
// tensor-core kernels; the arrival is made first or not at all
__global__ void k_wait_check(int arrive, uint64_t limit_ns, int* __restrict__ flag) {
  __shared__ __align__(8) uint64_t bar;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;\n");
  if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(&bar)) : "memory");
  if (!tc::mbar_wait(&bar, 0, limit_ns)) *flag = 1;
}

}  // namespace
}  // namespace shbim

extern "C" int shbim_check_wait(shbim_ctx* ctx, int arrive, void* stream) {
  if (!ctx) return SHBIM_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) return fail(ctx, SHBIM_ERR_NOMEM, "cudaMalloc wait flag");
  int h = 0, rc = SHBIM_OK;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_wait_check<<<1, 1, 0, s>>>(arrive, ctx->wait_ns, flag);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) rc = cuda_fail(ctx, e, "wait check");
  else if (h) rc = fail(ctx, SHBIM_ERR_TIMEOUT, "wait check: the bounded wait ran out");
  ctx->launches++;
  cudaFree(flag);
  return rc;
}
