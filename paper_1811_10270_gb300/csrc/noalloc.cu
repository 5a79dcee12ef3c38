// Allocation-free Laplace pair sum (shbim_pairs_laplace_noalloc).
//
// Same arithmetic as the FP64 all-pairs kernel of pairs.cu -- targets in tiles of 256, the
// sources split across CTAs, one partial sum per (split, target), then a reduction over the
// splits in a fixed order -- but for plain caller-supplied target and source arrays, with the
// partial sums kept in a fixed-size array in device global memory instead of a buffer the
// library allocates. It serves callers that must not allocate device memory at call time.
//
// The host-side name of a __device__ array is only a stand-in, not a device address: the
// address is obtained once per device with cudaGetSymbolAddress (with that device current)
// and passed to the kernels as a plain pointer.
#include <mutex>

#include "internal.h"

namespace shbim {
namespace {

constexpr int64_t kScratchDoubles = int64_t(1) << 21;  // 16 MiB of partial sums per device
constexpr int kMaxDevices = 64;
constexpr int kTileT = 256;
constexpr int kTileS = 256;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up on first use).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SHBIM_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SHBIM_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SHBIM_ERR_CUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return SHBIM_OK;
}

template <int KIND>  // 0: double layer with target normal, 1: single layer
__global__ void __launch_bounds__(128)
k_pairs_noalloc(const double* __restrict__ tgt, int64_t nt, const double* __restrict__ src, int64_t ns,
                int nsplit, double* __restrict__ scratch) {
  __shared__ double sh[4][kTileS];
  const int64_t chunk = (ns + nsplit - 1) / nsplit;
  const int64_t s0 = (int64_t)blockIdx.y * chunk;
  const int64_t s1 = min(ns, s0 + chunk);
  int64_t tg[2];
  bool ok[2];
  double X[2][3], Nn[2][3], acc[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    tg[k] = (int64_t)blockIdx.x * kTileT + threadIdx.x + k * 128;
    ok[k] = tg[k] < nt;
    const int64_t t = ok[k] ? tg[k] : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      X[k][c] = tgt[c * nt + t];
      Nn[k][c] = tgt[(3 + c) * nt + t];
    }
    acc[k] = 0.0;
  }
  for (int64_t base = s0; base < s1; base += kTileS) {
    const int cnt = (int)min((int64_t)kTileS, s1 - base);
    __syncthreads();
    for (int e = threadIdx.x; e < cnt; e += 128) {
#pragma unroll
      for (int c = 0; c < 4; ++c) sh[c][e] = src[c * ns + base + e];
    }
    __syncthreads();
    for (int e = 0; e < cnt; ++e) {
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const double dx = X[k][0] - sh[0][e], dy = X[k][1] - sh[1][e], dz = X[k][2] - sh[2][e];
        const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
        if (KIND == 1) {
          acc[k] = fma(sh[3][e], ri, acc[k]);
        } else {
          const double dn = dx * Nn[k][0] + dy * Nn[k][1] + dz * Nn[k][2];
          acc[k] = fma(sh[3][e] * ri * ri * ri, dn, acc[k]);
        }
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
    if (ok[k]) scratch[(int64_t)blockIdx.y * nt + tg[k]] = 0.07957747154594766788 * acc[k];
}

__global__ void k_reduce_noalloc(const double* __restrict__ scratch, int nsplit, int64_t nt,
                                 double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += scratch[(int64_t)k * nt + t];
  out[t] = s;
}

}  // namespace
}  // namespace shbim

using namespace shbim;

extern "C" int shbim_pairs_laplace_noalloc(int which, const double* tgt_dev, int64_t n_tgt,
                                           const double* src_dev, int64_t n_src, double* out_dev,
                                           void* stream) {
  // an error left pending by earlier, unrelated work belongs to that work: report it without
  // launching (and without clearing it), so it is not taken for this call's own failure
  if (cudaPeekAtLastError() != cudaSuccess) return SHBIM_ERR_CUDA;
  if (which != SHBIM_LAPLACE_DL && which != SHBIM_LAPLACE_SL) return SHBIM_ERR_ARG;
  if (n_tgt < 0 || n_src < 0) return SHBIM_ERR_ARG;
  if (n_tgt > kScratchDoubles) return SHBIM_ERR_ARG;
  if (n_tgt == 0) return SHBIM_OK;
  if (!tgt_dev || !out_dev || (n_src > 0 && !src_dev)) return SHBIM_ERR_ARG;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t tiles = (n_tgt + kTileT - 1) / kTileT;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    return SHBIM_ERR_CUDA;
  int64_t splits = ((int64_t)nsm * 8 + tiles - 1) / tiles;
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, n_src / kTileS));
  splits = std::min<int64_t>(splits, kScratchDoubles / n_tgt);
  splits = std::max<int64_t>(1, std::min<int64_t>(splits, 256));
  dim3 grid((unsigned)tiles, (unsigned)splits);
  if (which == SHBIM_LAPLACE_SL)
    k_pairs_noalloc<1><<<grid, 128, 0, s>>>(tgt_dev, n_tgt, src_dev, n_src, (int)splits, scratch);
  else
    k_pairs_noalloc<0><<<grid, 128, 0, s>>>(tgt_dev, n_tgt, src_dev, n_src, (int)splits, scratch);
  if (cudaGetLastError() != cudaSuccess) return SHBIM_ERR_CUDA;
  k_reduce_noalloc<<<(unsigned)((n_tgt + 255) / 256), 256, 0, s>>>(scratch, (int)splits, n_tgt, out_dev);
  if (cudaGetLastError() != cudaSuccess) return SHBIM_ERR_CUDA;
  return SHBIM_OK;
}
