// Allocation-free variant of the RED update with its step-norm reductions.
//
// Some callers cannot call cudaMalloc: code running inside another framework
// that owns all device memory through its own allocator, a process whose
// memory budget was fixed up front, or an inference server that must not
// allocate once it is serving.  For them ideq_red_update_noalloc takes only
// caller-owned inputs and outputs; the per-block FP64 partial sums that the
// context-based path keeps in its workspace live here in one file-scope device
// array of fixed size, which every GPU that loads this library holds until the
// process exits.
#include <mutex>

#include "common.cuh"
#include "ideq_internal.h"

namespace ideq {

// Scratch of the allocation-free update: 2 partial sums (||x_new - x||^2 and
// ||x||^2) for every (image, block) pair.  65536 doubles = 512 KiB per device.
constexpr int kNoallocMaxPartials = 65536;
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxPartials];

// Host-side table of the array's device address, one entry per device ordinal
// (the symbol's host-side name is not a device address).
constexpr int kMaxDevices = 64;
static double* g_noalloc_addr[kMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

static cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);  // with `dev` current
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

// Sum each image's block partials in a fixed order (one warp per image).
__global__ void noalloc_norms_kernel(int n, int nblk, const double* __restrict__ part,
                                     double* __restrict__ step_sq, double* __restrict__ x_sq) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= n) return;
  const double* ps = part;
  const double* px = part + (size_t)n * nblk;
  double s = 0.0, x = 0.0;
  for (int i = lane; i < nblk; i += 32) {
    s += ps[(size_t)b * nblk + i];
    x += px[(size_t)b * nblk + i];
  }
  s = warp_sum(s);
  x = warp_sum(x);
  if (lane == 0) {
    if (step_sq) step_sq[b] = s;
    if (x_sq) x_sq[b] = x;
  }
}

}  // namespace ideq

using namespace ideq;

extern "C" ideq_status ideq_red_update_noalloc(int n, int per_img, const float* z,
                                               const float* grad_f, const float* grad_g,
                                               const float* x, float* x_new, float lambda,
                                               float tau, double* step_sq, double* x_sq,
                                               void* stream) {
  (void)cudaGetLastError();  // clear a stale error an unrelated earlier call may have left
  if (n <= 0 || per_img <= 0 || !z || !grad_f || !grad_g || !x || !x_new) return IDEQ_ERR_ARG;
  const int nblk = update_blocks_per_image(per_img);
  if ((long long)n * nblk * 2 > kNoallocMaxPartials) return IDEQ_ERR_ARG;  // scratch too small
  double* part = nullptr;
  if (noalloc_scratch(&part) != cudaSuccess) return IDEQ_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  // every (image, block) slot is written by the update before it is read, so
  // nothing in the shared array needs clearing between calls
  if (launch_red_update(n, per_img, nblk, z, grad_f, grad_g, x, x_new, lambda, tau, nullptr,
                        part, part + (size_t)n * nblk, st) != cudaSuccess)
    return IDEQ_ERR_CUDA;
  noalloc_norms_kernel<<<(n + 3) / 4, 128, 0, st>>>(n, nblk, part, step_sq, x_sq);
  if (cudaGetLastError() != cudaSuccess) return IDEQ_ERR_CUDA;
  return IDEQ_OK;
}
