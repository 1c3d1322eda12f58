// Plain FP64 dot product: the comparator of the paper's approximation
// speedup (eq. approx-speedup: double-precision dot time / qdot time).
// Grid-stride over 128-bit loads with four independent fused multiply-add
// chains per thread, per-CTA partials, and a one-CTA final sum in a fixed
// order (deterministic for a given launch shape).
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

constexpr int kDotThreads = 256;
constexpr int kDotMaxGrid = 4096;

__global__ void __launch_bounds__(kDotThreads) k_dot(const double* __restrict__ x, const double* __restrict__ y,
                                                     long long n, double* __restrict__ part) {
  __shared__ double s[kDotThreads / 32];
  double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  const long long stride = (long long)gridDim.x * kDotThreads;
  long long i = (long long)blockIdx.x * kDotThreads + threadIdx.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0;
  if (vec) {
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const double2* y2 = reinterpret_cast<const double2*>(y);
    const long long n2 = n / 2;
    for (; i + stride < n2; i += 2 * stride) {
      double2 p = __ldcs(x2 + i), q = __ldcs(y2 + i);
      double2 r = __ldcs(x2 + i + stride), t = __ldcs(y2 + i + stride);
      a0 = fma(p.x, q.x, a0);
      a1 = fma(p.y, q.y, a1);
      a2 = fma(r.x, t.x, a2);
      a3 = fma(r.y, t.y, a3);
    }
    for (; i < n2; i += stride) {
      double2 p = __ldcs(x2 + i), q = __ldcs(y2 + i);
      a0 = fma(p.x, q.x, a0);
      a1 = fma(p.y, q.y, a1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) a2 = fma(x[n - 1], y[n - 1], a2);
  } else {
    for (; i < n; i += stride) a0 = fma(__ldcs(x + i), __ldcs(y + i), a0);
  }
  double v = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int w = 0; w < kDotThreads / 32; ++w) t += s[w];
    part[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(32) k_dot_final(const double* __restrict__ part, int np, double* __restrict__ out) {
  double v = 0;
  for (int i = threadIdx.x; i < np; i += 32) v += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

}  // namespace

size_t dot_fp64_workspace() { return sizeof(double) * kDotMaxGrid; }

cudaError_t launch_dot_fp64(const double* x, const double* y, int64_t n, double* out, void* ws, cudaStream_t st) {
  const DeviceInfo& di = device_info();
  int grid = (di.sms > 0 ? di.sms : 152) * 4;  // 1024 threads per SM, two loads in flight each
  if (grid > kDotMaxGrid) grid = kDotMaxGrid;
  double* part = static_cast<double*>(ws);
  k_dot<<<grid, kDotThreads, 0, st>>>(x, y, n, part);
  k_dot_final<<<1, 32, 0, st>>>(part, grid, out);
  return cudaGetLastError();
}

}  // namespace qd
