// Backward of z = qdot(x, y) with the forward's class map held fixed.
//
// With the classes frozen, z = sum_i q_c(x_i) q_c(y_i) over the components
// whose class c keeps them (half / single / double); read straight-through
// (each quantizer's derivative taken as 1), dz/dx_i = q_c(y_i) and
// dz/dy_i = q_c(x_i), and 0 for perforated and zero components.  With an
// upstream gradient g: gx_i = g * q_c(y_i), gy_i = g * q_c(x_i), one
// rounding each.
//
// The forward's class map is kept in the form that generates it: the class
// of every bin key (qdot_selection, 4224 bytes) or, for blocked binning, the
// pair (e_max, f) of the forward's result.  A component's class is a function
// of its own exponent key (exact binning, B = 1) or of its block's key
// ceil(log2 M_b) + u_b (Algorithm 2), so the backward re-derives it from the
// operands it reads anyway: 32 bytes of traffic per component (read x, y;
// write gx, gy) and no per-component map in memory.
//
// Layout: a warp walks items of 256 consecutive components.  With 16-byte
// aligned arrays, exact binning, blocks of one and blocks of 16 .. 256 use the
// forward kernels' item layout (k_backward_items, k_backward_batched_items:
// every warp-wide 16-byte access covers whole sectors).  Otherwise, and for
// blocks of 2 .. 8, lane l owns components row*256 + 8l + [0, 8): blocks of
// B <= 8 components sit inside a lane, blocks of 16 <= B <= 256 span B/8
// lanes (segmented shuffles).  Larger blocks take one CTA each (the block is
// read twice, the second time mostly from L2).
#include <algorithm>
#include <string>

#include "qdot_chunk.cuh"
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

constexpr int kBwThreads = 256;
constexpr int kBwVec = 8;
constexpr int kBwRow = 32 * kBwVec;
constexpr int kNoKey = -(1 << 30);

// q_c(v) as a double: v with its significand rounded to nearest-even at the
// class precision (exponent unbounded; a value past the double range is
// +-Inf), 0 for PERF / ZERO.
__device__ __forceinline__ double quantized_value(uint64_t b, int cls) {
  if (cls == kDouble) return __longlong_as_double((long long)b);
  if (cls != kHalf && cls != kSingle) return 0.0;
  if (is_nonfinite(b)) return __longlong_as_double((long long)b);
  if ((b >> 52) & 0x7FFu) {
    // normal: round the fraction field; a carry out of it moves into the
    // exponent field (reaching 0x7FF with a zero fraction = Inf)
    const int k = cls == kHalf ? 42 : 29;
    const uint64_t sign = b & 0x8000000000000000ull;
    const uint64_t mag = b & 0x7FFFFFFFFFFFFFFFull;
    uint64_t t = mag + ((1ull << (k - 1)) - 1ull) + ((mag >> k) & 1ull);
    t &= ~((1ull << k) - 1ull);
    return __longlong_as_double((long long)(sign | t));
  }
  if (is_zero(b)) return 0.0;
  return compose_double((uint32_t)(b >> 63), quantize_sig(significand_of(b), cls), exponent_of(b));
}

__device__ __forceinline__ int lut_index(int score) { return min(max(score - kKeyMin, 0), kKeyCount - 1); }

// vec: p is 16-byte aligned (base is a multiple of 8 components).
__device__ __forceinline__ void load8(const double* __restrict__ p, long long base, long long n, uint64_t (&v)[kBwVec],
                                      bool vec) {
  if (vec && base + kBwVec <= n) {
    const double2* p2 = reinterpret_cast<const double2*>(p + base);
#pragma unroll
    for (int k = 0; k < kBwVec / 2; ++k) {
      const double2 d = __ldcs(p2 + k);
      v[2 * k] = (uint64_t)__double_as_longlong(d.x);
      v[2 * k + 1] = (uint64_t)__double_as_longlong(d.y);
    }
  } else {
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) v[j] = base + j < n ? (uint64_t)__double_as_longlong(__ldcs(p + base + j)) : 0ull;
  }
}

__device__ __forceinline__ void store8(double* __restrict__ p, long long base, long long n, const double (&v)[kBwVec],
                                       bool vec) {
  if (!p) return;
  if (vec && base + kBwVec <= n) {
    double2* p2 = reinterpret_cast<double2*>(p + base);
#pragma unroll
    for (int k = 0; k < kBwVec / 2; ++k) __stcs(p2 + k, make_double2(v[2 * k], v[2 * k + 1]));
  } else {
#pragma unroll
    for (int j = 0; j < kBwVec; ++j)
      if (base + j < n) __stcs(p + base + j, v[j]);
  }
}

// Classes of one lane's 8 components.  LOG2B < 0: exact binning or B = 1
// (class by the component's own key, from the table); 1 <= LOG2B <= 8:
// blocks of 2^LOG2B (class by block key).  The class of a block key k is
// `cls_of(k)`.  Every lane of the warp must call this together.
template <int LOG2B, typename ClassOf>
__device__ __forceinline__ void lane_classes(const uint64_t (&xb)[kBwVec], const uint64_t (&yb)[kBwVec], long long base,
                                             long long n, ClassOf cls_of, int (&cls)[kBwVec]) {
  int key[kBwVec];
  bool nz[kBwVec];
#pragma unroll
  for (int j = 0; j < kBwVec; ++j) {
    nz[j] = base + j < n && !is_zero(xb[j]) && !is_zero(yb[j]);
    key[j] = nz[j] ? exponent_of(xb[j]) + exponent_of(yb[j]) : kNoKey;
  }
  if constexpr (LOG2B < 1) {
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) cls[j] = nz[j] ? cls_of(key[j]) : kZero;
  } else if constexpr (LOG2B <= 3) {
    constexpr int B = 1 << LOG2B;
#pragma unroll
    for (int g0 = 0; g0 < kBwVec; g0 += B) {
      int u = kNoKey;
      unsigned M = 0;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        u = max(u, key[g0 + j]);
        M += nz[g0 + j] ? 1u : 0u;
      }
      const int bc = M ? cls_of(ceil_log2_u32(M) + u) : kZero;
#pragma unroll
      for (int j = 0; j < B; ++j) cls[g0 + j] = nz[g0 + j] ? bc : kZero;
    }
  } else {
    int u = kNoKey;
    unsigned M = 0;
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) {
      u = max(u, key[j]);
      M += nz[j] ? 1u : 0u;
    }
    constexpr int kLanes = 1 << (LOG2B - 3);  // lanes per block: 2 .. 32
#pragma unroll
    for (int o = 1; o < kLanes; o <<= 1) {
      u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
      M += __shfl_xor_sync(0xffffffffu, M, o);
    }
    const int bc = M ? cls_of(ceil_log2_u32(M) + u) : kZero;
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) cls[j] = nz[j] ? bc : kZero;
  }
}

__device__ __forceinline__ void lane_grads(const uint64_t (&xb)[kBwVec], const uint64_t (&yb)[kBwVec],
                                           const int (&cls)[kBwVec], double g, long long base, long long n,
                                           double* __restrict__ gx, double* __restrict__ gy, bool vec) {
  double a[kBwVec];
  if (gx) {
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) a[j] = g * quantized_value(yb[j], cls[j]);
    store8(gx, base, n, a, vec);
  }
  if (gy) {
#pragma unroll
    for (int j = 0; j < kBwVec; ++j) a[j] = g * quantized_value(xb[j], cls[j]);
    store8(gy, base, n, a, vec);
  }
}

// Single problem, exact binning or B <= 256: class from the forward's table.
template <int LOG2B, bool VEC16>
__global__ void __launch_bounds__(kBwThreads, 4) k_backward_rows(const double* __restrict__ x,
                                                             const double* __restrict__ y, long long n,
                                                             const qdot_selection* __restrict__ sel,
                                                             const double* __restrict__ g, double* __restrict__ gx,
                                                             double* __restrict__ gy) {
  __shared__ uint8_t lut[kKeyCount];
  for (int k = threadIdx.x; k < kKeyCount; k += kBwThreads) lut[k] = sel->cls[k];
  __syncthreads();
  const double gv = *g;
  const int lane = threadIdx.x & 31;
  const long long nrows = (n + kBwRow - 1) / kBwRow;
  const long long nwarps = (long long)gridDim.x * (kBwThreads / 32);
  auto cls_of = [&](int k) { return (int)lut[lut_index(k)]; };
  for (long long row = (long long)blockIdx.x * (kBwThreads / 32) + (threadIdx.x >> 5); row < nrows; row += nwarps) {
    const long long base = row * kBwRow + lane * kBwVec;
    uint64_t xb[kBwVec], yb[kBwVec];
    load8(x, base, n, xb, VEC16);
    load8(y, base, n, yb, VEC16);
    int cls[kBwVec];
    lane_classes<LOG2B>(xb, yb, base, n, cls_of, cls);
    lane_grads(xb, yb, cls, gv, base, n, gx, gy, VEC16);
  }
}

// Single problem, blocks larger than 256: one CTA per block at a time.
template <bool VEC16>
__global__ void __launch_bounds__(kBwThreads) k_backward_blocks(const double* __restrict__ x,
                                                               const double* __restrict__ y, long long n, int log2b,
                                                               const qdot_selection* __restrict__ sel,
                                                               const double* __restrict__ g, double* __restrict__ gx,
                                                               double* __restrict__ gy) {
  __shared__ uint8_t lut[kKeyCount];
  __shared__ int s_u[kBwThreads / 32];
  __shared__ unsigned s_m[kBwThreads / 32];
  for (int k = threadIdx.x; k < kKeyCount; k += kBwThreads) lut[k] = sel->cls[k];
  __syncthreads();
  const double gv = *g;
  const long long B = 1ll << log2b;
  const long long nblocks = (n + B - 1) / B;
  for (long long blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const long long lo = blk * B, hi = min(n, lo + B);
    int u = kNoKey;
    unsigned M = 0;
    for (long long base = lo + (long long)threadIdx.x * kBwVec; base < hi; base += (long long)kBwThreads * kBwVec) {
      uint64_t xb[kBwVec], yb[kBwVec];
#pragma unroll
      for (int j = 0; j < kBwVec; ++j) {  // plain loads: the second sweep should find these lines in L2
        xb[j] = base + j < hi ? (uint64_t)__double_as_longlong(x[base + j]) : 0ull;
        yb[j] = base + j < hi ? (uint64_t)__double_as_longlong(y[base + j]) : 0ull;
      }
#pragma unroll
      for (int j = 0; j < kBwVec; ++j) {
        if (!is_zero(xb[j]) && !is_zero(yb[j])) {
          u = max(u, exponent_of(xb[j]) + exponent_of(yb[j]));
          ++M;
        }
      }
    }
    u = warp_max_i32(u);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) M += __shfl_xor_sync(0xffffffffu, M, o);
    if ((threadIdx.x & 31) == 0) {
      s_u[threadIdx.x >> 5] = u;
      s_m[threadIdx.x >> 5] = M;
    }
    __syncthreads();
    u = kNoKey;
    M = 0;
    for (int w = 0; w < kBwThreads / 32; ++w) {
      u = max(u, s_u[w]);
      M += s_m[w];
    }
    __syncthreads();  // s_u / s_m are rewritten by the next block
    const int bc = M ? (int)lut[lut_index(ceil_log2_u32(M) + u)] : kZero;
    for (long long base = lo + (long long)threadIdx.x * kBwVec; base < hi; base += (long long)kBwThreads * kBwVec) {
      uint64_t xb[kBwVec], yb[kBwVec];
      int cls[kBwVec];
#pragma unroll
      for (int j = 0; j < kBwVec; ++j) {
        xb[j] = base + j < hi ? (uint64_t)__double_as_longlong(x[base + j]) : 0ull;
        yb[j] = base + j < hi ? (uint64_t)__double_as_longlong(y[base + j]) : 0ull;
        cls[j] = (base + j < hi && !is_zero(xb[j]) && !is_zero(yb[j])) ? bc : kZero;
      }
      // the block's end is a multiple of 8 components except at the end of x
      lane_grads(xb, yb, cls, gv, base, hi, gx, gy, VEC16);
    }
  }
}

// Batched: the first row (item of 256 components) of every problem, an
// exclusive scan of ceil(n_j / 256) in row_start[0 .. count].
__global__ void k_bw_plan(const int64_t* __restrict__ ns, int count, long long* __restrict__ row_start) {
  // one CTA of 1024 threads: exclusive scan of ceil(n_j / 256)
  __shared__ long long s_tot[1024];
  const int per = (count + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(count, lo + per);
  long long t = 0;
  for (int j = lo; j < hi; ++j) t += (ns[j] > 0 ? (ns[j] + kBwRow - 1) / kBwRow : 0);
  s_tot[threadIdx.x] = t;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = threadIdx.x >= o ? s_tot[threadIdx.x - o] : 0;
    __syncthreads();
    s_tot[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = s_tot[threadIdx.x] - t;
  for (int j = lo; j < hi; ++j) {
    row_start[j] = run;
    run += (ns[j] > 0 ? (ns[j] + kBwRow - 1) / kBwRow : 0);
  }
  if (threadIdx.x == 1023) row_start[count] = s_tot[1023];
}

// ---------------------------------------------------------------------------
// Coalesced kernels (16-byte aligned x, y, gx, gy): warp items of 256
// components in the forward kernels' layout (qdot_chunk.cuh).  Lane l holds
// components item_offset<LB>(l, j), read and written as four 16-byte pieces
// of each array, so every warp-wide access covers whole 32-byte sectors
// (the layout above, 8 consecutive components per lane, touches each sector
// from two instructions).  LB = 8 for exact binning and blocks of one (class
// per component); LB = log2 B for blocks of 16 .. 256 (class per block, the
// block's L = B / 8 lanes reduce u_b and M_b by shuffles).
// ---------------------------------------------------------------------------

// Item `item` of (x, y): 16-byte loads for a whole item when ALIGNED, else
// (and at the vectors' end) one component at a time.
template <int LB>
__device__ __forceinline__ void bw_load(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                        long long item, int lane, bool aligned, chunk::Chunk& ch) {
  if (aligned) {
    chunk::load_item<LB>(x, y, n, item, lane, ch);
    return;
  }
  const long long start = item * chunk::kItem;
  ch.vmask = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long i = start + chunk::item_offset<LB>(lane, j);
    const bool in = i < n;
    ch.vmask |= in ? (1u << j) : 0u;
    ch.x[j] = in ? (uint64_t)__double_as_longlong(x[i]) : 0ull;
    ch.y[j] = in ? (uint64_t)__double_as_longlong(y[i]) : 0ull;
  }
}

template <int LB>
__device__ __forceinline__ void bw_store(double* __restrict__ p, long long n, long long item, int lane, bool aligned,
                                         const double (&v)[8]) {
  if (!p) return;
  constexpr int L = chunk::Map<LB>::L;
  const long long start = item * chunk::kItem;
  if (aligned && start + chunk::kItem <= n) {
    double2* p2 = reinterpret_cast<double2*>(p + start + chunk::item_offset<LB>(lane, 0));
#pragma unroll
    for (int j = 0; j < 4; ++j) __stcs(p2 + L * j, make_double2(v[2 * j], v[2 * j + 1]));
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = start + chunk::item_offset<LB>(lane, j);
      if (i < n) __stcs(p + i, v[j]);
    }
  }
}

// Classes of a lane's 8 components of one item: by the component's key
// (BLOCKS false) or by the block key ceil(log2 M_b) + u_b (BLOCKS true; every
// lane of the warp must call this together).  Components outside the vectors
// or with a zero factor are ZERO.
template <int LB, bool BLOCKS, typename ClassOf>
__device__ __forceinline__ void item_classes(const chunk::Chunk& ch, ClassOf cls_of, int (&cls)[8]) {
  int key[8];
  bool nz[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    nz[j] = ((ch.vmask >> j) & 1u) && !is_zero(ch.x[j]) && !is_zero(ch.y[j]);
    key[j] = nz[j] ? exponent_of(ch.x[j]) + exponent_of(ch.y[j]) : kNoKey;
  }
  if constexpr (!BLOCKS) {
#pragma unroll
    for (int j = 0; j < 8; ++j) cls[j] = nz[j] ? cls_of(key[j]) : kZero;
  } else {
    constexpr int L = chunk::Map<LB>::L;
    int u = kNoKey;
    unsigned M = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      u = max(u, key[j]);
      M += nz[j] ? 1u : 0u;
    }
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
      u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
      M += __shfl_xor_sync(0xffffffffu, M, o);
    }
    const int bc = M ? cls_of(ceil_log2_u32(M) + u) : kZero;
#pragma unroll
    for (int j = 0; j < 8; ++j) cls[j] = nz[j] ? bc : kZero;
  }
}

template <int LB>
__device__ __forceinline__ void item_grads(const chunk::Chunk& ch, const int (&cls)[8], double g, long long n,
                                           long long item, int lane, bool aligned, double* __restrict__ gx,
                                           double* __restrict__ gy) {
  double a[8];
  if (gx) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = g * quantized_value(ch.y[j], cls[j]);
    bw_store<LB>(gx, n, item, lane, aligned, a);
  }
  if (gy) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = g * quantized_value(ch.x[j], cls[j]);
    bw_store<LB>(gy, n, item, lane, aligned, a);
  }
}

// Single problem, exact binning or B in {1, 16, ..., 256}: class from the
// forward's table.
template <int LB, bool BLOCKS>
__global__ void __launch_bounds__(kBwThreads, 4) k_backward_items(const double* __restrict__ x,
                                                              const double* __restrict__ y, long long n,
                                                              const qdot_selection* __restrict__ sel,
                                                              const double* __restrict__ g, double* __restrict__ gx,
                                                              double* __restrict__ gy) {
  __shared__ uint8_t lut[kKeyCount];
  for (int k = threadIdx.x; k < kKeyCount; k += kBwThreads) lut[k] = sel->cls[k];
  __syncthreads();
  const double gv = *g;
  const int lane = threadIdx.x & 31;
  const long long nitems = (n + chunk::kItem - 1) / chunk::kItem;
  const long long nwarps = (long long)gridDim.x * (kBwThreads / 32);
  auto cls_of = [&](int k) { return (int)lut[lut_index(k)]; };
  for (long long it = (long long)blockIdx.x * (kBwThreads / 32) + (threadIdx.x >> 5); it < nitems; it += nwarps) {
    chunk::Chunk ch;
    chunk::load_item<LB>(x, y, n, it, lane, ch);
    int cls[8];
    item_classes<LB, BLOCKS>(ch, cls_of, cls);
    item_grads<LB>(ch, cls, gv, n, it, lane, true, gx, gy);
  }
}

// Batched, blocks of 32 .. 256: problem j's items follow those of problems
// 0 .. j-1 (row_start, rows of 256 = items).  Each warp takes one contiguous
// range of items, finds its first problem by binary search and then walks
// forward; class from the forward's (e_max, f) of each problem.
template <int LB>
__global__ void __launch_bounds__(kBwThreads, 4) k_backward_batched_items(
    const double* const* __restrict__ xs, const double* const* __restrict__ ys, const int64_t* __restrict__ ns,
    int count, const long long* __restrict__ row_start, const qdot_result* __restrict__ outs,
    const double* __restrict__ gs, double* const* __restrict__ gxs, double* const* __restrict__ gys, int mh,
    int ms) {
  const int lane = threadIdx.x & 31;
  const long long total = row_start[count];
  const long long nwarps = (long long)gridDim.x * (kBwThreads / 32);
  const long long gw = (long long)blockIdx.x * (kBwThreads / 32) + (threadIdx.x >> 5);
  const long long per = (total + nwarps - 1) / nwarps;
  const long long r0 = gw * per, r1 = min(total, r0 + per);
  if (r0 >= r1) return;  // warp-uniform
  int lo = 0, hi = count - 1;  // last j with row_start[j] <= r0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (row_start[mid] <= r0) lo = mid; else hi = mid - 1;
  }
  int j = lo;
  long long jend = row_start[j + 1];
  for (long long r = r0; r < r1; ++r) {
    while (r >= jend) {  // next problem with items (empty ones have none)
      ++j;
      jend = row_start[j + 1];
    }
    const double* x = xs[j];
    const double* y = ys[j];
    double* gx = gxs ? gxs[j] : nullptr;
    double* gy = gys ? gys[j] : nullptr;
    const long long n = ns[j];
    const int e_max = outs[j].e_max, f = outs[j].f;
    const bool ok = outs[j].status == QDOT_OK;
    const uintptr_t a = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) |
                        reinterpret_cast<uintptr_t>(gx) | reinterpret_cast<uintptr_t>(gy);
    const bool aligned = (a & 15u) == 0;
    const long long item = r - row_start[j];
    chunk::Chunk ch;
    if (ok) {
      bw_load<LB>(x, y, n, item, lane, aligned, ch);
    } else {
      ch.vmask = 0u;
#pragma unroll
      for (int k = 0; k < 8; ++k) ch.x[k] = ch.y[k] = 0ull;
    }
    int cls[8];
    auto cls_of = [&](int k) { return precision_of((long long)k - e_max - f + 1, mh, ms); };
    item_classes<LB, true>(ch, cls_of, cls);  // every lane joins the shuffles
    if (ok) {
      item_grads<LB>(ch, cls, gs[j], n, item, lane, aligned, gx, gy);
    } else {  // no valid forward selection for this problem
      double nan8[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) nan8[k] = __longlong_as_double(0x7FF8000000000000ll);
      bw_store<LB>(gx, n, item, lane, aligned, nan8);
      bw_store<LB>(gy, n, item, lane, aligned, nan8);
    }
  }
}

template <int LOG2B>
void launch_rows(bool al16, int grid, const double* x, const double* y, long long n, const qdot_selection* sel,
                 const double* g, double* gx, double* gy, cudaStream_t st) {
  if (al16)
    k_backward_rows<LOG2B, true><<<grid, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy);
  else
    k_backward_rows<LOG2B, false><<<grid, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy);
}

int bw_grid(long long units, int per_sm) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  return (int)std::max<long long>(1, std::min<long long>(units, (long long)sms * per_sm));
}

}  // namespace
}  // namespace qd

using namespace qd;

extern "C" {

qdot_status qdot_backward(const double* x, const double* y, int64_t n, const qdot_params* p,
                          const qdot_selection* sel, const double* g, double* gx, double* gy, void* stream) {
  clear_error();
  std::string why;
  if (!valid_params(n, p, &why)) {
    set_error("qdot_backward: " + why);
    return QDOT_ERR_ARG;
  }
  if (n == 0 || (!gx && !gy)) return QDOT_OK;
  if (!x || !y || !sel || !g) {
    set_error("qdot_backward: x, y, sel and g must be device pointers");
    return QDOT_ERR_ARG;
  }
  const uintptr_t a = reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) |
                      reinterpret_cast<uintptr_t>(gx) | reinterpret_cast<uintptr_t>(gy);
  if (a & 7u) {
    set_error("qdot_backward: x, y, gx and gy must be 8-byte aligned");
    return QDOT_ERR_ARG;
  }
  const bool al16 = (a & 15u) == 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long rows = (n + kBwRow - 1) / kBwRow;
  const int grid = bw_grid((rows + 7) / 8, 4);
  const int B = p->block;
  if (al16 && (B <= 1 || (B >= 16 && B <= 256))) {  // coalesced item layout
    const long long items = (n + chunk::kItem - 1) / chunk::kItem;
    const int gi = bw_grid((items + 7) / 8, 4);
    switch (B) {
      case 0:
      case 1: k_backward_items<8, false><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
      case 16: k_backward_items<4, true><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
      case 32: k_backward_items<5, true><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
      case 64: k_backward_items<6, true><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
      case 128: k_backward_items<7, true><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
      default: k_backward_items<8, true><<<gi, kBwThreads, 0, st>>>(x, y, n, sel, g, gx, gy); break;
    }
  } else switch (B) {
    case 0:
    case 1: launch_rows<-1>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 2: launch_rows<1>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 4: launch_rows<2>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 8: launch_rows<3>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 16: launch_rows<4>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 32: launch_rows<5>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 64: launch_rows<6>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 128: launch_rows<7>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    case 256: launch_rows<8>(al16, grid, x, y, n, sel, g, gx, gy, st); break;
    default: {
      const int log2b = 31 - __builtin_clz((unsigned)B);
      const long long nblocks = (n + B - 1) / B;
      const int gb = bw_grid(nblocks, 8);
      if (al16)
        k_backward_blocks<true><<<gb, kBwThreads, 0, st>>>(x, y, n, log2b, sel, g, gx, gy);
      else
        k_backward_blocks<false><<<gb, kBwThreads, 0, st>>>(x, y, n, log2b, sel, g, gx, gy);
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("qdot_backward launch: ") + cudaGetErrorString(e));
    return QDOT_ERR_CUDA;
  }
  return QDOT_OK;
}

size_t qdot_batched_backward_workspace_size(int32_t count) {
  return count < 0 ? 0 : align_up(sizeof(long long) * ((size_t)count + 1), 256);
}

qdot_status qdot_batched_backward(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                                  const qdot_params* p, const qdot_result* outs, const double* gs, double* const* gxs,
                                  double* const* gys, int32_t grid_ctas, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  std::string why;
  if (!valid_params(0, p, &why)) {
    set_error("qdot_batched_backward: " + why);
    return QDOT_ERR_ARG;
  }
  if (p->block < 32 || p->block > 256) {
    set_error("qdot_batched_backward: block must be 32, 64, 128 or 256");
    return QDOT_ERR_ARG;
  }
  if (count < 0 || grid_ctas < 0) {
    set_error("qdot_batched_backward: count and grid_ctas must be >= 0");
    return QDOT_ERR_ARG;
  }
  if (count == 0 || (!gxs && !gys)) return QDOT_OK;
  if (!xs || !ys || !ns || !outs || !gs) {
    set_error("qdot_batched_backward: xs, ys, ns, outs and gs must be device pointers");
    return QDOT_ERR_ARG;
  }
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < qdot_batched_backward_workspace_size(count)) {
    set_error("qdot_batched_backward: workspace missing, misaligned or too small");
    return QDOT_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  long long* row_start = static_cast<long long*>(ws);
  const int mh = p->mant_reading ? 11 : 10, ms = p->mant_reading ? 24 : 23;
  const int grid = grid_ctas > 0 ? grid_ctas : bw_grid(1ll << 40, 4);
  k_bw_plan<<<1, 1024, 0, st>>>(ns, count, row_start);
  switch (p->block) {
    case 32: k_backward_batched_items<5><<<grid, kBwThreads, 0, st>>>(xs, ys, ns, count, row_start, outs, gs, gxs, gys, mh, ms); break;
    case 64: k_backward_batched_items<6><<<grid, kBwThreads, 0, st>>>(xs, ys, ns, count, row_start, outs, gs, gxs, gys, mh, ms); break;
    case 128: k_backward_batched_items<7><<<grid, kBwThreads, 0, st>>>(xs, ys, ns, count, row_start, outs, gs, gxs, gys, mh, ms); break;
    default: k_backward_batched_items<8><<<grid, kBwThreads, 0, st>>>(xs, ys, ns, count, row_start, outs, gs, gxs, gys, mh, ms); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error(std::string("qdot_batched_backward launch: ") + cudaGetErrorString(e));
    return QDOT_ERR_CUDA;
  }
  return QDOT_OK;
}

}  // extern "C"
