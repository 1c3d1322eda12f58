// Two-pass qdot (Algorithm 3 = Algorithm 2 then Algorithm 1), any binning.
//
//   pass 1  k_stats   one read of x, y: exponent keys e_i = e(x_i) + e(y_i)
//                     (Algorithm 2, exponent preprocessing), e_max / e_min,
//                     N_bins, and the bin cardinalities the mode needs
//                     (exact binning: key histogram; large blocks: block keys).
//   select  k_select  one CTA: f = floor(log2(eps / N_bins)) exactly, bin
//                     score (eq. bin-score-def) and precision (eq.
//                     precision-def) of every key -> a 4224-entry class table.
//   pass 2  k_apply   second read: class of each component from the table,
//                     significands rounded to nearest-even at the class
//                     precision, exact products summed in a 128-bit fixed-point
//                     accumulator anchored at 2^(e_max - L) (Algorithm 1).
//           k_explain the same, writing class / q(x) / q(y) per component.
//   final   k_final   one CTA: exact sum of the per-CTA partials, one rounding.
//
// Each warp walks rows of 32*VEC consecutive components; lane l owns
// components row*32*VEC + l*VEC + [0, VEC).  Blocks of B <= 32*VEC components
// are lane segments (segmented warp reductions); larger blocks are processed
// one block per warp.
#include <climits>

#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kNeutralMax = -(1 << 30);
constexpr int kNeutralMin = (1 << 30);
constexpr int16_t kEmptyBlock = INT16_MIN;

struct StatsRec {
  int e_max, e_min;
  long long nbins, zeros;
  int nonfinite, pad;
};
struct ApplyRec {
  i128 sum;
  unsigned long long cnt[4];
};
struct Header {
  int L, lsb;         // fixed-point bits and anchor exponent of the accumulator
  long long zeros;    // ZERO components
  int status, nonfinite;
  int pad[2];
};

template <int VEC>
struct Row {
  uint64_t xb[VEC], yb[VEC];
  bool valid[VEC];
};

template <int VEC, bool STREAM>
__device__ __forceinline__ void load_row(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                         long long row, int lane, Row<VEC>& r) {
  long long base = row * (32 * VEC) + (long long)lane * VEC;
  if (base + VEC <= n) {
    if (VEC == 2) {
      double2 a, b;
      if (STREAM) {
        a = __ldcs(reinterpret_cast<const double2*>(x + base));
        b = __ldcs(reinterpret_cast<const double2*>(y + base));
      } else {
        a = __ldg(reinterpret_cast<const double2*>(x + base));
        b = __ldg(reinterpret_cast<const double2*>(y + base));
      }
      r.xb[0] = (uint64_t)__double_as_longlong(a.x);
      r.yb[0] = (uint64_t)__double_as_longlong(b.x);
      r.xb[VEC - 1] = (uint64_t)__double_as_longlong(a.y);
      r.yb[VEC - 1] = (uint64_t)__double_as_longlong(b.y);
    } else {
      r.xb[0] = (uint64_t)__double_as_longlong(STREAM ? __ldcs(x + base) : __ldg(x + base));
      r.yb[0] = (uint64_t)__double_as_longlong(STREAM ? __ldcs(y + base) : __ldg(y + base));
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) r.valid[j] = true;
  } else {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      r.valid[j] = base + j < n;
      r.xb[j] = r.valid[j] ? (uint64_t)__double_as_longlong(__ldg(x + base + j)) : 0ull;
      r.yb[j] = r.valid[j] ? (uint64_t)__double_as_longlong(__ldg(y + base + j)) : 0ull;
    }
  }
}

struct Decoded {
  bool nz;        // component belongs to a bin (valid, x != 0, y != 0)
  bool bad;       // NaN / Inf seen
  bool zero;      // valid ZERO component
  int key;        // e_i (valid when nz)
};

__device__ __forceinline__ Decoded decode(uint64_t xb, uint64_t yb, bool valid) {
  Decoded d;
  d.bad = valid && (is_nonfinite(xb) || is_nonfinite(yb));
  bool zx = is_zero(xb), zy = is_zero(yb);
  d.nz = valid && !zx && !zy && !d.bad;
  d.zero = valid && (zx || zy) && !d.bad;
  d.key = d.nz ? exponent_of(xb) + exponent_of(yb) : kNeutralMax;
  return d;
}

// Segmented (u, M) over lane groups of `lanes` lanes (power of two).
__device__ __forceinline__ void segment_reduce(int& u, int& M, int lanes) {
  for (int o = 1; o < lanes; o <<= 1) {
    u = max(u, __shfl_xor_sync(0xffffffffu, u, o));
    M += __shfl_xor_sync(0xffffffffu, M, o);
  }
}

// ---------------------------------------------------------------------------
// Pass 1
// ---------------------------------------------------------------------------
// Components of a row are "plain" when each of x_i, y_i is a normal double or
// zero; for plain rows the key is read from the exponent fields directly
// (e_i + 2046 = biased(x_i) + biased(y_i)), otherwise the general decoder runs.
__device__ __forceinline__ bool plain_pair(uint64_t a, uint64_t b) {
  const uint32_t ha = (uint32_t)(a >> 32), hb = (uint32_t)(b >> 32);
  const bool za = ((ha & 0x7FFFFFFFu) | (uint32_t)a) == 0u, zb = ((hb & 0x7FFFFFFFu) | (uint32_t)b) == 0u;
  return ((ha & 0x7FF00000u) - 0x00100000u < 0x7FE00000u || za) &&
         ((hb & 0x7FF00000u) - 0x00100000u < 0x7FE00000u || zb);
}

template <bool GENERAL>
__device__ __forceinline__ Decoded decode_fast(uint64_t xb, uint64_t yb, bool valid) {
  if (GENERAL) return decode(xb, yb, valid);
  Decoded d;
  const uint32_t hx = (uint32_t)(xb >> 32), hy = (uint32_t)(yb >> 32);
  const bool z = (((hx & 0x7FFFFFFFu) | (uint32_t)xb) == 0u) || (((hy & 0x7FFFFFFFu) | (uint32_t)yb) == 0u);
  d.bad = false;
  d.nz = valid && !z;
  d.zero = valid && z;
  d.key = d.nz ? (int)(((hx & 0x7FF00000u) + (hy & 0x7FF00000u)) >> 20) - 2046 : kNeutralMax;
  return d;
}

template <int MODE, int VEC, bool GENERAL>
__device__ __forceinline__ void stats_row(const Row<VEC>& rw, int lane, int seg_lanes, int& emax, int& emin,
                                          long long& nb, long long& zeros, int& bad, unsigned int* s_hist) {
  int u = kNeutralMax, M = 0;
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    Decoded d = decode_fast<GENERAL>(rw.xb[j], rw.yb[j], rw.valid[j]);
    bad |= d.bad;
    zeros += d.zero;
    if (d.nz) {
      emin = min(emin, d.key);
      u = max(u, d.key);
      M += 1;
      if (MODE == kModeExact) atomicAdd(&s_hist[d.key - kKeyMin], 1u);
    }
  }
  emax = max(emax, u);
  if (MODE == kModeBlock1) nb += M;
  if (MODE == kModeBlockSmall) {
    segment_reduce(u, M, seg_lanes);
    if ((lane & (seg_lanes - 1)) == 0) nb += (M > 0);
  }
}

template <int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, 4) k_stats(const double* __restrict__ x, const double* __restrict__ y,
                                                    long long n, int log2b, StatsRec* __restrict__ recs,
                                                    unsigned long long* __restrict__ hist,
                                                    int16_t* __restrict__ bkeys) {
  __shared__ unsigned int s_hist[MODE == kModeExact ? kKeyCount : 1];
  __shared__ StatsRec s_part[kWarps];
  if (MODE == kModeExact) {
    for (int i = threadIdx.x; i < kKeyCount; i += kThreads) s_hist[i] = 0;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kThreads) >> 5;
  constexpr int R = 32 * VEC;
  int emax = kNeutralMax, emin = kNeutralMin;
  long long nb = 0, zeros = 0;
  int bad = 0;

  if (MODE != kModeBlockLarge) {
    const long long nrows = (n + R - 1) / R;
    const int seg_lanes = (MODE == kModeBlockSmall) ? ((1 << log2b) / VEC) : 1;
    long long row = gwarp;
    // two rows in flight per warp
    for (; row + nwarps < nrows; row += 2 * nwarps) {
      Row<VEC> r0, r1;
      load_row<VEC, false>(x, y, n, row, lane, r0);
      load_row<VEC, false>(x, y, n, row + nwarps, lane, r1);
      bool plain = true;
#pragma unroll
      for (int j = 0; j < VEC; ++j) plain &= plain_pair(r0.xb[j], r0.yb[j]) && plain_pair(r1.xb[j], r1.yb[j]);
      if (__all_sync(0xffffffffu, plain)) {
        stats_row<MODE, VEC, false>(r0, lane, seg_lanes, emax, emin, nb, zeros, bad, s_hist);
        stats_row<MODE, VEC, false>(r1, lane, seg_lanes, emax, emin, nb, zeros, bad, s_hist);
      } else {
        stats_row<MODE, VEC, true>(r0, lane, seg_lanes, emax, emin, nb, zeros, bad, s_hist);
        stats_row<MODE, VEC, true>(r1, lane, seg_lanes, emax, emin, nb, zeros, bad, s_hist);
      }
    }
    for (; row < nrows; row += nwarps) {
      Row<VEC> r0;
      load_row<VEC, false>(x, y, n, row, lane, r0);
      stats_row<MODE, VEC, true>(r0, lane, seg_lanes, emax, emin, nb, zeros, bad, s_hist);
    }
  } else {
    const long long B = 1ll << log2b;
    const long long nblk = (n + B - 1) / B;
    const long long rows_per_block = B / R;
    for (long long blk = gwarp; blk < nblk; blk += nwarps) {
      int u = kNeutralMax, M = 0;
      for (long long rr = 0; rr < rows_per_block; ++rr) {
        long long row = blk * rows_per_block + rr;
        if (row * R >= n) break;
        Row<VEC> rw;
        load_row<VEC, false>(x, y, n, row, lane, rw);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          Decoded d = decode(rw.xb[j], rw.yb[j], rw.valid[j]);
          bad |= d.bad;
          zeros += d.zero;
          if (d.nz) {
            emax = max(emax, d.key);
            emin = min(emin, d.key);
            u = max(u, d.key);
            M += 1;
          }
        }
      }
      u = __reduce_max_sync(0xffffffffu, u);
      M = (int)__reduce_add_sync(0xffffffffu, (unsigned)M);
      if (lane == 0) {
        nb += (M > 0);
        bkeys[blk] = M > 0 ? (int16_t)(ceil_log2_u32((uint32_t)M) + u) : kEmptyBlock;
      }
    }
  }

  // CTA reduction of the statistics.
  emax = __reduce_max_sync(0xffffffffu, emax);
  emin = __reduce_min_sync(0xffffffffu, emin);
  nb = (long long)warp_sum_u64((unsigned long long)nb);
  zeros = (long long)warp_sum_u64((unsigned long long)zeros);
  bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
  const int w = threadIdx.x >> 5;
  if (lane == 0) s_part[w] = StatsRec{emax, emin, nb, zeros, bad, 0};
  __syncthreads();
  if (threadIdx.x == 0) {
    StatsRec r = s_part[0];
    for (int i = 1; i < kWarps; ++i) {
      r.e_max = max(r.e_max, s_part[i].e_max);
      r.e_min = min(r.e_min, s_part[i].e_min);
      r.nbins += s_part[i].nbins;
      r.zeros += s_part[i].zeros;
      r.nonfinite |= s_part[i].nonfinite;
    }
    recs[blockIdx.x] = r;
  }
  if (MODE == kModeExact) {
    __syncthreads();
    for (int i = threadIdx.x; i < kKeyCount; i += kThreads)
      if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
  }
}

// ---------------------------------------------------------------------------
// Selection (one CTA of 1024 threads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ceil_log2_u64(unsigned long long m) {
  return m <= 1ull ? 0 : 64 - __clzll((long long)(m - 1ull));
}

__global__ void __launch_bounds__(1024) k_select(const StatsRec* __restrict__ recs, int nrecs,
                                                 const unsigned long long* __restrict__ hist, int mode,
                                                 long long n, qdot_params prm, qdot_selection* __restrict__ sel,
                                                 Header* __restrict__ hdr) {
  __shared__ int s_emax[32], s_emin[32], s_bad[32];
  __shared__ long long s_nb[32], s_z[32];
  __shared__ int s_f;
  int emax = kNeutralMax, emin = kNeutralMin, bad = 0;
  long long nb = 0, z = 0;
  for (int i = threadIdx.x; i < nrecs; i += blockDim.x) {
    StatsRec r = recs[i];
    emax = max(emax, r.e_max);
    emin = min(emin, r.e_min);
    nb += r.nbins;
    z += r.zeros;
    bad |= r.nonfinite;
  }
  if (mode == kModeExact)
    for (int i = threadIdx.x; i < kKeyCount; i += blockDim.x) nb += hist[i] != 0ull;
  emax = __reduce_max_sync(0xffffffffu, emax);
  emin = __reduce_min_sync(0xffffffffu, emin);
  bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
  nb = (long long)warp_sum_u64((unsigned long long)nb);
  z = (long long)warp_sum_u64((unsigned long long)z);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_emax[w] = emax;
    s_emin[w] = emin;
    s_bad[w] = bad;
    s_nb[w] = nb;
    s_z[w] = z;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 1; i < nw; ++i) {
      emax = max(emax, s_emax[i]);
      emin = min(emin, s_emin[i]);
      bad |= s_bad[i];
      nb += s_nb[i];
      z += s_z[i];
    }
    if (nb == 0) {
      emax = 0;
      emin = 0;
    }
    int f = nb > 0 ? floor_log2_ratio(prm.eps, prm.split_budget ? (unsigned long long)nb : 1ull) : 0;
    s_f = f;
    sel->e_max = emax;
    sel->e_min = emin;
    sel->f = f;
    sel->status = bad ? QDOT_ERR_NONFINITE : QDOT_OK;
    sel->n_bins = nb;
    sel->block = prm.block;
    sel->key_min = kKeyMin;
    sel->m_half = prm.mant_reading ? 11 : 10;
    sel->m_single = prm.mant_reading ? 24 : 23;
    sel->reserved[0] = sel->reserved[1] = 0;
    hdr->L = fixed_point_bits(n);
    hdr->lsb = emax - hdr->L;
    hdr->zeros = z;
    hdr->status = bad ? QDOT_ERR_NONFINITE : QDOT_OK;
    hdr->nonfinite = bad;
  }
  __syncthreads();
  const int e_max = sel->e_max, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  for (int k = threadIdx.x; k < kKeyCount; k += blockDim.x) {
    long long s = (long long)kKeyMin + k;
    long long sigma;
    if (mode == kModeExact) {
      unsigned long long M = hist[k];
      sigma = M ? (long long)ceil_log2_u64(M) + s - e_max - f + 1 : -1;
    } else {
      sigma = s - e_max - f + 1;  // the block key already holds ceil(log2 M_b)
    }
    sel->cls[k] = (uint8_t)precision_of(sigma, mh, ms);
  }
}

// ---------------------------------------------------------------------------
// Pass 2
// ---------------------------------------------------------------------------
struct Counts {
  unsigned long long packed = 0;  // four 16-bit counters
  unsigned long long total[4] = {0, 0, 0, 0};
  int since_flush = 0;
  __device__ __forceinline__ void add(int cls) {
    if (cls < 4) packed += 1ull << (cls * 16);
  }
  __device__ __forceinline__ void add_many(int cls, unsigned m) {
#pragma unroll
    for (int c = 0; c < 4; ++c) total[c] += (cls == c) ? m : 0u;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int c = 0; c < 4; ++c) total[c] += (packed >> (16 * c)) & 0xFFFFull;
    packed = 0;
  }
};

template <bool EXPLAIN>
__device__ __forceinline__ void accumulate(uint64_t xb, uint64_t yb, int key, int cls, int e_max, int shift0,
                                           i128& acc, long long idx, uint8_t* cls_out, double* qx_out,
                                           double* qy_out) {
  uint64_t X = significand_of(xb), Y = significand_of(yb);
  uint64_t Xq = quantize_sig(X, cls), Yq = quantize_sig(Y, cls);
  int s = shift0 + (e_max - key);  // product LSB 2^(key-104) -> accumulator LSB 2^(e_max-L)
  u128 prod = (u128)Xq * (u128)Yq;
  u128 v = s >= 128 ? (u128)0 : (prod >> s);
  uint32_t neg = (uint32_t)((xb ^ yb) >> 63);
  acc += neg ? -(i128)v : (i128)v;
  if (EXPLAIN) {
    if (cls_out) cls_out[idx] = (uint8_t)cls;
    if (qx_out) qx_out[idx] = compose_double((uint32_t)(xb >> 63), Xq, exponent_of(xb));
    if (qy_out) qy_out[idx] = compose_double((uint32_t)(yb >> 63), Yq, exponent_of(yb));
  }
}

template <int MODE, int VEC, bool EXPLAIN>
__global__ void __launch_bounds__(kThreads) k_apply(const double* __restrict__ x, const double* __restrict__ y,
                                                    long long n, int log2b, const qdot_selection* __restrict__ sel,
                                                    const Header* __restrict__ hdr,
                                                    const int16_t* __restrict__ bkeys, ApplyRec* __restrict__ recs,
                                                    uint8_t* __restrict__ cls_out, double* __restrict__ qx_out,
                                                    double* __restrict__ qy_out) {
  __shared__ __align__(16) uint8_t s_lut[kKeyCount];  // filled as 32-bit words
  __shared__ i128 s_sum[kWarps];
  __shared__ unsigned long long s_cnt[kWarps][4];
  for (int i = threadIdx.x; i < kKeyCount / 4; i += kThreads)
    reinterpret_cast<uint32_t*>(s_lut)[i] = reinterpret_cast<const uint32_t*>(sel->cls)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kThreads) >> 5;
  constexpr int R = 32 * VEC;
  const int e_max = sel->e_max;
  const int shift0 = 104 - hdr->L;
  const bool skip = hdr->status != QDOT_OK;
  i128 acc = 0;
  Counts cnt;

  if (!skip && MODE != kModeBlockLarge) {
    const long long nrows = (n + R - 1) / R;
    const int seg_lanes = (MODE == kModeBlockSmall) ? ((1 << log2b) / VEC) : 1;
    for (long long row = gwarp; row < nrows; row += nwarps) {
      Row<VEC> rw;
      load_row<VEC, true>(x, y, n, row, lane, rw);
      Decoded d[VEC];
      int u = kNeutralMax, M = 0;
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        d[j] = decode(rw.xb[j], rw.yb[j], rw.valid[j]);
        u = max(u, d[j].key);
        M += d[j].nz;
      }
      int block_cls = kZero;
      if (MODE == kModeBlockSmall) {
        segment_reduce(u, M, seg_lanes);
        block_cls = M > 0 ? (int)s_lut[ceil_log2_u32((uint32_t)M) + u - kKeyMin] : kZero;
        if ((lane & (seg_lanes - 1)) == 0) cnt.add_many(block_cls, (unsigned)M);
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        int cls;
        if (MODE == kModeBlockSmall) {
          cls = d[j].nz ? block_cls : kZero;
        } else {
          cls = d[j].nz ? (int)s_lut[d[j].key - kKeyMin] : kZero;
          cnt.add(cls);
        }
        if (EXPLAIN) {
          if (!rw.valid[j]) continue;
          if (!d[j].nz) {
            long long idx = row * R + (long long)lane * VEC + j;
            if (cls_out) cls_out[idx] = (uint8_t)kZero;
            if (qx_out) qx_out[idx] = 0.0;
            if (qy_out) qy_out[idx] = 0.0;
            continue;
          }
        }
        if (d[j].nz)
          accumulate<EXPLAIN>(rw.xb[j], rw.yb[j], d[j].key, cls, e_max, shift0, acc,
                              row * R + (long long)lane * VEC + j, cls_out, qx_out, qy_out);
      }
      if (MODE != kModeBlockSmall && ++cnt.since_flush >= 16384) {
        cnt.flush();
        cnt.since_flush = 0;
      }
    }
  } else if (!skip) {
    const long long B = 1ll << log2b;
    const long long nblk = (n + B - 1) / B;
    const long long rows_per_block = B / R;
    for (long long blk = gwarp; blk < nblk; blk += nwarps) {
      int16_t kb = bkeys[blk];
      if (kb == kEmptyBlock) {
        if (EXPLAIN) {
          for (long long i = blk * B + lane; i < n && i < (blk + 1) * B; i += 32) {
            if (cls_out) cls_out[i] = (uint8_t)kZero;
            if (qx_out) qx_out[i] = 0.0;
            if (qy_out) qy_out[i] = 0.0;
          }
        }
        continue;
      }
      const int block_cls = (int)s_lut[(int)kb - kKeyMin];
      unsigned M = 0;
      for (long long rr = 0; rr < rows_per_block; ++rr) {
        long long row = blk * rows_per_block + rr;
        if (row * R >= n) break;
        Row<VEC> rw;
        load_row<VEC, true>(x, y, n, row, lane, rw);
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
          Decoded d = decode(rw.xb[j], rw.yb[j], rw.valid[j]);
          long long idx = row * R + (long long)lane * VEC + j;
          if (d.nz) {
            M += 1;
            accumulate<EXPLAIN>(rw.xb[j], rw.yb[j], d.key, block_cls, e_max, shift0, acc, idx, cls_out, qx_out,
                                qy_out);
          } else if (EXPLAIN && rw.valid[j]) {
            if (cls_out) cls_out[idx] = (uint8_t)kZero;
            if (qx_out) qx_out[idx] = 0.0;
            if (qy_out) qy_out[idx] = 0.0;
          }
        }
      }
      cnt.add_many(block_cls, M);
    }
  }
  cnt.flush();

  // CTA reduction (exact).
  acc = warp_sum_i128(acc);
  unsigned long long c[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) c[k] = warp_sum_u64(cnt.total[k]);
  const int w = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[w] = acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ApplyRec r;
    r.sum = 0;
    for (int k = 0; k < 4; ++k) r.cnt[k] = 0;
    for (int i = 0; i < kWarps; ++i) {
      r.sum += s_sum[i];
      for (int k = 0; k < 4; ++k) r.cnt[k] += s_cnt[i][k];
    }
    recs[blockIdx.x] = r;
  }
}

// ---------------------------------------------------------------------------
// Pass 2, fast form (no per-component output).
//
// With the classes known, component i contributes q(x_i) q(y_i).  Both
// quantized operands are formed as doubles with their significand in [1, 2]:
// x_i's exponent field is set to 1023 - d (d = e_max - e_i, so the product is
// scaled by 2^-e_max), y_i's to 1023, and the significand is rounded to the
// class precision (ties to even) by an integer add-and-mask on the bit pattern
// (a carry out of the significand moves into the exponent field, as it
// should).  One fused multiply-add per component accumulates the exact
// product on the FP64 pipe; every 32 rows the FP64 partial (at most 64 terms,
// relative error <= 64 * 2^-53) is added exactly into the 128-bit fixed-point
// accumulator.
// ---------------------------------------------------------------------------
struct ClassRound {
  unsigned long long add;   // 2^(k-1) - 1 for rounding at bit k
  unsigned long long keep;  // clears the k dropped bits (0 for PERF / ZERO)
  unsigned long long lsb;   // 2^k (0 when nothing is dropped)
  unsigned long long inc;   // packed class counter increment
};

__device__ __forceinline__ i128 double_to_fixed(double v, int L) {
  // v * 2^L truncated toward zero (|v| < 2^12)
  const uint64_t b = (uint64_t)__double_as_longlong(v);
  const int be = (int)((b >> 52) & 0x7FFu);
  if (be == 0) return 0;  // |v| < 2^-1022: below any LSB used here
  const uint64_t M = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = be - 1075 + L;  // v = M 2^(be - 1075)
  i128 m = sh >= 0 ? ((i128)M << sh) : (sh <= -64 ? (i128)0 : (i128)(M >> (-sh)));
  return (b >> 63) ? -m : m;
}

template <bool GENERAL>
__device__ __forceinline__ double quantized_operand(uint64_t bits, uint32_t exp_field, const ClassRound& t) {
  uint64_t P;
  if (GENERAL) {
    const uint64_t X = significand_of(bits);  // normalises subnormals
    P = (bits & 0x8000000000000000ull) | ((uint64_t)exp_field << 52) | (X & 0x000FFFFFFFFFFFFFull);
  } else {
    P = (bits & 0x800FFFFFFFFFFFFFull) | ((uint64_t)exp_field << 52);
  }
  P = (P + t.add + ((P & t.lsb) ? 1ull : 0ull)) & t.keep;
  return __longlong_as_double((long long)P);
}

template <bool GENERAL>
__device__ __forceinline__ void apply_component(uint64_t xb, uint64_t yb, int key, int cls, int e_max,
                                                const ClassRound* tab, double& acc, unsigned long long& packed) {
  const ClassRound t = tab[cls];
  const int d = min(e_max - key, 1022);
  const double qx = quantized_operand<GENERAL>(xb, (uint32_t)(1023 - d), t);
  const double qy = quantized_operand<GENERAL>(yb, 1023u, t);
  acc = fma(qx, qy, acc);
  packed += t.inc;
}

template <int MODE, int VEC, bool GENERAL>
__device__ __forceinline__ void apply_row(const Row<VEC>& rw, int lane, int seg_lanes, const uint8_t* lut,
                                          const ClassRound* tab, int e_max, double (&acc)[VEC],
                                          unsigned long long& packed, int block_cls_in) {
  Decoded d[VEC];
  int u = kNeutralMax, M = 0;
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    d[j] = decode_fast<GENERAL>(rw.xb[j], rw.yb[j], rw.valid[j]);
    u = max(u, d[j].key);
    M += d[j].nz;
  }
  int bcls = block_cls_in;
  if (MODE == kModeBlockSmall) {
    segment_reduce(u, M, seg_lanes);
    bcls = M > 0 ? (int)lut[ceil_log2_u32((uint32_t)M) + u - kKeyMin] : kZero;
  }
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    int cls;
    if (MODE == kModeBlockSmall || MODE == kModeBlockLarge)
      cls = d[j].nz ? bcls : kZero;
    else
      cls = d[j].nz ? (int)lut[d[j].key - kKeyMin] : kZero;
    apply_component<GENERAL>(rw.xb[j], rw.yb[j], d[j].key, cls, e_max, tab, acc[j], packed);
  }
}

template <int MODE, int VEC>
__global__ void __launch_bounds__(kThreads, 4) k_apply_fast(const double* __restrict__ x,
                                                         const double* __restrict__ y, long long n, int log2b,
                                                         const qdot_selection* __restrict__ sel,
                                                         const Header* __restrict__ hdr,
                                                         const int16_t* __restrict__ bkeys,
                                                         ApplyRec* __restrict__ recs) {
  __shared__ __align__(16) uint8_t s_lut[kKeyCount];  // filled as 32-bit words
  __shared__ ClassRound s_tab[5];
  __shared__ i128 s_sum[kWarps];
  __shared__ unsigned long long s_cnt[kWarps][4];
  for (int i = threadIdx.x; i < kKeyCount / 4; i += kThreads)
    reinterpret_cast<uint32_t*>(s_lut)[i] = reinterpret_cast<const uint32_t*>(sel->cls)[i];
  if (threadIdx.x < 5) {
    const int c = threadIdx.x;
    const int k = c == kHalf ? 42 : (c == kSingle ? 29 : 0);
    ClassRound t;
    t.add = k ? (1ull << (k - 1)) - 1ull : 0ull;
    t.keep = (c == kPerf || c == kZero) ? 0ull : ~((1ull << k) - 1ull);
    t.lsb = k ? (1ull << k) : 0ull;
    t.inc = c < 4 ? (1ull << (16 * c)) : 0ull;
    s_tab[c] = t;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kThreads) >> 5;
  constexpr int R = 32 * VEC;
  const int e_max = sel->e_max;
  const int L = hdr->L;
  const bool skip = hdr->status != QDOT_OK;
  i128 acc = 0;
  double facc[VEC];
#pragma unroll
  for (int j = 0; j < VEC; ++j) facc[j] = 0.0;
  unsigned long long packed = 0, cnt[4] = {0, 0, 0, 0};
  int rows_since = 0;
  auto flush = [&]() {
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      acc += double_to_fixed(facc[j], L);
      facc[j] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) cnt[c] += (packed >> (16 * c)) & 0xFFFFull;
    packed = 0;
    rows_since = 0;
  };

  if (!skip && MODE != kModeBlockLarge) {
    const long long nrows = (n + R - 1) / R;
    const int seg_lanes = (MODE == kModeBlockSmall) ? ((1 << log2b) / VEC) : 1;
    long long row = gwarp;
    for (; row + nwarps < nrows; row += 2 * nwarps) {
      Row<VEC> r0, r1;
      load_row<VEC, true>(x, y, n, row, lane, r0);
      load_row<VEC, true>(x, y, n, row + nwarps, lane, r1);
      bool plain = true;
#pragma unroll
      for (int j = 0; j < VEC; ++j) plain &= plain_pair(r0.xb[j], r0.yb[j]) && plain_pair(r1.xb[j], r1.yb[j]);
      if (__all_sync(0xffffffffu, plain)) {
        apply_row<MODE, VEC, false>(r0, lane, seg_lanes, s_lut, s_tab, e_max, facc, packed, kZero);
        apply_row<MODE, VEC, false>(r1, lane, seg_lanes, s_lut, s_tab, e_max, facc, packed, kZero);
      } else {
        apply_row<MODE, VEC, true>(r0, lane, seg_lanes, s_lut, s_tab, e_max, facc, packed, kZero);
        apply_row<MODE, VEC, true>(r1, lane, seg_lanes, s_lut, s_tab, e_max, facc, packed, kZero);
      }
      if (++rows_since >= 16) flush();
    }
    for (; row < nrows; row += nwarps) {
      Row<VEC> r0;
      load_row<VEC, true>(x, y, n, row, lane, r0);
      apply_row<MODE, VEC, true>(r0, lane, seg_lanes, s_lut, s_tab, e_max, facc, packed, kZero);
    }
  } else if (!skip) {
    const long long B = 1ll << log2b;
    const long long nblk = (n + B - 1) / B;
    const long long rows_per_block = B / R;
    for (long long blk = gwarp; blk < nblk; blk += nwarps) {
      const int16_t kb = bkeys[blk];
      if (kb == kEmptyBlock) continue;
      const int bcls = (int)s_lut[(int)kb - kKeyMin];
      for (long long rr = 0; rr < rows_per_block; ++rr) {
        const long long row = blk * rows_per_block + rr;
        if (row * R >= n) break;
        Row<VEC> rw;
        load_row<VEC, true>(x, y, n, row, lane, rw);
        apply_row<MODE, VEC, true>(rw, lane, 1, s_lut, s_tab, e_max, facc, packed, bcls);
        if (++rows_since >= 32) flush();
      }
    }
  }
  flush();

  acc = warp_sum_i128(acc);
#pragma unroll
  for (int k = 0; k < 4; ++k) cnt[k] = warp_sum_u64(cnt[k]);
  const int w = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[w] = acc;
#pragma unroll
    for (int k = 0; k < 4; ++k) s_cnt[w][k] = cnt[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ApplyRec r;
    r.sum = 0;
    for (int k = 0; k < 4; ++k) r.cnt[k] = 0;
    for (int i = 0; i < kWarps; ++i) {
      r.sum += s_sum[i];
      for (int k = 0; k < 4; ++k) r.cnt[k] += s_cnt[i][k];
    }
    recs[blockIdx.x] = r;
  }
}

// ---------------------------------------------------------------------------
// Final (one CTA of 256 threads)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_final(const ApplyRec* __restrict__ recs, int nrecs,
                                               const qdot_selection* __restrict__ sel,
                                               const Header* __restrict__ hdr, qdot_result* __restrict__ out) {
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][4];
  i128 acc = 0;
  unsigned long long c[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < nrecs; i += blockDim.x) {
    acc += recs[i].sum;
    for (int k = 0; k < 4; ++k) c[k] += recs[i].cnt[k];
  }
  acc = warp_sum_i128(acc);
  for (int k = 0; k < 4; ++k) c[k] = warp_sum_u64(c[k]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s_sum[w] = acc;
    for (int k = 0; k < 4; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      acc += s_sum[i];
      for (int k = 0; k < 4; ++k) c[k] += s_cnt[i][k];
    }
    qdot_result r;
    r.status = hdr->status;
    r.n_bins = sel->n_bins;
    r.e_max = sel->e_max;
    r.e_min = sel->e_min;
    r.f = sel->f;
    for (int k = 0; k < 4; ++k) r.count[k] = (int64_t)c[k];
    r.count[4] = hdr->zeros;
    if (r.status != QDOT_OK) {
      r.value = __longlong_as_double(0x7FF8000000000000ll);
      r.bound = r.value;
    } else {
      r.value = fixed_to_double(acc, hdr->lsb);
      r.bound = r.n_bins > 0 ? fixed_to_double((i128)r.n_bins, r.e_max + r.f) : 0.0;
    }
    *out = r;
  }
}

template <int MODE, int VEC>
cudaError_t launch_mode(const double* x, const double* y, int64_t n, const qdot_params* p, const TwoPassPlan& pl,
                        char* ws, qdot_result* out, uint8_t* cls, double* qx, double* qy, cudaStream_t st) {
  auto* sel = reinterpret_cast<qdot_selection*>(ws + pl.off_sel);
  auto* hdr = reinterpret_cast<Header*>(ws + pl.off_hdr);
  auto* srec = reinterpret_cast<StatsRec*>(ws + pl.off_stats);
  auto* arec = reinterpret_cast<ApplyRec*>(ws + pl.off_apply);
  auto* hist = reinterpret_cast<unsigned long long*>(ws + pl.off_hist);
  auto* bkeys = reinterpret_cast<int16_t*>(ws + pl.off_keys);
  cudaError_t e;
  if (MODE == kModeExact) {
    e = cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * kKeyCount, st);
    if (e != cudaSuccess) return e;
  }
  k_stats<MODE, VEC><<<pl.grid_stats, kThreads, 0, st>>>(x, y, n, pl.log2b, srec, hist, bkeys);
  k_select<<<1, 1024, 0, st>>>(srec, pl.grid_stats, hist, MODE, n, *p, sel, hdr);
  const bool explain = cls || qx || qy;
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  if (explain)
    k_apply<MODE, VEC, true><<<pl.grid_apply, kThreads, 0, st>>>(x, y, n, pl.log2b, sel, hdr, bkeys, arec, cls,
                                                                 qx, qy);
  else
    k_apply_fast<MODE, VEC><<<pl.grid_apply, kThreads, 0, st>>>(x, y, n, pl.log2b, sel, hdr, bkeys, arec);
  if (ev1) cudaEventRecord(ev1, st);
  k_final<<<1, 256, 0, st>>>(arec, pl.grid_apply, sel, hdr, out);
  return cudaGetLastError();
}

template <int VEC>
cudaError_t launch_vec(const double* x, const double* y, int64_t n, const qdot_params* p, const TwoPassPlan& pl,
                       char* ws, qdot_result* out, uint8_t* cls, double* qx, double* qy, cudaStream_t st) {
  switch (pl.mode) {
    case kModeExact: return launch_mode<kModeExact, VEC>(x, y, n, p, pl, ws, out, cls, qx, qy, st);
    case kModeBlock1: return launch_mode<kModeBlock1, VEC>(x, y, n, p, pl, ws, out, cls, qx, qy, st);
    case kModeBlockSmall: return launch_mode<kModeBlockSmall, VEC>(x, y, n, p, pl, ws, out, cls, qx, qy, st);
    default: return launch_mode<kModeBlockLarge, VEC>(x, y, n, p, pl, ws, out, cls, qx, qy, st);
  }
}

}  // namespace

TwoPassPlan plan_two_pass(int64_t n, const qdot_params* p, bool aligned16) {
  TwoPassPlan pl;
  pl.vec = aligned16 ? 2 : 1;
  const int R = 32 * pl.vec;
  if (p->block == 0) {
    pl.mode = kModeExact;
  } else {
    int lb = 0;
    while ((1 << lb) < p->block) ++lb;
    pl.log2b = lb;
    if (p->block == 1)
      pl.mode = kModeBlock1;
    else if (p->block <= R)
      pl.mode = kModeBlockSmall;
    else
      pl.mode = kModeBlockLarge;
  }
  const DeviceInfo& di = device_info();
  const int sms = di.sms > 0 ? di.sms : 152;
  pl.grid_stats = sms * 4;   // 1024 threads per SM, two rows in flight per warp
  pl.grid_apply = sms * 4;
  pl.nblocks = (p->block > 0) ? (n + p->block - 1) / p->block : 0;
  size_t off = 0;
  pl.off_sel = off;
  off = align_up(off + sizeof(qdot_selection), 256);
  pl.off_hdr = off;
  off = align_up(off + sizeof(Header), 256);
  pl.off_stats = off;
  off = align_up(off + sizeof(StatsRec) * pl.grid_stats, 256);
  pl.off_apply = off;
  off = align_up(off + sizeof(ApplyRec) * pl.grid_apply, 256);
  pl.off_hist = off;
  off = align_up(off + sizeof(unsigned long long) * kKeyCount, 256);
  pl.off_keys = off;
  if (pl.mode == kModeBlockLarge) off = align_up(off + sizeof(int16_t) * (size_t)pl.nblocks, 256);
  pl.total = off;
  return pl;
}

cudaError_t launch_two_pass(const double* x, const double* y, int64_t n, const qdot_params* p,
                            const TwoPassPlan& plan, void* ws, qdot_result* out, qdot_selection* sel, uint8_t* cls,
                            double* qx, double* qy, cudaStream_t stream) {
  char* w = static_cast<char*>(ws);
  cudaError_t e = plan.vec == 2 ? launch_vec<2>(x, y, n, p, plan, w, out, cls, qx, qy, stream)
                                : launch_vec<1>(x, y, n, p, plan, w, out, cls, qx, qy, stream);
  if (e != cudaSuccess) return e;
  if (sel) e = cudaMemcpyAsync(sel, w + plan.off_sel, sizeof(qdot_selection), cudaMemcpyDeviceToDevice, stream);
  return e;
}

}  // namespace qd
