// Per-block work shared by the one-pass kernels (single call and batched):
// loading a warp item of 256 components, the exponent keys, and the exact
// half / single / double candidate sums of each block (see qdot_onepass.cu
// for the method and its error analysis).
//
// Mapping.  A warp item is 256 consecutive components: 256 / B blocks of B
// components, L = B / 8 lanes per block, 8 components per lane.  Lane l
// serves block g = l / L of the item; its components are
// g*B + 2*(l % L) + 2*L*j + {0, 1}, j = 0..3, read as four 16-byte loads of x
// and of y.  The whole block is in registers at once, so its maximum key u_b
// is known (a shuffle reduction over its L lanes) before any candidate is
// accumulated.
#pragma once

#include <climits>

#include "qdot_common.cuh"

namespace qd {
namespace chunk {

constexpr int kNone = -(1 << 29);  // "no key" sentinel for component keys (biased by 2046)
constexpr int kItem = 256;         // components per warp item

// Candidate masks (bit = class number).
constexpr unsigned kCandH = 1u << QDOT_HALF;
constexpr unsigned kCandS = 1u << QDOT_SINGLE;
constexpr unsigned kCandD = 1u << QDOT_DOUBLE;
constexpr unsigned kCandAll = kCandH | kCandS | kCandD;

struct BlockRec {      // one per block, written by 4 of the block's lanes
  long long h, s, d;   // candidate sums at LSB 2^(u_b - 60 + log2 B)
  short key, u;        // s_b and u_b (unbiased); key == kEmptyKey for an empty block
  unsigned int m;      // M_b in bits 0..15; the candidates present (kCand*) in bits 16..19
};
constexpr short kEmptyKey = -32768;

__device__ __forceinline__ unsigned rec_count(unsigned m) { return m & 0xFFFFu; }
__device__ __forceinline__ unsigned rec_cands(unsigned m) { return m >> 16; }

// Per-component work of the streaming kernels, on 32-bit words.
//   x = (-1)^sx * mx:lx * 2^(e_x - 52): mx = top 21 bits of the 53-bit
//   significand (implicit one at bit 20), lx = its low 32 bits.
// With u the block's maximum key (biased by 2046, like the component keys)
// and d = u - e_i >= 0, the candidates as integers on a per-block grid:
//   H: q_half(x) q_half(y)    = Ph 2^(e_i - 20), Ph = Xh Yh  (|Ph| <= 2^22),
//      grid 2^(u - 60 + K)
//   S: q_single(x) q_single(y) = Ps 2^(e_i - 46), Ps = Xs Ys  (|Ps| <= 2^48),
//      grid 2^(u - 52): the term is (Xs * (Ys * 64)) >> d, the 2^6 folded
//      into the 32-bit operand of one widening multiply
//   D: x y, on the FP64 pipe as (x / 2^e_x) (y / 2^(e_y + d)) with one fused
//      multiply-add per component (exact operands), grid 2^(u - 60 + K).
// Every term is below 2^(62 - K), so a block's sum fits in 64 bits; the
// truncation costs at most one grid unit per component, a relative error of
// at most B 2^-52 <= 2^-44 of the block's sum of |x_i y_i|.

// Round the 53-bit significand mx:lx to 11 bits (ties to even).
__device__ __forceinline__ uint32_t half_sig(uint32_t mx, uint32_t lx) {
  const uint32_t t = mx | min(lx, 1u);  // lx folds into a sticky bit below the cut
  return (t + 0x1FFu + ((t >> 10) & 1u)) >> 10;
}
// ... to 24 bits.
__device__ __forceinline__ uint32_t single_sig(uint32_t mx, uint32_t lx) {
  const uint32_t keep = __funnelshift_l(lx, mx, 3);  // (mx << 3) | (lx >> 29)
  return keep + (((lx & 0x1FFFFFFFu) + 0x0FFFFFFFu + (keep & 1u)) >> 29);
}

// Arithmetic shift right; amounts of 64 and more give the sign (PTX clamps).
__device__ __forceinline__ long long sar64(long long v, int s) {
  long long r;
  asm("shr.s64 %0, %1, %2;" : "=l"(r) : "l"(v), "r"(s));
  return r;
}

// +1 or -1: the sign of x y from the high words of x and y.
__device__ __forceinline__ int product_sign(uint32_t hx, uint32_t hy) {
  return (int)((hx ^ hy) | 0x7FFFFFFFu) >> 30;
}

// Exponent of the grid of candidate class cls for a block with maximum key u
// (unbiased) and blocks of 2^log2b.
__device__ __forceinline__ int candidate_grid(int cls, int u, int log2b) {
  return cls == kSingle ? u - 52 : u - 60 + log2b;
}

__device__ __forceinline__ double make_double(uint32_t hi, uint32_t lo) {
  return __hiloint2double((int)hi, (int)lo);
}

struct Chunk {
  uint64_t x[8], y[8];
  unsigned vmask;  // bit j: component j lies inside the vector (0xFF for a full item)
};

template <int LOG2B>
struct Map {
  static constexpr int L = 1 << (LOG2B - 3);  // lanes per block
  static constexpr int BPI = kItem >> LOG2B;  // blocks per item
};

// Index of component j (0..7) of lane `lane` within its item.
template <int LOG2B>
__device__ __forceinline__ int item_offset(int lane, int j) {
  constexpr int L = Map<LOG2B>::L;
  return (lane / L) * (1 << LOG2B) + 2 * (lane % L) + 2 * L * (j >> 1) + (j & 1);
}

// Load warp item `item` of a vector pair of length n.  The loads are marked
// streaming (evict first) unless KEEP: a kernel that reads the item again
// later (from L2) keeps the default cache policy.
template <int LOG2B, bool KEEP = false>
__device__ __forceinline__ void load_item(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                          long long item, int lane, Chunk& ch) {
  constexpr int L = Map<LOG2B>::L;
  const long long start = item * kItem;
  const long long base = start + item_offset<LOG2B>(lane, 0);
  if (start + kItem <= n) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double2* px = reinterpret_cast<const double2*>(x + base + 2 * L * j);
      const double2* py = reinterpret_cast<const double2*>(y + base + 2 * L * j);
      const double2 a = KEEP ? __ldg(px) : __ldcs(px);
      const double2 b = KEEP ? __ldg(py) : __ldcs(py);
      ch.x[2 * j] = (uint64_t)__double_as_longlong(a.x);
      ch.x[2 * j + 1] = (uint64_t)__double_as_longlong(a.y);
      ch.y[2 * j] = (uint64_t)__double_as_longlong(b.x);
      ch.y[2 * j + 1] = (uint64_t)__double_as_longlong(b.y);
    }
    ch.vmask = 0xFFu;
  } else {
    ch.vmask = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = start + item_offset<LOG2B>(lane, j);
      const bool in = i < n;
      ch.vmask |= in ? (1u << j) : 0u;
      ch.x[j] = in ? (uint64_t)__double_as_longlong(x[i]) : 0ull;
      ch.y[j] = in ? (uint64_t)__double_as_longlong(y[i]) : 0ull;
    }
  }
}

// ---------------------------------------------------------------------------
// Shared-memory staging of warp items with cp.async (16-byte copies that hold
// no registers while in flight).  Every lane copies its own 16-byte pieces
// (pieces j = 0..3 of x, then of y) into a per-warp ring of kStages items laid
// out [stage][array][j][lane], and later reads back exactly those pieces, so
// no lane ever reads what another lane wrote.
// ---------------------------------------------------------------------------
constexpr int kStages = 2;
constexpr int kStageWords = 2 * 4 * 32;              // uint4 per stage
constexpr int kRingBytes = kStages * kStageWords * 16;  // per warp: 8 KB

__device__ __forceinline__ void cp_async16(uint4* dst, const void* src, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Start the copy of warp item `item` into one stage of the ring.  Pieces past
// the end are zero-filled (a partial piece copies its in-range 8 bytes).
template <int LOG2B>
__device__ __forceinline__ void issue_item(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                           long long item, int lane, uint4* stage) {
  constexpr int L = Map<LOG2B>::L;
  const long long base = item * kItem + item_offset<LOG2B>(lane, 0);
  if (item * kItem + kItem <= n) {  // the whole item is inside the vectors
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cp_async16(stage + j * 32 + lane, x + base + 2 * L * j, 16);
      cp_async16(stage + (4 + j) * 32 + lane, y + base + 2 * L * j, 16);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const long long i = base + 2 * L * j;
    const int bytes = i + 2 <= n ? 16 : (i < n ? 8 : 0);
    const long long src = bytes ? i : 0;  // an address inside x, y even when nothing is read
    cp_async16(stage + j * 32 + lane, x + src, bytes);
    cp_async16(stage + (4 + j) * 32 + lane, y + src, bytes);
  }
}

// Read a staged item back into registers.
template <int LOG2B>
__device__ __forceinline__ void read_item(const uint4* stage, long long n, long long item, int lane, Chunk& ch) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const ulonglong2 a = reinterpret_cast<const ulonglong2*>(stage)[j * 32 + lane];
    const ulonglong2 b = reinterpret_cast<const ulonglong2*>(stage)[(4 + j) * 32 + lane];
    ch.x[2 * j] = a.x;
    ch.x[2 * j + 1] = a.y;
    ch.y[2 * j] = b.x;
    ch.y[2 * j + 1] = b.y;
  }
  if (item * kItem + kItem <= n) {
    ch.vmask = 0xFFu;
  } else {
    ch.vmask = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) ch.vmask |= item * kItem + item_offset<LOG2B>(lane, j) < n ? (1u << j) : 0u;
  }
}

// Reductions over the L lanes of a block.
template <int L>
__device__ __forceinline__ int group_max(int v) {
#pragma unroll
  for (int o = 1; o < L; o <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int L>
__device__ __forceinline__ long long group_sum(long long v) {
#pragma unroll
  for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int L>
__device__ __forceinline__ int group_sum_i(int v) {
#pragma unroll
  for (int o = 1; o < L; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Keys of a lane's components and whether every component is present,
// finite, normal and nonzero ("plain": the fast path applies).  Keys are
// biased by 2046.  kmin is updated only on the plain path.
__device__ __forceinline__ bool chunk_keys(const Chunk& ch, int (&key)[8], int& cmax, int& kmin) {
  uint32_t amin = 0xFFFFFFFFu, amax = 0u;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t ax = (uint32_t)(ch.x[j] >> 32) & 0x7FF00000u, ay = (uint32_t)(ch.y[j] >> 32) & 0x7FF00000u;
    amin = min(amin, min(ax, ay));
    amax = max(amax, max(ax, ay));
    key[j] = (int)((ax + ay) >> 20);
    cmax = max(cmax, key[j]);
  }
  // exponent fields in [1, 2046] on both sides: no zero, subnormal, Inf or NaN
  const bool plain = ch.vmask == 0xFFu && amin != 0u && amax != 0x7FF00000u;
  if (plain) {
#pragma unroll
    for (int j = 0; j < 8; ++j) kmin = min(kmin, key[j]);
  }
  return plain;
}

// The bit pattern of a double with its significand rounded to 52 - K
// fraction bits, ties to even (K = 29: SINGLE, K = 42: HALF); a carry out
// of the fraction moves into the exponent field.
template <int K>
__device__ __forceinline__ uint64_t round_bits(uint64_t v) {
  return (v + ((1ull << (K - 1)) - 1ull) + ((v >> K) & 1ull)) & ~((1ull << K) - 1ull);
}

// Candidates of the plain path for the classes in MASK, with u the block's
// maximum key (biased).  The highest class in MASK goes through the FP64
// pipe: one fused multiply-add of the exponent-rescaled operands (rounded to
// that class's precision first, so the product is exact for HALF and
// SINGLE) into aF; the other classes use the 64-bit integer path into aH /
// aS.  The FP64 pipe sustains about one fused multiply-add per component at
// full bandwidth, so only one class takes it.
template <int LOG2B, unsigned MASK>
__device__ __forceinline__ void acc_fast(const Chunk& ch, const int (&key)[8], int u, long long& aH, long long& aS,
                                         double& aF) {
  constexpr int K = LOG2B;
  constexpr unsigned TOP = (MASK & kCandD) ? kCandD : ((MASK & kCandS) ? kCandS : kCandH);
  constexpr unsigned INT_MASK = MASK & (kCandH | kCandS) & ~TOP;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hx = (uint32_t)(ch.x[j] >> 32), lx = (uint32_t)ch.x[j];
    const uint32_t hy = (uint32_t)(ch.y[j] >> 32), ly = (uint32_t)ch.y[j];
    const int d = u - key[j];
    if (INT_MASK) {
      const uint32_t mx = (hx & 0xFFFFFu) | 0x100000u, my = (hy & 0xFFFFFu) | 0x100000u;
      const int sgn = product_sign(hx, hy);
      if (INT_MASK & kCandH) {
        const int yh = (int)half_sig(my, ly) * sgn;
        aH += sar64((long long)((int)half_sig(mx, lx) * yh) << (40 - K), d);
      }
      if (INT_MASK & kCandS) {
        const int ys = (int)single_sig(my, ly) * (sgn * 64);
        aS += sar64((long long)(int)single_sig(mx, lx) * (long long)ys, d);
      }
    }
    if (MASK) {
      const uint32_t ye = 0x3FF00000u - (uint32_t)min(d, 1022) * 0x00100000u;  // exponent field 1023 - d
      uint64_t xo = ((uint64_t)((hx & 0x800FFFFFu) | 0x3FF00000u) << 32) | lx;
      uint64_t yo = ((uint64_t)((hy & 0x800FFFFFu) | ye) << 32) | ly;
      if (TOP == kCandS) {
        xo = round_bits<29>(xo);
        yo = round_bits<29>(yo);
      } else if (TOP == kCandH) {
        xo = round_bits<42>(xo);
        yo = round_bits<42>(yo);
      }
      aF = fma(__longlong_as_double((long long)xo), __longlong_as_double((long long)yo), aF);
    }
  }
}

template <int LOG2B>
__device__ __forceinline__ void acc_fast_mask(unsigned mask, const Chunk& ch, const int (&key)[8], int u,
                                              long long& aH, long long& aS, double& aD) {
  switch (mask >> 1) {  // warp-uniform
    case 0: break;
    case 1: acc_fast<LOG2B, kCandH>(ch, key, u, aH, aS, aD); break;
    case 2: acc_fast<LOG2B, kCandS>(ch, key, u, aH, aS, aD); break;
    case 3: acc_fast<LOG2B, kCandH | kCandS>(ch, key, u, aH, aS, aD); break;
    case 4: acc_fast<LOG2B, kCandD>(ch, key, u, aH, aS, aD); break;
    case 5: acc_fast<LOG2B, kCandH | kCandD>(ch, key, u, aH, aS, aD); break;
    case 6: acc_fast<LOG2B, kCandS | kCandD>(ch, key, u, aH, aS, aD); break;
    default: acc_fast<LOG2B, kCandAll>(ch, key, u, aH, aS, aD); break;
  }
}

// Candidates of the single-call paths (one-pass, fused) and of their
// recomputations share ONE definition, whatever route computes them, so a
// result does not depend on which candidates a speculation kept:
//   C_b(c) = sum over the lanes of block b of trunc(A_lane(c) * 2^G_c),
//   A_lane(c) = fl(fma(r_c(x^_7), r_c(y^_7), ... fma(r_c(x^_0), r_c(y^_0), 0))),
// the fused multiply-adds taken over the lane's nonzero components in the
// order j = 0..7 of the streaming layout, with
//   x^_j = sign(x) 1.m_x (the significand of x, exponent field 1023),
//   y^_j = sign(y) 1.m_y 2^-min(d_j, 1022), d_j = u_b - e_j,
// r_c the rounding of the significand to 11 (HALF) or 24 (SINGLE) bits, ties
// to even (a carry moves into the exponent field), r_D the identity, and
// G_H = G_D = 60 - log2 B, G_S = 52 (grids 2^(u_b - 60 + log2 B) and 2^(u_b - 52)).
// HALF and SINGLE products of rounded operands are exact in FP64; the lane
// sums of at most 8 terms below 4 each stay below 2^5, so every truncated lane
// value fits in 64 bits with room for the sum over a block's lanes.

// The chain operands of a finite nonzero pair (x, y), d = u_b - e (>= 0).
__device__ __forceinline__ void chain_operands(uint64_t xb, uint64_t yb, int d, uint64_t& xo, uint64_t& yo) {
  constexpr uint64_t kFrac = 0x000FFFFFFFFFFFFFull, kSign = 0x8000000000000000ull;
  xo = (xb & kSign) | 0x3FF0000000000000ull | (significand_of(xb) & kFrac);
  yo = (yb & kSign) | ((uint64_t)(1023 - min(d, 1022)) << 52) | (significand_of(yb) & kFrac);
}

// One fused multiply-add of the chain of class cls (kHalf, kSingle, kDouble).
__device__ __forceinline__ double chain_step(uint64_t xo, uint64_t yo, int cls, double a) {
  if (cls == kHalf) {
    xo = round_bits<42>(xo);
    yo = round_bits<42>(yo);
  } else if (cls == kSingle) {
    xo = round_bits<29>(xo);
    yo = round_bits<29>(yo);
  }
  return fma(__longlong_as_double((long long)xo), __longlong_as_double((long long)yo), a);
}

// Scale of the grid of class cls relative to 2^u_b (2^G_c above).
template <int LOG2B>
__device__ __forceinline__ double chain_scale(int cls) {
  return cls == kSingle ? 4503599627370496.0 : (double)(1ll << (60 - LOG2B));  // 2^52, 2^(60 - log2 B)
}

// Per-lane variant for the single-call stream: each lane's block has its own
// primary class `prim` (its highest wanted candidate), computed on the FP64
// pipe with that lane's rounding: SINGLE lanes round both operands to 24
// bits, HALF lanes to 11 bits, DOUBLE lanes (and lanes with no candidate)
// keep them.  RMODE (warp-uniform) has bit 0 set when some lane is SINGLE,
// bit 1 when some lane is HALF.  The SINGLE rounding uses per-lane constants
// that leave the other lanes' operands unchanged (the same bits as
// round_bits<29>); the HALF rounding is a branch (HALF lanes are usually few,
// next to perforated ones).  IMASK (warp-uniform) names the secondary classes
// some block wants besides its primary; they take chains of their own in
// every lane (aH2, aS2), and each block keeps only its own.  Every chain is
// the one defined above.
template <int LOG2B, int RMODE, unsigned IMASK>
__device__ __forceinline__ void acc_lane(const Chunk& ch, const int (&key)[8], int u, unsigned prim, double& aH2,
                                         double& aS2, double& aF) {
  const bool rs = prim == kCandS, rh = prim == kCandH;
  // SINGLE: round to nearest even at bit 29 of the 64-bit pattern
  const uint32_t s_inc = rs ? 0x0FFFFFFFu : 0u;    // half an ulp less one
  const uint32_t s_bit = rs ? 1u : 0u;             // picks the lsb (ties to even)
  const uint32_t s_mask = rs ? 0xE0000000u : ~0u;  // clears the bits below the cut
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hx = (uint32_t)(ch.x[j] >> 32), lx = (uint32_t)ch.x[j];
    const uint32_t hy = (uint32_t)(ch.y[j] >> 32), ly = (uint32_t)ch.y[j];
    const int d = u - key[j];
    const uint32_t ye = 0x3FF00000u - (uint32_t)min(d, 1022) * 0x00100000u;  // exponent field 1023 - d
    uint64_t xo = ((uint64_t)((hx & 0x800FFFFFu) | 0x3FF00000u) << 32) | lx;
    uint64_t yo = ((uint64_t)((hy & 0x800FFFFFu) | ye) << 32) | ly;
    if (IMASK & kCandH) aH2 = chain_step(xo, yo, kHalf, aH2);
    if (IMASK & kCandS) aS2 = chain_step(xo, yo, kSingle, aS2);
    if (RMODE & 1) {  // a carry out of the fraction moves into the exponent field
      xo = (xo + (s_inc + (((uint32_t)xo >> 29) & s_bit))) & (0xFFFFFFFF00000000ull | s_mask);
      yo = (yo + (s_inc + (((uint32_t)yo >> 29) & s_bit))) & (0xFFFFFFFF00000000ull | s_mask);
    }
    if ((RMODE & 2) && rh) {  // HALF lanes: round at bit 42
      xo = round_bits<42>(xo);
      yo = round_bits<42>(yo);
    }
    aF = fma(__longlong_as_double((long long)xo), __longlong_as_double((long long)yo), aF);
  }
}

template <int LOG2B, int RMODE>
__device__ __forceinline__ void acc_lane_i(unsigned imask, const Chunk& ch, const int (&key)[8], int u, unsigned prim,
                                           double& aH2, double& aS2, double& aF) {
  switch (imask >> 1) {  // warp-uniform
    case 0: acc_lane<LOG2B, RMODE, 0u>(ch, key, u, prim, aH2, aS2, aF); break;
    case 1: acc_lane<LOG2B, RMODE, kCandH>(ch, key, u, prim, aH2, aS2, aF); break;
    case 2: acc_lane<LOG2B, RMODE, kCandS>(ch, key, u, prim, aH2, aS2, aF); break;
    default: acc_lane<LOG2B, RMODE, kCandH | kCandS>(ch, key, u, prim, aH2, aS2, aF); break;
  }
}

// rounds: the primaries of the warp's lanes (OR); imask: their secondaries (OR).
template <int LOG2B>
__device__ __forceinline__ void acc_lane_mask(unsigned rounds, unsigned imask, const Chunk& ch, const int (&key)[8],
                                              int u, unsigned prim, double& aH2, double& aS2, double& aF) {
  switch (((rounds & kCandS) ? 1 : 0) | ((rounds & kCandH) ? 2 : 0)) {  // warp-uniform
    case 0: acc_lane_i<LOG2B, 0>(imask, ch, key, u, prim, aH2, aS2, aF); break;
    case 1: acc_lane_i<LOG2B, 1>(imask, ch, key, u, prim, aH2, aS2, aF); break;
    case 2: acc_lane_i<LOG2B, 2>(imask, ch, key, u, prim, aH2, aS2, aF); break;
    default: acc_lane_i<LOG2B, 3>(imask, ch, key, u, prim, aH2, aS2, aF); break;
  }
}

// Any component (zeros, subnormals, non-finite values, past the end) on the
// chains defined above: the lane's chains of the classes in MASK, the block
// maximum key (biased; kNone if the block has no nonzero component)
// returned, the lane's counts added.
template <int LOG2B, unsigned MASK = kCandAll>
__device__ __forceinline__ int chunk_general_chains(const Chunk& ch, double& aH, double& aS, double& aD, int& M,
                                                    int& zeros, int& kmin, int& bad) {
  int key[8];
  bool nz[8];
  int cmax = kNone;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t a = ch.x[j], b = ch.y[j];
    const bool in = (ch.vmask >> j) & 1u;
    const bool fin = !(is_nonfinite(a) || is_nonfinite(b));
    bad |= in && !fin;
    const bool z = is_zero(a) || is_zero(b);
    nz[j] = in && fin && !z;
    zeros += in && fin && z;
    M += nz[j];
    key[j] = nz[j] ? exponent_of(a) + exponent_of(b) + 2046 : kNone;  // biased like the fast path
    cmax = max(cmax, key[j]);
    if (nz[j]) kmin = min(kmin, key[j]);
  }
  const int u = group_max<Map<LOG2B>::L>(cmax);
  for (int j = 0; j < 8; ++j) {
    if (!nz[j]) continue;
    uint64_t xo, yo;
    chain_operands(ch.x[j], ch.y[j], u - key[j], xo, yo);
    if (MASK & kCandH) aH = chain_step(xo, yo, kHalf, aH);
    if (MASK & kCandS) aS = chain_step(xo, yo, kSingle, aS);
    if (MASK & kCandD) aD = chain_step(xo, yo, kDouble, aD);
  }
  return u;
}

// Candidates of one component with key e (biased) in a block with maximum
// key u (biased), any finite nonzero x, y given by their bits.
template <int LOG2B>
__device__ __forceinline__ void component_candidates(uint64_t xb, uint64_t yb, int e, int u, unsigned mask,
                                                     long long& aH, long long& aS, double& aD) {
  constexpr int K = LOG2B;
  const uint64_t X = significand_of(xb), Y = significand_of(yb);
  const uint32_t mx = (uint32_t)(X >> 32), lx = (uint32_t)X, my = (uint32_t)(Y >> 32), ly = (uint32_t)Y;
  const int sgn = product_sign((uint32_t)(xb >> 32), (uint32_t)(yb >> 32));
  const int d = u - e;
  if (mask & kCandH) {
    const int yh = (int)half_sig(my, ly) * sgn;
    aH += sar64((long long)((int)half_sig(mx, lx) * yh) << (40 - K), d);
  }
  if (mask & kCandS) {
    const int ys = (int)single_sig(my, ly) * (sgn * 64);
    aS += sar64((long long)(int)single_sig(mx, lx) * (long long)ys, d);
  }
  if (mask & kCandD) {
    const uint32_t sx = (uint32_t)(xb >> 63), sy = (uint32_t)(yb >> 63);
    const double xd = make_double((sx << 31) | 0x3FF00000u | (mx & 0xFFFFFu), lx);
    const uint32_t ye = (uint32_t)(1023 - min(d, 1022)) << 20;
    const double yd = make_double((sy << 31) | ye | (my & 0xFFFFFu), ly);
    aD = fma(xd, yd, aD);
  }
}

// Any component: zeros, subnormals, non-finite values, or past the end.
// Computes every candidate; returns the block maximum key (biased; kNone if
// the block has no nonzero component) and adds the lane's counts.
template <int LOG2B>
__device__ __forceinline__ int chunk_general(const Chunk& ch, long long& aH, long long& aS, double& aD, int& M,
                                             int& zeros, int& kmin, int& bad) {
  int key[8];
  bool nz[8];
  int cmax = kNone;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t a = ch.x[j], b = ch.y[j];
    const bool in = (ch.vmask >> j) & 1u;
    const bool fin = !(is_nonfinite(a) || is_nonfinite(b));
    bad |= in && !fin;
    const bool z = is_zero(a) || is_zero(b);
    nz[j] = in && fin && !z;
    zeros += in && fin && z;
    M += nz[j];
    key[j] = nz[j] ? exponent_of(a) + exponent_of(b) + 2046 : kNone;  // biased like the fast path
    cmax = max(cmax, key[j]);
    if (nz[j]) kmin = min(kmin, key[j]);
  }
  const int u = group_max<Map<LOG2B>::L>(cmax);
  for (int j = 0; j < 8; ++j)
    if (nz[j]) component_candidates<LOG2B>(ch.x[j], ch.y[j], key[j], u, kCandAll, aH, aS, aD);
  return u;
}

// Block totals over the L lanes of a block, then the block's record word
// for lane sub = l % L < 4 (0: H, 1: S, 2: D, 3: key / u / M / candidates).
// u is biased by 2046 (kNone for an empty block).
template <int LOG2B>
__device__ __forceinline__ long long block_record_word(long long aH, long long aS, double aD, int M, int u_b,
                                                      unsigned cands, int sub, int* key_out, int* u_out,
                                                      int* m_out, unsigned top = kCandD) {
  constexpr int L = Map<LOG2B>::L;
  long long aDi = 0;
  if (top == kCandS)  // aD holds the class `top` (see acc_fast)
    aS = __double2ll_rz(aD * 4503599627370496.0);  // 2^52
  else if (top == kCandH)
    aH = __double2ll_rz(aD * (double)(1ll << (60 - LOG2B)));
  else
    aDi = __double2ll_rz(aD * (double)(1ll << (60 - LOG2B)));
  aH = group_sum<L>(aH);
  aS = group_sum<L>(aS);
  aDi = group_sum<L>(aDi);
  M = group_sum_i<L>(M);
  const int u = u_b - 2046;
  const int key = M > 0 ? ceil_log2_u32((uint32_t)M) + u : (int)kEmptyKey;
  *key_out = key;
  *u_out = u;
  *m_out = M;
  if (sub == 0) return aH;
  if (sub == 1) return aS;
  if (sub == 2) return aDi;
  return (long long)(((unsigned long long)(uint16_t)(short)key) |
                     ((unsigned long long)(uint16_t)(short)(M > 0 ? u : 0) << 16) |
                     ((unsigned long long)((unsigned)M | (cands << 16)) << 32));
}

// Compact record of one block (single-call path): two candidate slots and a
// 32-bit meta word
//   meta = (s_b + kMetaKeyBias) | M_b << 13 | (stored >> 1) << 22 | ceil(log2 M_b) << 25,
//   0 = empty block,
// where `stored` (kCand* bits) names the candidates kept: the higher class in
// slot 0, the next in slot 1; when all three are kept (a warp's first items)
// the HALF candidate goes to a third, short array indexed by block.
// u_b = s_b - ceil(log2 M_b).
constexpr int kMetaKeyBias = 4096;

// Record of a general block (single-call stream): aH, aS, aD are the lane's
// chains of every class (chunk_general_chains), moved to their grids here.
template <int LOG2B>
__device__ __forceinline__ void block_record_compact(double aH, double aS, double aD, int M, int u_b,
                                                     unsigned stored, int sub, int* key_out, int* u_out, int* m_out,
                                                     long long* slot, unsigned* meta, long long* half_out) {
  constexpr int L = Map<LOG2B>::L;
  const long long h = group_sum<L>(__double2ll_rz(aH * chain_scale<LOG2B>(kHalf)));
  const long long s = group_sum<L>(__double2ll_rz(aS * chain_scale<LOG2B>(kSingle)));
  const long long d = group_sum<L>(__double2ll_rz(aD * chain_scale<LOG2B>(kDouble)));
  M = group_sum_i<L>(M);
  const int u = u_b - 2046;
  const int key = M > 0 ? ceil_log2_u32((uint32_t)M) + u : (int)kEmptyKey;
  *key_out = key;
  *u_out = u;
  *m_out = M;
  *half_out = h;
  long long hi, lo;
  if (stored & kCandD) {
    hi = d;
    lo = (stored & kCandS) ? s : h;
  } else if (stored & kCandS) {
    hi = s;
    lo = h;
  } else {
    hi = h;
    lo = 0;
  }
  *slot = sub == 0 ? hi : lo;
  *meta = M > 0 ? ((unsigned)(key + kMetaKeyBias) | ((unsigned)M << 13) | ((stored >> 1) << 22) |
                    ((unsigned)(key - u) << 25))
                 : 0u;
}

// Compact record of a plain block (B nonzero components, M_b = B): every lane
// of the block holds the same primary class `prim` in aF, so one group sum
// covers it; the secondaries (chains aH2, aS2 of the classes in `imask`,
// warp-uniform) are summed only when some block of the warp keeps one.
template <int LOG2B>
__device__ __forceinline__ void block_record_plain(double aH2, double aS2, double aF, unsigned prim, unsigned imask,
                                                   int u_b, unsigned stored, int sub, int* u_out, long long* slot,
                                                   unsigned* meta, long long* half_out) {
  constexpr int L = Map<LOG2B>::L;
  const long long hi = group_sum<L>(__double2ll_rz(aF * chain_scale<LOG2B>(prim == kCandS ? kSingle : kDouble)));
  long long lo = 0, h = 0, s = 0;
  if (imask & kCandH) h = group_sum<L>(__double2ll_rz(aH2 * chain_scale<LOG2B>(kHalf)));
  if (imask & kCandS) s = group_sum<L>(__double2ll_rz(aS2 * chain_scale<LOG2B>(kSingle)));
  if (stored & ~prim & kCandS) lo = s;
  else if (stored & ~prim & kCandH) lo = h;
  const int u = u_b - 2046;
  *u_out = u;
  *half_out = h;
  *slot = sub == 0 ? hi : lo;
  *meta = (unsigned)(LOG2B + u + kMetaKeyBias) | ((unsigned)(1 << LOG2B) << 13) | ((stored >> 1) << 22) |
          ((unsigned)LOG2B << 25);
}

__device__ __forceinline__ void unpack_meta(unsigned meta, int* key, int* u, unsigned* m, unsigned* stored) {
  *key = (int)(meta & 0x1FFFu) - kMetaKeyBias;
  *m = (meta >> 13) & 0x1FFu;
  *stored = ((meta >> 22) & 7u) << 1;
  *u = *key - (int)((meta >> 25) & 0xFu);
}

// A block candidate of class cls on its grid, moved to the fixed-point grid
// 2^lsb.
__device__ __forceinline__ i128 candidate_to_fixed(long long v, int cls, int u, int log2b, int lsb) {
  const int shift = candidate_grid(cls, u, log2b) - lsb;
  const i128 sv = (i128)v;
  if (shift >= 0) return shift >= 127 ? (i128)0 : (sv << shift);
  return (-shift) >= 127 ? (sv < 0 ? (i128)-1 : (i128)0) : (sv >> (-shift));
}

// Candidate of class cls from a record, moved from its grid to the
// fixed-point grid 2^lsb.
__device__ __forceinline__ i128 record_candidate(long long h, long long s, long long d, int u, int cls, int log2b,
                                                 int lsb) {
  if (cls == kPerf || cls == kZero) return 0;
  const long long v = cls == kHalf ? h : (cls == kSingle ? s : d);
  const int shift = candidate_grid(cls, u, log2b) - lsb;
  i128 sv = (i128)v;
  if (shift >= 0) return shift >= 127 ? (i128)0 : (sv << shift);
  return (-shift) >= 127 ? (sv < 0 ? (i128)-1 : (i128)0) : (sv >> (-shift));
}

// The candidate of class cls of block blk, recomputed from x and y at the
// record's grid (u unbiased), as the batched stream forms its candidates
// (HALF and SINGLE products truncated to the grid one by one, DOUBLE on one
// chain): used by the batched finisher when the stream skipped it.
template <int LOG2B>
__device__ long long recompute_candidate(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                         long long blk, int u, int cls) {
  const long long lo = blk << LOG2B, hi = min(n, lo + (1ll << LOG2B));
  long long aH = 0, aS = 0;
  double aD = 0.0;
  const unsigned mask = 1u << cls;
  for (long long i = lo; i < hi; ++i) {
    const uint64_t a = (uint64_t)__double_as_longlong(x[i]), b = (uint64_t)__double_as_longlong(y[i]);
    if (is_zero(a) || is_zero(b)) continue;
    const int e = exponent_of(a) + exponent_of(b) + 2046;
    component_candidates<LOG2B>(a, b, e, u + 2046, mask, aH, aS, aD);
  }
  if (cls == kHalf) return aH;
  if (cls == kSingle) return aS;
  return __double2ll_rz(aD * (double)(1ll << (60 - LOG2B)));
}

// recompute_candidate() by one warp: lane l takes components l, l + 32, ...;
// the H / S partial sums add exactly, each lane's D partial is moved to the
// grid before the sum.  Every lane returns the total.
template <int LOG2B>
__device__ long long recompute_candidate_warp(const double* __restrict__ x, const double* __restrict__ y,
                                              long long n, long long blk, int u, int cls, int lane) {
  const long long lo = blk << LOG2B, hi = min(n, lo + (1ll << LOG2B));
  long long aH = 0, aS = 0;
  double aD = 0.0;
  const unsigned mask = 1u << cls;
  for (long long i = lo + lane; i < hi; i += 32) {
    const uint64_t a = (uint64_t)__double_as_longlong(x[i]), b = (uint64_t)__double_as_longlong(y[i]);
    if (is_zero(a) || is_zero(b)) continue;
    const int e = exponent_of(a) + exponent_of(b) + 2046;
    component_candidates<LOG2B>(a, b, e, u + 2046, mask, aH, aS, aD);
  }
  long long v = cls == kHalf ? aH : (cls == kSingle ? aS : __double2ll_rz(aD * (double)(1ll << (60 - LOG2B))));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lane `sub` of block blk (0 <= sub < B / 8) recomputed on its chain of
// class cls (the definition above; u the block maximum, unbiased): the same
// components, in the same order, as in the streaming layout.  Returns the
// lane's truncated value on the class grid.
template <int LOG2B>
__device__ __forceinline__ long long recompute_chain_lane(const double* __restrict__ x, const double* __restrict__ y,
                                                          long long n, long long blk, int u, int cls, int sub) {
  constexpr int L = Map<LOG2B>::L;
  const long long base = (blk << LOG2B) + 2 * sub;
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const long long i = base + 2 * L * (j >> 1) + (j & 1);
    if (i >= n) continue;
    const uint64_t xb = (uint64_t)__double_as_longlong(x[i]), yb = (uint64_t)__double_as_longlong(y[i]);
    if (is_zero(xb) || is_zero(yb)) continue;
    uint64_t xo, yo;
    chain_operands(xb, yb, u - (exponent_of(xb) + exponent_of(yb)), xo, yo);
    a = chain_step(xo, yo, cls, a);
  }
  return __double2ll_rz(a * chain_scale<LOG2B>(cls));
}

// recompute_chain_lane() on components the warp has already loaded in the
// streaming layout (`ch`, from load_item): the same chain, the same value.
template <int LOG2B>
__device__ __forceinline__ long long chain_lane_loaded(const Chunk& ch, int u, int cls) {
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!((ch.vmask >> j) & 1u)) continue;
    const uint64_t xb = ch.x[j], yb = ch.y[j];
    if (is_zero(xb) || is_zero(yb)) continue;
    uint64_t xo, yo;
    chain_operands(xb, yb, u - (exponent_of(xb) + exponent_of(yb)), xo, yo);
    a = chain_step(xo, yo, cls, a);
  }
  return __double2ll_rz(a * chain_scale<LOG2B>(cls));
}

// The candidate of class cls of block blk by one thread (every lane's chain
// in turn) ...
template <int LOG2B>
__device__ long long recompute_chain(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                     long long blk, int u, int cls) {
  long long v = 0;
  for (int sub = 0; sub < Map<LOG2B>::L; ++sub) v += recompute_chain_lane<LOG2B>(x, y, n, blk, u, cls, sub);
  return v;
}

// ... or by one warp (lane l < B / 8 takes chain l).  Every lane returns the
// total; both give the value the streaming kernel gives.
template <int LOG2B>
__device__ long long recompute_chain_warp(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                          long long blk, int u, int cls, int lane) {
  long long v = lane < Map<LOG2B>::L ? recompute_chain_lane<LOG2B>(x, y, n, blk, u, cls, lane) : 0ll;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Quantized products of a lane's 8 components into aF (FP64, relative to
// 2^u), each with its own class cls[j] (kPerf .. kDouble).  RMODE
// (warp-uniform): bit 0 some component is SINGLE, bit 1 some is HALF, bit 2
// some is perforated.
template <int RMODE>
__device__ __forceinline__ void acc_components(const Chunk& ch, const int (&key)[8], int u, const int (&cls)[8],
                                               double& aF) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hx = (uint32_t)(ch.x[j] >> 32), lx = (uint32_t)ch.x[j];
    const uint32_t hy = (uint32_t)(ch.y[j] >> 32), ly = (uint32_t)ch.y[j];
    const int d = u - key[j];
    const uint32_t ye = 0x3FF00000u - (uint32_t)min(d, 1022) * 0x00100000u;  // exponent field 1023 - d
    uint64_t xo = ((uint64_t)((hx & 0x800FFFFFu) | 0x3FF00000u) << 32) | lx;
    uint64_t yo = ((uint64_t)((hy & 0x800FFFFFu) | ye) << 32) | ly;
    if (RMODE & 1) {  // SINGLE components: round to nearest even at bit 29
      const bool rs = cls[j] == kSingle;
      const uint32_t inc = rs ? 0x0FFFFFFFu : 0u, bit = rs ? 1u : 0u, mask = rs ? 0xE0000000u : ~0u;
      xo = (xo + (inc + (((uint32_t)xo >> 29) & bit))) & (0xFFFFFFFF00000000ull | mask);
      yo = (yo + (inc + (((uint32_t)yo >> 29) & bit))) & (0xFFFFFFFF00000000ull | mask);
    }
    if ((RMODE & 2) && cls[j] == kHalf) {
      xo = round_bits<42>(xo);
      yo = round_bits<42>(yo);
    }
    if ((RMODE & 4) && cls[j] == kPerf) xo = 0ull;
    aF = fma(__longlong_as_double((long long)xo), __longlong_as_double((long long)yo), aF);
  }
}

// The same rounding for components of any class through one table lookup
// per component instead of per-class code: the operand bits v become
// (v + inc + tie) & mask, tie = 1 when v & lsb != 0.  HALF: round to nearest
// even at bit 42 (inc = 2^41 - 1, mask clears bits 0..41, lsb = bit 42);
// SINGLE: at bit 29; DOUBLE: the identity; PERF: zero.  These are the bits
// round_bits<42>, the SINGLE add-and-mask and the PERF zero of
// acc_components give, so both return the same chain.
struct RoundTab {
  uint4 a[4];  // per class: inc low, inc high, mask low, mask high
  uint2 b[4];  // per class: lsb low, lsb high
};

// Entry c (0 <= c < 4) of the table.
__device__ __forceinline__ void round_tab_fill(RoundTab* t, int c) {
  if (c == kHalf) {
    t->a[c] = make_uint4(0xFFFFFFFFu, 0x1FFu, 0u, 0xFFFFFC00u);
    t->b[c] = make_uint2(0u, 1u << 10);
  } else if (c == kSingle) {
    t->a[c] = make_uint4(0x0FFFFFFFu, 0u, 0xE0000000u, 0xFFFFFFFFu);
    t->b[c] = make_uint2(1u << 29, 0u);
  } else if (c == kDouble) {
    t->a[c] = make_uint4(0u, 0u, 0xFFFFFFFFu, 0xFFFFFFFFu);
    t->b[c] = make_uint2(0u, 0u);
  } else {  // kPerf
    t->a[c] = make_uint4(0u, 0u, 0u, 0u);
    t->b[c] = make_uint2(0u, 0u);
  }
}

__device__ __forceinline__ uint64_t round_by_tab(uint64_t v, uint4 a, uint2 b) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const uint32_t tie = min((lo & b.x) | (hi & b.y), 1u);
  const uint64_t inc = ((uint64_t)a.y << 32) | a.x;
  const uint64_t mask = ((uint64_t)a.w << 32) | a.z;
  return (v + inc + tie) & mask;
}

// acc_components<7> through the table (tab in shared memory).
__device__ __forceinline__ void acc_components_tab(const Chunk& ch, const int (&key)[8], int u, const int (&cls)[8],
                                                   const RoundTab* tab, double& aF) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hx = (uint32_t)(ch.x[j] >> 32), lx = (uint32_t)ch.x[j];
    const uint32_t hy = (uint32_t)(ch.y[j] >> 32), ly = (uint32_t)ch.y[j];
    const int d = u - key[j];
    const uint32_t ye = 0x3FF00000u - (uint32_t)min(d, 1022) * 0x00100000u;  // exponent field 1023 - d
    const uint4 a = tab->a[cls[j]];
    const uint2 b = tab->b[cls[j]];
    const uint64_t xo = round_by_tab(((uint64_t)((hx & 0x800FFFFFu) | 0x3FF00000u) << 32) | lx, a, b);
    const uint64_t yo = round_by_tab(((uint64_t)((hy & 0x800FFFFFu) | ye) << 32) | ly, a, b);
    aF = fma(__longlong_as_double((long long)xo), __longlong_as_double((long long)yo), aF);
  }
}

__device__ __forceinline__ void acc_components_mode(unsigned rmode, const Chunk& ch, const int (&key)[8], int u,
                                                    const int (&cls)[8], double& aF) {
  switch (rmode) {  // warp-uniform
    case 0: acc_components<0>(ch, key, u, cls, aF); break;
    case 1: acc_components<1>(ch, key, u, cls, aF); break;
    case 2: acc_components<2>(ch, key, u, cls, aF); break;
    case 3: acc_components<3>(ch, key, u, cls, aF); break;
    case 4: acc_components<4>(ch, key, u, cls, aF); break;
    case 5: acc_components<5>(ch, key, u, cls, aF); break;
    case 6: acc_components<6>(ch, key, u, cls, aF); break;
    default: acc_components<7>(ch, key, u, cls, aF); break;
  }
}

// One item recomputed by a warp with the final classes, on the streaming
// layout and the chains of the streaming kernel (any components: zeros,
// subnormals, the vectors' end).  Returns the item's sum on the grid
// 2^(u - 52) (u its largest key, unbiased, in *u_out; kNone if the item has no
// nonzero component), adds the lane's class counts to c and, when tcls is
// given (qdot_trace), writes each component's class.
template <int LOG2B, typename Lut = const uint8_t*>
__device__ long long recompute_item(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                    long long item, Lut lut, int lane, int* u_out,
                                    unsigned long long (&c)[5], uint8_t* __restrict__ tcls) {
  constexpr int LB = LOG2B ? LOG2B : 8;  // the item layout (blocks of one: that of 256)
  constexpr int L = Map<LB>::L;
  Chunk ch;
  load_item<LB>(x, y, n, item, lane, ch);
  int key[8];
  bool nz[8];
  int cmax = kNone, m = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t a = ch.x[j], b = ch.y[j];
    nz[j] = ((ch.vmask >> j) & 1u) && !(is_zero(a) || is_zero(b) || is_nonfinite(a) || is_nonfinite(b));
    key[j] = nz[j] ? exponent_of(a) + exponent_of(b) + 2046 : kNone;  // biased
    cmax = max(cmax, key[j]);
    m += nz[j];
  }
  const int u = __reduce_max_sync(0xffffffffu, cmax);
  int cls[8];
  if (LOG2B == 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) cls[j] = nz[j] ? (int)lut[key[j] - 2046 - kKeyMin] : kZero;
  } else {  // the block key s_b = ceil(log2 M_b) + u_b over the block's L lanes
    const int ub = group_max<L>(cmax), mb = group_sum_i<L>(m);
    const int cb = mb ? (int)lut[ceil_log2_u32((uint32_t)mb) + ub - 2046 - kKeyMin] : kPerf;
#pragma unroll
    for (int j = 0; j < 8; ++j) cls[j] = nz[j] ? cb : kZero;
  }
  if (tcls) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if ((ch.vmask >> j) & 1u) tcls[item * kItem + item_offset<LB>(lane, j)] = (uint8_t)cls[j];
  }
  *u_out = u == kNone ? kNone : u - 2046;
  if (u == kNone) return 0;  // warp-uniform
  double a = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!nz[j]) continue;
    c[cls[j]] += 1;
    if (cls[j] == kPerf) continue;
    uint64_t xo, yo;
    chain_operands(ch.x[j], ch.y[j], u - key[j], xo, yo);
    a = chain_step(xo, yo, cls[j], a);
  }
  long long v = __double2ll_rz(a * 4503599627370496.0);  // grid 2^(u - 52)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int LOG2B, typename Lut = const uint8_t*>
__device__ long long recompute_loaded_item(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                           long long item, const Chunk& ch, Lut lut,
                                           int lane, int* u_out, unsigned long long (&c)[5],
                                           uint8_t* __restrict__ tcls);

// The selection's class table as a formula: entry k (the key kKeyMin + k) has
// the class of the score kKeyMin + k - e_max - f + 1 (a bin or block key; eq.
// bin-score-def, eq. precision-def).  Stands in for the 4224-byte table where
// every item may belong to a different problem.
struct ClassByAnchor {
  int e_max, f, mh, ms;
  __device__ __forceinline__ int operator[](int k) const {
    return precision_of((long long)kKeyMin + k - e_max - f + 1, mh, ms);
  }
};

// recompute_item() on the streaming kernel's arithmetic, for an item whose
// components are all in range, nonzero, normal and finite: the lanes load it
// in the streaming layout and quantize with the final classes from the table
// (per component, or per block from the block key log2 B + u_b).  Any other
// item goes to recompute_item().
template <int LOG2B, typename Lut = const uint8_t*>
__device__ long long recompute_item_fast(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                         long long item, Lut lut, int lane, int* u_out,
                                         unsigned long long (&c)[5], uint8_t* __restrict__ tcls) {
  constexpr int LB = LOG2B ? LOG2B : 8;
  Chunk ch;
  load_item<LB>(x, y, n, item, lane, ch);
  return recompute_loaded_item<LOG2B, Lut>(x, y, n, item, ch, lut, lane, u_out, c, tcls);
}

// recompute_item_fast() on an item the warp has already loaded (in the
// streaming layout, `ch`); an item that is not plain goes to recompute_item(),
// which reads it again.
template <int LOG2B, typename Lut>
__device__ long long recompute_loaded_item(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                           long long item, const Chunk& ch, Lut lut,
                                           int lane, int* u_out, unsigned long long (&c)[5],
                                           uint8_t* __restrict__ tcls) {
  constexpr int LB = LOG2B ? LOG2B : 8;
  constexpr int L = Map<LB>::L;
  int key[8];
  int cmax = kNone, kmin = INT_MAX;
  if (!__all_sync(0xffffffffu, chunk_keys(ch, key, cmax, kmin)))
    return recompute_item<LOG2B, Lut>(x, y, n, item, lut, lane, u_out, c, tcls);
  const int u = __reduce_max_sync(0xffffffffu, cmax);  // biased
  *u_out = u - 2046;
  double aF = 0.0;
  if (LOG2B == 0) {
    int cls[8];
    unsigned seen = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      cls[j] = lut[key[j] - 2046 - kKeyMin];
      seen |= 1u << cls[j];
      c[cls[j]] += 1;
    }
    seen = __reduce_or_sync(0xffffffffu, seen);
    acc_components_mode(((seen >> kSingle) & 1u) | (((seen >> kHalf) & 1u) << 1) | ((seen & 1u) << 2), ch, key, u,
                        cls, aF);
    if (tcls) {
#pragma unroll
      for (int j = 0; j < 8; ++j) tcls[item * kItem + item_offset<LB>(lane, j)] = (uint8_t)cls[j];
    }
  } else {
    const int cls = lut[LB + group_max<L>(cmax) - 2046 - kKeyMin];  // the block key s_b = log2 B + u_b
    c[cls] += 8;
    const unsigned prim = cls == kPerf ? 0u : 1u << cls;
    double aH2 = 0.0, aS2 = 0.0;
    acc_lane_mask<LB>(__reduce_or_sync(0xffffffffu, prim), 0u, ch, key, u, prim, aH2, aS2, aF);
    if (!prim) aF = 0.0;
    if (tcls) {
#pragma unroll
      for (int j = 0; j < 8; ++j) tcls[item * kItem + item_offset<LB>(lane, j)] = (uint8_t)cls;
    }
  }
  long long v = __double2ll_rz(aF * 4503599627370496.0);  // grid 2^(u - 52)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace chunk
}  // namespace qd
