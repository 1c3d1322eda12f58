// Per-block work shared by the one-pass kernels (single call and batched):
// loading a 32-component chunk of a block, the exponent keys, and the exact
// half / single / double candidate sums of the block (see qdot_onepass.cu for
// the method and its error analysis).
#pragma once

#include <climits>

#include "qdot_common.cuh"

namespace qd {
namespace chunk {

constexpr int kNone = -(1 << 29);  // "no key" sentinel for component keys (biased by 2046)
constexpr int kBlocksPerWarp = 8;  // blocks processed together by one warp (4 lanes each)

struct BlockRec {      // one per block, written by the block's 4 lanes
  long long h, s, d;   // candidate sums at LSB 2^(u_b - 60 + log2 B)
  short key, u;        // s_b and u_b (unbiased); key == kEmptyKey for an empty block
  unsigned int m;      // M_b
};
constexpr short kEmptyKey = -32768;

// Per-component work of the streaming kernel, on 32-bit words.
//   x = (-1)^sx * mx:lx * 2^(e_x - 52): mx = top 21 bits of the 53-bit
//   significand (implicit one at bit 20), lx = its low 32 bits.
// With u the block's running maximum key (biased by 2046, like the component
// keys) and d = u - e_i >= 0, the candidates at the block grid 2^(u - 60 + K):
//   H: q_half(x) q_half(y)    = Ph 2^(e_i - 20), Ph = Xh Yh  (|Ph| <= 2^22)
//   S: q_single(x) q_single(y) = Ps 2^(e_i - 46), Ps = Xs Ys  (|Ps| <= 2^48)
//   D: x y, on the FP64 pipe as (x / 2^e_x) (y / 2^(e_y + d)) with one fused
//      multiply-add per component (exact operands).

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

__device__ __forceinline__ double make_double(uint32_t hi, uint32_t lo) {
  return __hiloint2double((int)hi, (int)lo);
}

struct Chunk {
  uint64_t x[8], y[8];
  bool valid[8];
};

// Load chunk c (32 components) of the lane group's block.
template <int LOG2B>
__device__ __forceinline__ void load_chunk(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                           long long blk, int c, int sub, Chunk& ch) {
  const long long base = (blk << LOG2B) + c * 32 + sub * 2;
  if (base - sub * 2 + 32 <= n) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const double2 a = __ldcs(reinterpret_cast<const double2*>(x + base + j * 8));
      const double2 b = __ldcs(reinterpret_cast<const double2*>(y + base + j * 8));
      ch.x[2 * j] = (uint64_t)__double_as_longlong(a.x);
      ch.x[2 * j + 1] = (uint64_t)__double_as_longlong(a.y);
      ch.y[2 * j] = (uint64_t)__double_as_longlong(b.x);
      ch.y[2 * j + 1] = (uint64_t)__double_as_longlong(b.y);
      ch.valid[2 * j] = ch.valid[2 * j + 1] = true;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const long long i = base + (j >> 1) * 8 + (j & 1);
      ch.valid[j] = i < n;
      ch.x[j] = ch.valid[j] ? (uint64_t)__double_as_longlong(x[i]) : 0ull;
      ch.y[j] = ch.valid[j] ? (uint64_t)__double_as_longlong(y[i]) : 0ull;
    }
  }
}

__device__ __forceinline__ void rebase(int cmax, int& u_run, long long& aH, long long& aS, double& aD) {
  if (cmax > u_run) {
    if (u_run != kNone) {
      const int dlt = min(cmax - u_run, 63);
      aH >>= dlt;
      aS >>= dlt;
      aD = ldexp(aD, -dlt);
    }
    u_run = cmax;
  }
}

// Keys of a chunk and whether every component is present, finite, normal and
// nonzero ("plain": the fast path applies).  Keys are biased by 2046.
__device__ __forceinline__ bool chunk_keys(const Chunk& ch, int (&key)[8], int& cmax, int& kmin) {
  uint32_t amin = 0xFFFFFFFFu, amax = 0u;
  bool all_valid = true;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t ax = (uint32_t)(ch.x[j] >> 32) & 0x7FF00000u, ay = (uint32_t)(ch.y[j] >> 32) & 0x7FF00000u;
    amin = min(amin, min(ax, ay));
    amax = max(amax, max(ax, ay));
    all_valid &= ch.valid[j];
    key[j] = (int)((ax + ay) >> 20);
    cmax = max(cmax, key[j]);
  }
  // exponent fields in [1, 2046] on both sides: no zero, subnormal, Inf or NaN
  const bool plain = all_valid && amin != 0u && amax != 0x7FF00000u;
  if (plain) {
#pragma unroll
    for (int j = 0; j < 8; ++j) kmin = min(kmin, key[j]);
  }
  return plain;
}

template <int LOG2B>
__device__ __forceinline__ void chunk_fast(const Chunk& ch, const int (&key)[8], int cmax, int& u_run,
                                           long long& aH, long long& aS, double& aD) {
  constexpr int K = LOG2B;
  cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, 1));
  cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, 2));
  rebase(cmax, u_run, aH, aS, aD);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t hx = (uint32_t)(ch.x[j] >> 32), lx = (uint32_t)ch.x[j];
    const uint32_t hy = (uint32_t)(ch.y[j] >> 32), ly = (uint32_t)ch.y[j];
    const uint32_t mx = (hx & 0xFFFFFu) | 0x100000u, my = (hy & 0xFFFFFu) | 0x100000u;
    const int sg = (int)(hx ^ hy) >> 31;  // 0 or -1
    const int d = u_run - key[j];
    const int sh = min(d, 63);
    const int xh = (int)(half_sig(mx, lx) ^ (uint32_t)sg) - sg;
    aH += ((long long)(xh * (int)half_sig(my, ly)) << (40 - K)) >> sh;
    const int xs = (int)(single_sig(mx, lx) ^ (uint32_t)sg) - sg;
    aS += (((long long)xs * (long long)single_sig(my, ly)) << (14 - K)) >> sh;
    const uint32_t ye = 0x3FF00000u - (uint32_t)min(d, 1022) * 0x00100000u;  // exponent field 1023 - d
    aD = fma(make_double((hx & 0x800FFFFFu) | 0x3FF00000u, lx), make_double((hy & 0x800FFFFFu) | ye, ly), aD);
  }
}

// Any component: zeros, subnormals, non-finite values, or past the end.
template <int LOG2B>
__device__ __forceinline__ void chunk_general(const Chunk& ch, int& u_run, long long& aH, long long& aS, double& aD,
                                              int& M, int& zeros, int& kmin, int& bad) {
  constexpr int K = LOG2B;
  int key[8];
  bool nz[8];
  int cmax = kNone;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint64_t a = ch.x[j], b = ch.y[j];
    const bool fin = !(is_nonfinite(a) || is_nonfinite(b));
    bad |= ch.valid[j] && !fin;
    const bool z = is_zero(a) || is_zero(b);
    nz[j] = ch.valid[j] && fin && !z;
    zeros += ch.valid[j] && fin && z;
    M += nz[j];
    key[j] = nz[j] ? exponent_of(a) + exponent_of(b) + 2046 : kNone;  // biased like the fast path
    cmax = max(cmax, key[j]);
    if (nz[j]) kmin = min(kmin, key[j]);
  }
  cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, 1));
  cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, 2));
  rebase(cmax, u_run, aH, aS, aD);
  for (int j = 0; j < 8; ++j) {
    if (!nz[j]) continue;
    const uint64_t X = significand_of(ch.x[j]), Y = significand_of(ch.y[j]);
    const uint32_t mx = (uint32_t)(X >> 32), lx = (uint32_t)X, my = (uint32_t)(Y >> 32), ly = (uint32_t)Y;
    const int sg = (int)((uint32_t)(ch.x[j] >> 32) ^ (uint32_t)(ch.y[j] >> 32)) >> 31;
    const int d = u_run - key[j];
    const int sh = min(d, 63);
    const int xh = (int)(half_sig(mx, lx) ^ (uint32_t)sg) - sg;
    aH += ((long long)(xh * (int)half_sig(my, ly)) << (40 - K)) >> sh;
    const int xs = (int)(single_sig(mx, lx) ^ (uint32_t)sg) - sg;
    aS += (((long long)xs * (long long)single_sig(my, ly)) << (14 - K)) >> sh;
    const uint32_t sx = (uint32_t)(ch.x[j] >> 63), sy = (uint32_t)(ch.y[j] >> 63);
    const double xd = make_double((sx << 31) | 0x3FF00000u | (mx & 0xFFFFFu), lx);
    const uint32_t ye = (uint32_t)(1023 - min(d, 1022)) << 20;
    const double yd = make_double((sy << 31) | ye | (my & 0xFFFFFu), ly);
    aD = fma(xd, yd, aD);
  }
}


// Block totals over the 4 lanes of a block, then the block's record word for
// lane `sub` (0: H, 1: S, 2: D, 3: key / u / M).  u_run is biased by 2046.
template <int LOG2B>
__device__ __forceinline__ long long block_record_word(long long aH, long long aS, double aD, int M, int u_run,
                                                      int sub, int* key_out, int* u_out, int* m_out) {
  long long aDi = __double2ll_rz(aD * (double)(1ll << (60 - LOG2B)));
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    aH += __shfl_xor_sync(0xffffffffu, aH, o);
    aS += __shfl_xor_sync(0xffffffffu, aS, o);
    aDi += __shfl_xor_sync(0xffffffffu, aDi, o);
    M += __shfl_xor_sync(0xffffffffu, M, o);
  }
  const int u = u_run - 2046;
  const int key = M > 0 ? ceil_log2_u32((uint32_t)M) + u : (int)kEmptyKey;
  *key_out = key;
  *u_out = u;
  *m_out = M;
  if (sub == 0) return aH;
  if (sub == 1) return aS;
  if (sub == 2) return aDi;
  return (long long)(((unsigned long long)(uint16_t)(short)key) |
                     ((unsigned long long)(uint16_t)(short)(M > 0 ? u : 0) << 16) |
                     ((unsigned long long)(unsigned)M << 32));
}

// Candidate of class cls from a record, moved from the block grid
// 2^(u - 60 + log2 B) to the fixed-point grid 2^lsb.
__device__ __forceinline__ i128 record_candidate(long long h, long long s, long long d, int u, int cls, int log2b,
                                                 int lsb) {
  if (cls == kPerf || cls == kZero) return 0;
  const long long v = cls == kHalf ? h : (cls == kSingle ? s : d);
  const int shift = (u - 60 + log2b) - lsb;
  i128 sv = (i128)v;
  if (shift >= 0) return shift >= 127 ? (i128)0 : (sv << shift);
  return (-shift) >= 127 ? (sv < 0 ? (i128)-1 : (i128)0) : (sv >> (-shift));
}

}  // namespace chunk
}  // namespace qd
