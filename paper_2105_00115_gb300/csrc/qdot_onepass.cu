// One-pass qdot with deferred selection, blocked binning, 32 <= B <= 256.
//
// The class of a block depends on the global e_max and N_bins (eq.
// bin-score-def), which are only known after every component has been read.
// One read of x and y is still enough: for every block b the streaming kernel
// forms the three candidate sums the block can need,
//     H_b = sum q_half(x_i) q_half(y_i),  S_b = sum q_single(x_i) q_single(y_i),
//     D_b = sum x_i y_i,
// exactly (fixed point below the block maximum u_b) and writes them, with the
// block key s_b = ceil(log2 M_b) + u_b, as a 32-byte record.  Selection is
// deferred: once e_max and N_bins are known, a gather kernel reads the records
// (6.25% of the input bytes for B = 32, 0.8% for B = 256), takes for each
// block the candidate of the class eq. (precision-def) assigns to
// sigma_b = s_b - e_max - f + 1, and sums exactly.
//
// Mapping: a warp handles 8 blocks at a time, 4 lanes per block; per chunk of
// 32 components of a block each lane loads 4 x 16 bytes of x and of y, and the
// next chunk is loaded while the current one is processed.  Candidate values
// are formed at the scale 2^(e_i - 60) and shifted right by (u - e_i) + K,
// K = log2 B, so 64-bit block sums stay below 2^62 and are exact up to one
// unit of 2^(u - 60 + K) per component (relative error <= B^2 2^-60 per
// block, 2^-44 for B = 256).  The double candidate is accumulated on the FP64
// pipe with one fused multiply-add per component on exponent-rescaled
// operands (relative error <= (B/4) 2^-53 per lane), then converted to the
// same grid.
#include <algorithm>
#include <climits>
#include <cmath>

#include "qdot_chunk.cuh"
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

using namespace chunk;

constexpr int kOpThreads = 256;
constexpr int kOpWarps = kOpThreads / 32;
constexpr int kOpCtasPerSm = 3;                       // 3 x 64 KB of staging per SM
constexpr int kOpSmem = kOpWarps * kRingBytes;

// Per-warp record written to the workspace.
struct WarpStats {
  int e_max;           // largest block maximum u_b
  int e_min;           // smallest component key
  int nonfinite;
  int pad;
  long long nbins;     // non-empty blocks
  long long zeros;     // ZERO components
};

struct OpHeader {
  int L, lsb;
  int status;
  int erun;            // running lower bound of e_max shared by the streaming warps (biased)
  long long zeros;
  unsigned done;       // gather CTAs that have written their partial (zeroed by k_op_select)
};
struct OpPart {
  i128 sum;
  unsigned long long cnt[4];
  unsigned long long repairs;  // blocks whose candidate the gather recomputed
};


// Speculation windows: a block gets the SINGLE candidate when its score may
// lie up to kWinS below its upper bound sigma_hi, the HALF candidate up to
// kWinH below.  For a block of B nonzero components the score is sigma_hi
// less (e_max - e_lo) less (f - f_spec); once the running bound e_lo has
// caught up with e_max, and unless many blocks are empty (f > f_spec), that
// difference is 0, so each block gets one candidate: the class of sigma_hi.
// During the first 1/kEarlyDiv of a warp's items, while the bound still
// climbs, both windows widen by kWinEarly, and a warp's first two items get
// every candidate.  A block whose class falls outside its window is
// recomputed by the gather.
constexpr int kWinS = 0, kWinH = 0, kWinEarly = 8, kEarlyDiv = 32;
// The windows also stay wide until the warp's bound e_lo has held for kCalm
// items: while it still rises (short vectors, heavy tails) it may be short
// of e_max by more than a window of 0 allows.
constexpr int kCalm = 4;
// The warps share their bounds of e_max through one word: each raises it
// when it sees a larger key and reads it every kExchange items, using each
// read kExchange items later (the first read, at item 1, at item 2).
constexpr int kExchange = 2;

// Blocks a gather CTA can queue for recomputation by its warps together.
constexpr int kRepairQueue = 512;

// The candidates a block with maximum key u (biased; kNone if empty) should
// get, after folding u into the warp's running bound e_lo of e_max.  e_lo
// also takes in erun, the bound shared by all warps, on the schedule above;
// each read has a few items' time to complete before its value is used.
template <int LOG2B>
__device__ __forceinline__ unsigned candidates_wanted(int u, int lane, int iter, long long early_items, int f_spec,
                                                      int mh, int ms, int* erun, int& e_lo, int& pending,
                                                      int& raised) {
  constexpr int L = Map<LOG2B>::L;
  int wmax = u;
#pragma unroll
  for (int o = L; o < 32; o <<= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  if ((iter & (kExchange - 1)) == 1) {
    const int seen = __shfl_sync(0xffffffffu, pending, 0);  // loaded kExchange items ago (none at the first read)
    if (lane == 0) pending = *(volatile int*)erun;
    if (seen > e_lo) {
      e_lo = seen;
      raised = iter;
    }
  }
  if (iter == 2) {  // the read issued at item 1
    const int seen = __shfl_sync(0xffffffffu, pending, 0);
    if (seen > e_lo) {
      e_lo = seen;
      raised = iter;
    }
  }
  if (wmax > e_lo) {
    e_lo = wmax;
    raised = iter;
    if (lane == 0) atomicMax(erun, wmax);
  }
  if (u == kNone) return 0;
  if (iter < 2) return kCandAll;  // before the first exchange e_lo is this warp's alone
  // sigma_hi >= the block's score (e_lo <= e_max, f_spec <= f, ceil(log2 M_b) <= log2 B);
  // candidates for the classes of scores in the window below sigma_hi
  const int sig_hi = LOG2B + u - e_lo - f_spec + 1;
  const int wide = (iter < early_items || iter - raised < kCalm) ? kWinEarly : 0;
  unsigned want = 0;
  if (sig_hi >= ms) want |= kCandD;
  if (sig_hi >= mh && sig_hi - kWinS - wide < ms) want |= kCandS;
  if (sig_hi >= 0 && sig_hi - kWinH - wide < mh) want |= kCandH;
  return want;
}

template <int LOG2B>
__global__ void __launch_bounds__(kOpThreads, kOpCtasPerSm) k_onepass(const double* __restrict__ x,
                                                           const double* __restrict__ y, long long n, int f_spec,
                                                           int mh, int ms, int* __restrict__ erun,
                                                           WarpStats* __restrict__ wstats,
                                                           long long* __restrict__ slots,
                                                           long long* __restrict__ slots1,
                                                           unsigned* __restrict__ metas,
                                                           long long* __restrict__ slot3) {
  constexpr int L = Map<LOG2B>::L, BPI = Map<LOG2B>::BPI;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, sub = lane % L;
  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;

  const long long nblocks = (n + (1ll << LOG2B) - 1) >> LOG2B;
  const long long nitems = (n + kItem - 1) / kItem;
  const long long gwarp = ((long long)blockIdx.x * kOpThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kOpThreads) >> 5;

  int e_lo = kNone;     // lower bound of e_max (biased), the same in every lane
  int pending = kNone;  // lane 0: the value erun held at its last read
  int raised = 0;       // the item at which e_lo last rose
  int iter = 0;
  const long long my_items = gwarp < nitems ? (nitems - gwarp + nwarps - 1) / nwarps : 0;
  const long long early_items = (my_items + kEarlyDiv - 1) / kEarlyDiv;
  extern __shared__ uint4 s_ring[];
  uint4* ring = s_ring + (threadIdx.x >> 5) * (kStages * kStageWords);
  // prologue: items it, it + nwarps, ... (kStages - 1 of them) in flight
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    const long long item = gwarp + s * nwarps;
    if (item < nitems) issue_item<LOG2B>(x, y, n, item, lane, ring + s * kStageWords);
    cp_async_commit();
  }
  int stage = 0;
  long long it = gwarp;
  Chunk cur;
  while (it < nitems) {
    {  // refill the stage read in the previous iteration, kStages - 1 items ahead
      const long long ahead = it + (long long)(kStages - 1) * nwarps;
      const int st = stage == 0 ? kStages - 1 : stage - 1;
      if (ahead < nitems) issue_item<LOG2B>(x, y, n, ahead, lane, ring + st * kStageWords);
      cp_async_commit();
    }
    cp_async_wait<kStages - 1>();  // this lane's copies of item `it` have landed
    read_item<LOG2B>(ring + stage * kStageWords, n, it, lane, cur);
    stage = stage == kStages - 1 ? 0 : stage + 1;
    long long aH = 0, aS = 0;
    double aD = 0.0;
    int M = 0, zeros = 0, u;
    unsigned want = 0;
    int key[8];
    int cmax = kNone;
    int ub, mb;
    long long slot, half;
    unsigned meta;
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      u = group_max<L>(cmax);
      want = candidates_wanted<LOG2B>(u, lane, iter, early_items, f_spec, mh, ms, erun, e_lo, pending, raised);
      const unsigned prim = want ? (1u << (31 - __clz((int)want))) : 0u;  // the block's primary class
      const unsigned both = __reduce_or_sync(0xffffffffu, prim | (want & ~prim) << 4);
      const unsigned rounds = both & 0xFu, imask = both >> 4;
      acc_lane_mask<LOG2B>(rounds, imask, cur, key, u, prim, aH, aS, aD);
      block_record_plain<LOG2B>(aH, aS, aD, prim, imask, u, want, sub, &ub, &slot, &meta, &half);
      mb = 1 << LOG2B;
    } else {
      u = chunk_general<LOG2B>(cur, aH, aS, aD, M, zeros, kmin, bad);  // every candidate
      want = candidates_wanted<LOG2B>(u, lane, iter, early_items, f_spec, mh, ms, erun, e_lo, pending, raised);
      int kb;
      block_record_compact<LOG2B>(aH, aS, aD, kCandD, M, u, want, sub, &kb, &ub, &mb, &slot, &meta, &half);
    }
    // the record keeps the block's wanted candidates
    const long long blk = it * BPI + g;
    zeros_l += zeros;
    if (blk < nblocks) {
      if (mb > 0) {
        nbins += (sub == 0);
        emax_l = max(emax_l, ub);
      }
      if (sub == 0) {
        slots[blk] = slot;
        metas[blk] = meta;
      }
      if (sub == 1 && (want & (want - 1u)) != 0u) slots1[blk] = slot;  // the next one, if kept
      if (sub == 3 && want == kCandAll && blk < 2 * nwarps * BPI) slot3[blk] = half;  // first two items only
    }
    it += nwarps;
    ++iter;
  }
  cp_async_wait<0>();

  // per-warp record
  emax_l = __reduce_max_sync(0xffffffffu, emax_l);
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  nbins = (long long)warp_sum_u64((unsigned long long)nbins);
  zeros_l = (long long)warp_sum_u64((unsigned long long)zeros_l);
  if (lane == 0) {
    WarpStats st;
    st.e_max = emax_l;
    st.e_min = kmin == INT_MAX ? INT_MAX : kmin - 2046;
    st.nonfinite = bad;
    st.pad = 0;
    st.nbins = nbins;
    st.zeros = zeros_l;
    wstats[gwarp] = st;
  }
}

// Global statistics and the class table (one CTA).
__global__ void __launch_bounds__(1024) k_op_select(const WarpStats* __restrict__ ws, int nw, long long n,
                                                    qdot_params prm, qdot_selection* __restrict__ sel,
                                                    OpHeader* __restrict__ hdr) {
  __shared__ int s_emax[32], s_emin[32], s_bad[32];
  __shared__ long long s_nb[32], s_z[32];
  __shared__ int s_f;
  int emax = kNone, emin = INT_MAX, bad = 0;
  long long nb = 0, z = 0;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) {
    WarpStats s = ws[i];
    emax = max(emax, s.e_max);
    emin = min(emin, s.e_min);
    bad |= s.nonfinite;
    nb += s.nbins;
    z += s.zeros;
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  emin = __reduce_min_sync(0xffffffffu, emin);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
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
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
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
    const int status = bad ? QDOT_ERR_NONFINITE : QDOT_OK;
    sel->e_max = emax;
    sel->e_min = emin;
    sel->f = f;
    sel->status = status;
    sel->n_bins = nb;
    sel->block = prm.block;
    sel->key_min = kKeyMin;
    sel->m_half = prm.mant_reading ? 11 : 10;
    sel->m_single = prm.mant_reading ? 24 : 23;
    sel->reserved[0] = sel->reserved[1] = 0;
    hdr->L = fixed_point_bits(n);
    hdr->lsb = emax - hdr->L;
    hdr->status = status;
    hdr->zeros = z;
    hdr->done = 0u;
  }
  __syncthreads();
  const int e_max = sel->e_max, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  for (int k = threadIdx.x; k < kKeyCount; k += blockDim.x)
    sel->cls[k] = (uint8_t)precision_of((long long)kKeyMin + k - e_max - f + 1, mh, ms);
}

// Deferred selection: per block record pick the candidate of the block's
// class and add it exactly to a fixed-point sum anchored at 2^(e_max - L).
// A candidate the streaming kernel skipped is recomputed here from x and y.
// The last CTA to finish adds the CTA partials in order and writes the result.
template <int LOG2B>
__global__ void __launch_bounds__(256, 4) k_op_gather(const long long* __restrict__ slots,
                                                   const long long* __restrict__ slots1,
                                                   const unsigned* __restrict__ metas,
                                                   const long long* __restrict__ slot3, long long n_early,
                                                   long long nblocks, qdot_selection* __restrict__ sel,
                                                   OpHeader* __restrict__ hdr, OpPart* __restrict__ parts,
                                                   const double* __restrict__ x, const double* __restrict__ y,
                                                   long long n, qdot_result* __restrict__ out) {
  __shared__ uint8_t s_lut[kKeyCount];
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][5];
  __shared__ long long s_qblk[kRepairQueue];  // blocks to recompute ...
  __shared__ int s_qinfo[kRepairQueue];       // ... with u << 2 | class
  __shared__ int s_nqueue;
  __shared__ bool s_last;
  for (int i = threadIdx.x; i < kKeyCount / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(s_lut)[i] = reinterpret_cast<const uint32_t*>(sel->cls)[i];
  if (threadIdx.x == 0) s_nqueue = 0;
  __syncthreads();
  const int lsb = hdr->lsb;
  const bool ok = hdr->status == QDOT_OK;
  i128 acc = 0;                               // recomputed candidates
  unsigned long long acc_lo = 0;              // the others: a 128-bit sum in two words
  long long acc_hi = 0;
  unsigned long long c_ph = 0, c_sd = 0;      // components per class, two 32-bit counts per word
  unsigned long long c_rep = 0;               // recomputed blocks
  // one block: its meta word and its first candidate slot
  auto take = [&](unsigned mw, long long sl0, long long blk) {
    int key, u;
    unsigned m, stored;
    unpack_meta(mw, &key, &u, &m, &stored);    // m = 0 for an empty block (mw = 0)
    const int cls = mw ? (int)s_lut[mw ? key - kKeyMin : 0] : kPerf;
    const unsigned long long cm = (unsigned long long)m << ((cls & 1) << 5);
    if (cls < 2) c_ph += cm; else c_sd += cm;
    const int top = 31 - __clz((int)(stored | 1u));  // the highest kept class sits in slot 0
    long long v = sl0;
    bool keep = cls != kPerf;
    if (keep && cls != top) {  // a second kept candidate, or a missing one
      if (stored == kCandAll && cls == kHalf && blk >= n_early) stored = 0;  // never written
      if (stored & (1u << cls)) {
        v = (stored == kCandAll && cls == kHalf) ? slot3[blk]  // blk < n_early by construction
                                                 : slots1[blk];
      } else {
        ++c_rep;
        keep = false;
        const int q = atomicAdd(&s_nqueue, 1);
        if (q < kRepairQueue) {  // the CTA's warps recompute it together after the sweep
          s_qblk[q] = blk;
          s_qinfo[q] = (u << 2) | cls;
        } else {  // queue full: this thread recomputes it alone
          acc += candidate_to_fixed(recompute_candidate<LOG2B>(x, y, n, blk, u, cls), cls, u, LOG2B, lsb);
        }
      }
    }
    // v on its grid 2^g, moved to 2^lsb: g - lsb <= L - 52 <= 52 (u <= e_max, L <= 104);
    // a negative shift truncates, as the fixed-point sum does
    const int sh = candidate_grid(cls, u, LOG2B) - lsb;
    const int sl = min(max(sh, 0), 63), sr = min(max(-sh, 0), 63);
    const long long w = keep ? (v >> sr) : 0ll;
    const unsigned long long lo = (unsigned long long)w << sl;
    const long long hi = (w >> 1) >> (63 - sl);  // the bits shifted out of lo, sign-extended
    acc_lo += lo;
    acc_hi += hi + (acc_lo < lo ? 1 : 0);
  };
  // four consecutive blocks per quad: their meta words (16 bytes) and first
  // slots (32 bytes) are independent loads; a second slot is read only for
  // a block whose class is its second kept candidate
  const long long nquads = nblocks >> 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const uint4* m4 = reinterpret_cast<const uint4*>(metas);
  const longlong2* s4 = reinterpret_cast<const longlong2*>(slots);
  for (long long qa = (long long)blockIdx.x * blockDim.x + threadIdx.x; ok && qa < nquads; qa += stride) {
    const uint4 ma = m4[qa];
    const longlong2 sa = s4[2 * qa], sb = s4[2 * qa + 1];
    take(ma.x, sa.x, 4 * qa);
    take(ma.y, sa.y, 4 * qa + 1);
    take(ma.z, sb.x, 4 * qa + 2);
    take(ma.w, sb.y, 4 * qa + 3);
  }
  {  // the last nblocks % 4 blocks
    const long long blk = 4 * nquads + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (ok && blk < nblocks) take(metas[blk], slots[blk], blk);
  }
  // queued recomputations: one warp per block, lanes striding over its
  // components (coalesced), partial candidates summed over the warp
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nq = min(s_nqueue, kRepairQueue);
  for (int qi = w; qi < nq; qi += (int)(blockDim.x >> 5)) {
    const long long blk = s_qblk[qi];
    const int cls = s_qinfo[qi] & 3, u = s_qinfo[qi] >> 2;
    const long long v = recompute_candidate_warp<LOG2B>(x, y, n, blk, u, cls, lane);
    if (lane == 0) acc += candidate_to_fixed(v, cls, u, LOG2B, lsb);
  }
  acc += (i128)(((unsigned __int128)(unsigned long long)acc_hi << 64) | acc_lo);
  unsigned long long c[5] = {c_ph & 0xFFFFFFFFull, c_ph >> 32, c_sd & 0xFFFFFFFFull, c_sd >> 32, c_rep};
  acc = warp_sum_i128(acc);
  for (int k = 0; k < 5; ++k) c[k] = warp_sum_u64(c[k]);
  if (lane == 0) {
    s_sum[w] = acc;
    for (int k = 0; k < 5; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    OpPart p;
    p.sum = 0;
    for (int k = 0; k < 4; ++k) p.cnt[k] = 0;
    p.repairs = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      p.sum += s_sum[i];
      for (int k = 0; k < 4; ++k) p.cnt[k] += s_cnt[i][k];
      p.repairs += s_cnt[i][4];
    }
    parts[blockIdx.x] = p;
    __threadfence();  // the partial is visible before the arrival is counted
    s_last = atomicAdd(&hdr->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  // last CTA: the exact sum of the partials, in CTA order, then one rounding
  __threadfence();
  const int np = gridDim.x;
  acc = 0;
  for (int k = 0; k < 5; ++k) c[k] = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const unsigned long long* pw = reinterpret_cast<const unsigned long long*>(parts + i);
    const unsigned long long lo = __ldcg(pw), hi = __ldcg(pw + 1);
    acc += (i128)(((unsigned __int128)hi << 64) | lo);
    for (int k = 0; k < 4; ++k) c[k] += __ldcg(&parts[i].cnt[k]);
    c[4] += __ldcg(&parts[i].repairs);
  }
  acc = warp_sum_i128(acc);
  for (int k = 0; k < 5; ++k) c[k] = warp_sum_u64(c[k]);
  __syncthreads();  // s_sum, s_cnt are reused
  if (lane == 0) {
    s_sum[w] = acc;
    for (int k = 0; k < 5; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      acc += s_sum[i];
      for (int k = 0; k < 5; ++k) c[k] += s_cnt[i][k];
    }
    sel->reserved[0] = (int32_t)(c[4] < 0x7FFFFFFFull ? c[4] : 0x7FFFFFFFull);
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

// The largest k with N * 2^k <= eps (host side; only steers which candidates
// the streaming kernel computes, so an off-by-one costs time, not accuracy).
int host_floor_log2_ratio(double eps, unsigned long long N) {
  const double dn = (double)N;
  int k = std::ilogb(eps) - std::ilogb(dn);
  for (int i = 0; i < 4 && std::ldexp(dn, k) > eps; ++i) --k;
  for (int i = 0; i < 4 && std::ldexp(dn, k + 1) <= eps; ++i) ++k;
  return k;
}

template <int LOG2B>
cudaError_t launch_lb(const double* x, const double* y, int64_t n, const qdot_params* p, const OnePassPlan& pl,
                      char* ws, qdot_result* out, cudaStream_t st) {
  auto* sel = reinterpret_cast<qdot_selection*>(ws + pl.off_sel);
  auto* hdr = reinterpret_cast<OpHeader*>(ws + pl.off_hdr);
  auto* wst = reinterpret_cast<WarpStats*>(ws + pl.off_rec);
  auto* slots = reinterpret_cast<long long*>(ws + pl.off_misc);
  auto* slots1 = reinterpret_cast<long long*>(ws + pl.off_slot1);
  auto* metas = reinterpret_cast<unsigned*>(ws + pl.off_meta);
  auto* slot3 = reinterpret_cast<long long*>(ws + pl.off_slot3);
  auto* parts = reinterpret_cast<OpPart*>(ws + pl.off_sel + align_up(sizeof(qdot_selection), 256) +
                                          align_up(sizeof(OpHeader), 256));
  const long long nblocks = (n + (1ll << LOG2B) - 1) >> LOG2B;
  // f if every block is non-empty (a lower bound of the real f)
  const int f_spec = host_floor_log2_ratio(p->eps, p->split_budget ? (unsigned long long)nblocks : 1ull);
  const int mh = p->mant_reading ? 11 : 10, ms = p->mant_reading ? 24 : 23;
  cudaError_t e = cudaMemsetAsync(&hdr->erun, 0x80, sizeof(int), st);  // very negative
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  static bool smem_set = false;  // per instantiation
  if (!smem_set) {
    e = cudaFuncSetAttribute(k_onepass<LOG2B>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOpSmem);
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  k_onepass<LOG2B><<<pl.grid, kOpThreads, kOpSmem, st>>>(x, y, n, f_spec, mh, ms, &hdr->erun, wst, slots, slots1,
                                                          metas, slot3);
  if (ev1) cudaEventRecord(ev1, st);
  const int nw = pl.grid * kOpWarps;
  k_op_select<<<1, 1024, 0, st>>>(wst, nw, n, *p, sel, hdr);
  const int gather_grid = 4 * (device_info().sms > 0 ? device_info().sms : 152);
  k_op_gather<LOG2B><<<gather_grid, 256, 0, st>>>(slots, slots1, metas, slot3, 2ll * pl.grid * kOpWarps * Map<LOG2B>::BPI,
                                                    nblocks, sel, hdr, parts, x, y, n, out);
  return cudaGetLastError();
}

}  // namespace

bool one_pass_supported(int64_t n, const qdot_params* p, bool aligned16) {
  return aligned16 && n > 0 && p->block >= 32 && p->block <= 256;
}

int one_pass_launches(int64_t, const qdot_params*) { return 3; }  // stream, select, gather

OnePassPlan plan_one_pass(int64_t n, const qdot_params* p) {
  OnePassPlan pl;
  int lb = 0;
  while ((1 << lb) < p->block) ++lb;
  pl.log2b = lb;
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  pl.grid = sms * kOpCtasPerSm;
  const long long nblocks = (n + p->block - 1) / p->block;
  size_t off = 0;
  pl.off_sel = off;
  off = align_up(off + sizeof(qdot_selection), 256);
  pl.off_hdr = off;
  off = align_up(off + sizeof(OpHeader), 256);
  off = align_up(off + sizeof(OpPart) * 4 * sms, 256);  // gather partials
  pl.off_rec = off;
  off = align_up(off + sizeof(WarpStats) * pl.grid * kOpWarps, 256);
  pl.off_misc = off;  // the first candidate slot of every block
  off = align_up(off + sizeof(long long) * (size_t)nblocks, 256);
  pl.off_slot1 = off;  // the second, written for blocks that keep two or more
  off = align_up(off + sizeof(long long) * (size_t)nblocks, 256);
  pl.off_meta = off;  // one meta word per block
  off = align_up(off + sizeof(unsigned) * (size_t)nblocks, 256);
  pl.off_slot3 = off;  // HALF candidates of the blocks of every warp's first two items
  const long long early_blocks = 2ll * pl.grid * kOpWarps * (kItem / p->block);
  off = align_up(off + sizeof(long long) * (size_t)std::min(nblocks, early_blocks), 256);
  pl.total = off;
  return pl;
}

cudaError_t launch_one_pass(const double* x, const double* y, int64_t n, const qdot_params* p,
                            const OnePassPlan& plan, void* ws, qdot_result* out, qdot_selection* sel,
                            cudaStream_t stream) {
  char* w = static_cast<char*>(ws);
  cudaError_t e;
  switch (plan.log2b) {
    case 5: e = launch_lb<5>(x, y, n, p, plan, w, out, stream); break;
    case 6: e = launch_lb<6>(x, y, n, p, plan, w, out, stream); break;
    case 7: e = launch_lb<7>(x, y, n, p, plan, w, out, stream); break;
    default: e = launch_lb<8>(x, y, n, p, plan, w, out, stream); break;
  }
  if (e != cudaSuccess) return e;
  if (sel) e = cudaMemcpyAsync(sel, w + plan.off_sel, sizeof(qdot_selection), cudaMemcpyDeviceToDevice, stream);
  return e;
}

}  // namespace qd
