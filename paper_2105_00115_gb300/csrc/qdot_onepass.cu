// One-pass qdot with deferred selection: blocked binning (32 <= B <= 256)
// and blocks of one component (B = 1).
//
// The class of a block depends on the global e_max and N_bins (eq.
// bin-score-def), which are only known after every component has been read.
// One read of x and y is still enough.
//
// 32 <= B <= 256.  For every block b the streaming kernel forms the candidate
// sums the block may need, of the form
//     H_b = sum q_half(x_i) q_half(y_i),  S_b = sum q_single(x_i) q_single(y_i),
//     D_b = sum x_i y_i,
// on a fixed-point grid below the block maximum u_b, and writes a record: an
// 8-byte slot per kept candidate and a 4-byte meta word with the block key
// s_b = ceil(log2 M_b) + u_b.  Which candidates a block keeps is speculated
// from a running lower bound of e_max (one, after the first items).  Once e_max
// and N_bins are known, a gather kernel takes for each block the candidate of
// the class eq. (precision-def) assigns to sigma_b = s_b - e_max - f + 1 and
// sums exactly; a candidate the speculation skipped is recomputed from x, y.
//
// B = 1.  Each warp item of 256 components is summed on the grid 2^(u - 52)
// of its own largest key u, every component quantized to the class it gets if
// the warp's bound of e_max were exact; the record keeps that bound, and the
// gather accepts the item when it was exact and recomputes it otherwise.
//
// Mapping: a warp streams items of 256 components (8 per lane) through a
// shared-memory ring with cp.async; a block spans B/8 lanes.  Candidates are
// formed at the scale of the block maximum, so 64-bit block sums stay below
// 2^62 and are exact up to one unit of the grid per component (relative
// error <= B 2^-52 of the block's sum of |x_i y_i|).  The primary candidate
// of a block goes through the FP64 pipe, one fused multiply-add per
// component on exponent-rescaled, class-rounded operands.
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
  unsigned done;       // CTAs that have written their partial (zeroed by k_op_select)
  unsigned pad;
  unsigned long long nredo;  // item records: items the gather listed for k_items_redo (zeroed by k_op_select)
  unsigned long long nfix;   // item records of blocks: blocks the gather listed for k_items_redo (zeroed too)
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

// Blocks of 32: from this n on, one-pass qdot keeps one record per item of
// 256 components (classes per block, the item summed on its own grid and
// recomputed if the bound of e_max it used was not exact) instead of
// candidate records per block.  Below it, warps have too few items for the
// bound to settle early.  Larger blocks keep the block records: with 4 or
// fewer blocks per item their gather is already short, and the items every
// warp recomputes (its first two) would cost more than they save.
constexpr long long kItemPathMinN = 1ll << 25;
// Blocks of 32 take the item records from kItemPathMinN on: one 16-byte
// record per 256 components instead of 12 to 20 bytes per block, and a
// gather that reads 16 times less.
constexpr bool kItemPathForBlocks = true;

// Blocks a gather CTA can queue for recomputation by its warps together.
constexpr int kRepairQueue = 512;

// The candidates a block with maximum key u (biased; kNone if empty) should
// get, after folding u into the warp's running bound e_lo of e_max.  e_lo
// also takes in erun, the bound shared by all warps, on the schedule above;
// each read has a few items' time to complete before its value is used.
// Fold the warp's largest key of this item, wmax (biased), and the shared
// word erun into the warp's bound e_lo; `raised` records the item of its
// last rise.
__device__ __forceinline__ void track_bound(int wmax, int lane, int iter, int* erun, int& e_lo, int& pending,
                                            int& raised) {
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
}

template <int LOG2B>
__device__ __forceinline__ unsigned candidates_wanted(int u, int lane, int iter, long long early_items, int f_spec,
                                                      int mh, int ms, int* erun, int& e_lo, int& pending,
                                                      int& raised) {
  constexpr int L = Map<LOG2B>::L;
  int wmax = u;
#pragma unroll
  for (int o = L; o < 32; o <<= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  track_bound(wmax, lane, iter, erun, e_lo, pending, raised);
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
    double aH = 0.0, aS = 0.0, aD = 0.0;  // the lane's chains (see qdot_chunk.cuh)
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
      u = chunk_general_chains<LOG2B>(cur, aH, aS, aD, M, zeros, kmin, bad);  // every candidate
      want = candidates_wanted<LOG2B>(u, lane, iter, early_items, f_spec, mh, ms, erun, e_lo, pending, raised);
      int kb;
      block_record_compact<LOG2B>(aH, aS, aD, M, u, want, sub, &kb, &ub, &mb, &slot, &meta, &half);
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
    hdr->nredo = 0ull;
    hdr->nfix = 0ull;
  }
  __syncthreads();
  const int e_max = sel->e_max, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  for (int k = threadIdx.x; k < kKeyCount; k += blockDim.x)
    sel->cls[k] = (uint8_t)precision_of((long long)kKeyMin + k - e_max - f + 1, mh, ms);
}

// The end of a gather kernel: this thread's partial sum acc and counts c
// (components per class, recomputed blocks) are summed over the CTA and
// published; the last CTA to arrive adds all partials in CTA order and writes
// the result, rounding once.
__device__ __noinline__ void finish_gather(i128 acc, unsigned long long (&c)[5], OpPart* __restrict__ parts,
                              OpHeader* __restrict__ hdr, qdot_selection* __restrict__ sel,
                              qdot_result* __restrict__ out, int slot0 = 0, bool final = true) {
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][5];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  acc = warp_sum_i128(acc);
  #pragma unroll
  for (int k = 0; k < 5; ++k) c[k] = warp_sum_u64(c[k]);
  if (lane == 0) {
    s_sum[w] = acc;
    #pragma unroll
    for (int k = 0; k < 5; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    OpPart p;
    p.sum = 0;
    #pragma unroll
    for (int k = 0; k < 4; ++k) p.cnt[k] = 0;
    p.repairs = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      p.sum += s_sum[i];
      #pragma unroll
      for (int k = 0; k < 4; ++k) p.cnt[k] += s_cnt[i][k];
      p.repairs += s_cnt[i][4];
    }
    parts[slot0 + blockIdx.x] = p;
    if (final) {
      __threadfence();  // the partial is visible before the arrival is counted
      s_last = atomicAdd(&hdr->done, 1u) == gridDim.x - 1;
    }
  }
  if (!final) return;  // a later kernel of the same stream adds the partials
  __syncthreads();
  if (!s_last) return;
  // last CTA: the exact sum of the partials (slots 0 .. slot0 + grid - 1, in
  // order), then one rounding
  __threadfence();
  const int np = slot0 + (int)gridDim.x;
  acc = 0;
  #pragma unroll
  for (int k = 0; k < 5; ++k) c[k] = 0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const unsigned long long* pw = reinterpret_cast<const unsigned long long*>(parts + i);
    const unsigned long long lo = __ldcg(pw), hi = __ldcg(pw + 1);
    acc += (i128)(((unsigned __int128)hi << 64) | lo);
    #pragma unroll
    for (int k = 0; k < 4; ++k) c[k] += __ldcg(&parts[i].cnt[k]);
    c[4] += __ldcg(&parts[i].repairs);
  }
  acc = warp_sum_i128(acc);
  #pragma unroll
  for (int k = 0; k < 5; ++k) c[k] = warp_sum_u64(c[k]);
  __syncthreads();  // s_sum, s_cnt are reused
  if (lane == 0) {
    s_sum[w] = acc;
    #pragma unroll
    for (int k = 0; k < 5; ++k) s_cnt[w][k] = c[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      acc += s_sum[i];
      #pragma unroll
      for (int k = 0; k < 5; ++k) c[k] += s_cnt[i][k];
    }
    sel->reserved[0] = (int32_t)(c[4] < 0x7FFFFFFFull ? c[4] : 0x7FFFFFFFull);
    qdot_result r;
    r.status = hdr->status;
    r.n_bins = sel->n_bins;
    r.e_max = sel->e_max;
    r.e_min = sel->e_min;
    r.f = sel->f;
    #pragma unroll
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
                                                   long long n, qdot_result* __restrict__ out,
                                                   qdot_trace_unit* __restrict__ trace) {
  __shared__ __align__(16) uint8_t s_lut[kKeyCount];  // filled as 32-bit words
  __shared__ long long s_qblk[kRepairQueue];  // blocks to recompute ...
  __shared__ int s_qinfo[kRepairQueue];       // ... with u << 2 | class
  __shared__ int s_nqueue;
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
    int src = keep ? QDOT_TRACE_SLOT0 : QDOT_TRACE_NONE;
    if (keep && cls != top) {  // a second kept candidate, or a missing one
      if (stored == kCandAll && cls == kHalf && blk >= n_early) stored = 0;  // never written
      if (stored & (1u << cls)) {
        const bool third = stored == kCandAll && cls == kHalf;
        v = third ? slot3[blk]  // blk < n_early by construction
                  : slots1[blk];
        src = third ? QDOT_TRACE_SLOT3 : QDOT_TRACE_SLOT1;
      } else {
        ++c_rep;
        keep = false;
        src = QDOT_TRACE_RECOMPUTED;
        const int q = atomicAdd(&s_nqueue, 1);
        if (q < kRepairQueue) {  // the CTA's warps recompute it together after the sweep
          s_qblk[q] = blk;
          s_qinfo[q] = (u << 2) | cls;
        } else {  // queue full: this thread recomputes it alone
          const long long rv = recompute_chain<LOG2B>(x, y, n, blk, u, cls);
          acc += candidate_to_fixed(rv, cls, u, LOG2B, lsb);
          if (trace) trace[blk] = qdot_trace_unit{rv, candidate_grid(cls, u, LOG2B), (uint8_t)cls, (uint8_t)src, 0};
        }
      }
    }
    if (trace && src != QDOT_TRACE_RECOMPUTED)
      trace[blk] = qdot_trace_unit{keep ? v : 0ll, keep ? candidate_grid(cls, u, LOG2B) : 0,
                                   (uint8_t)(mw ? cls : kZero), (uint8_t)src, 0};
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
    const long long v = recompute_chain_warp<LOG2B>(x, y, n, blk, u, cls, lane);
    if (lane == 0) {
      acc += candidate_to_fixed(v, cls, u, LOG2B, lsb);
      if (trace)
        trace[blk] = qdot_trace_unit{v, candidate_grid(cls, u, LOG2B), (uint8_t)cls, (uint8_t)QDOT_TRACE_RECOMPUTED, 0};
    }
  }
  acc += (i128)(((unsigned __int128)(unsigned long long)acc_hi << 64) | acc_lo);
  unsigned long long c[5] = {c_ph & 0xFFFFFFFFull, c_ph >> 32, c_sd & 0xFFFFFFFFull, c_sd >> 32, c_rep};
  finish_gather(acc, c, parts, hdr, sel, out);
}

// ---------------------------------------------------------------------------
// Blocks of one component (B = 1).
// ---------------------------------------------------------------------------

// Item record for B = 1: the item's sum on the grid 2^(u - 52) (u its
// largest key) and a meta word
//   u_biased | e_lo_biased << 12 | n_half << 24 | n_single << 33 | n_double << 42,
// bit 63 set when the gather must recompute the item (zeros, subnormals,
// non-finite values or the vectors' end inside it).
constexpr unsigned long long kItemRecompute = 1ull << 63;


// The largest key (biased) of the items the streaming warps take first (the
// first kSeedRounds items of every warp, in the streaming kernel's order)
// into the shared bound erun before the stream starts.  Without it a warp
// sums its first items with its own bound alone, which is far below e_max;
// with it those items start from the bound the warps would otherwise learn
// only after a few exchanges.  The items stay in L2 for the stream (about
// 0.7% of the vectors at 2^28).  Any value it writes is a key of the vectors,
// so a lower bound of e_max.
constexpr int kSeedRounds = 2;

__global__ void __launch_bounds__(kOpThreads) k_seed_bound(const double* __restrict__ x,
                                                           const double* __restrict__ y, long long n,
                                                           long long nwarps_stream, int* __restrict__ erun) {
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nitems = (n + kItem - 1) / kItem;
  int wmax = kNone;
  for (int r = 0; r < kSeedRounds; ++r) {
    const long long item = gwarp + r * nwarps_stream;
    if (item >= nitems) break;  // warp-uniform
    Chunk ch;
    load_item<8, true>(x, y, n, item, lane, ch);  // the layout does not matter for a maximum
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t a = ch.x[j], b = ch.y[j];
      const bool ok = ((ch.vmask >> j) & 1u) && !is_zero(a) && !is_zero(b) && !is_nonfinite(a) && !is_nonfinite(b);
      if (ok) wmax = max(wmax, exponent_of(a) + exponent_of(b) + 2046);
    }
  }
  wmax = __reduce_max_sync(0xffffffffu, wmax);
  if (lane == 0 && wmax != kNone) atomicMax(erun, wmax);
}

// Streaming kernel with item records.  LOG2B = 0: blocks of one component,
// each quantized to the class of its score key - e_lo - f_spec + 1.  LOG2B =
// 5..8: blocks of 2^LOG2B, each block's components to the class of the block
// score log2 B + u_b - e_lo - f_spec + 1.  Either is the true score if the
// warp's bound e_lo equals e_max and f equals f_spec (no empty blocks).
template <int LOG2B>
__global__ void __launch_bounds__(kOpThreads, kOpCtasPerSm) k_onepass_items(const double* __restrict__ x,
                                                                 const double* __restrict__ y, long long n,
                                                                 int f_spec, int mh, int ms, int* __restrict__ erun,
                                                                 WarpStats* __restrict__ wstats,
                                                                 long long* __restrict__ isum,
                                                                 unsigned long long* __restrict__ imeta,
                                                                 unsigned long long* __restrict__ iblk,
                                                                 uint8_t* __restrict__ tcls) {
  constexpr int LB = LOG2B ? LOG2B : 8;  // the item layout (blocks of one: that of 256)
  constexpr int L = Map<LB>::L;
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;
  const long long nitems = (n + kItem - 1) / kItem;
  const long long gwarp = ((long long)blockIdx.x * kOpThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kOpThreads) >> 5;
  int e_lo = kNone, pending = kNone, raised = 0, iter = 0;
  {  // the bound k_seed_bound left: the largest key of every warp's first items
    int seeded = kNone;
    if (lane == 0) seeded = *(volatile int*)erun;
    e_lo = max(kNone, __shfl_sync(0xffffffffu, seeded, 0));
  }
  extern __shared__ uint4 s_ring[];
  __shared__ RoundTab s_rtab;  // blocks of one: the rounding constants per class
  if (LOG2B == 0) {
    if (threadIdx.x < 4) round_tab_fill(&s_rtab, threadIdx.x);
    __syncthreads();
  }
  uint4* ring = s_ring + (threadIdx.x >> 5) * (kStages * kStageWords);
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    const long long item = gwarp + st * nwarps;
    if (item < nitems) issue_item<LB>(x, y, n, item, lane, ring + st * kStageWords);
    cp_async_commit();
  }
  int stage = 0;
  long long it = gwarp;
  Chunk cur;
  while (it < nitems) {
    {
      const long long ahead = it + (long long)(kStages - 1) * nwarps;
      const int st = stage == 0 ? kStages - 1 : stage - 1;
      if (ahead < nitems) issue_item<LB>(x, y, n, ahead, lane, ring + st * kStageWords);
      cp_async_commit();
    }
    cp_async_wait<kStages - 1>();
    read_item<LB>(ring + stage * kStageWords, n, it, lane, cur);
    stage = stage == kStages - 1 ? 0 : stage + 1;
    int key[8];
    int cmax = kNone;
    long long slot = 0;
    unsigned long long meta = kItemRecompute;
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      const int u = __reduce_max_sync(0xffffffffu, cmax);  // the item's largest key (biased)
      track_bound(u, lane, iter, erun, e_lo, pending, raised);
      const int a = e_lo + f_spec - 1;  // score = key - a
      double aF = 0.0;
      unsigned cnt = 0;  // per-class counts of the lane's components, 8-bit fields
      if (LOG2B == 0) {
        int cls[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {  // eq. (precision-def): PERF 0, HALF 1, SINGLE 2, DOUBLE 3
          const int sg = key[j] - a;
          cls[j] = (sg >= 0) + (sg >= mh) + (sg >= ms);
          cnt += 1u << (cls[j] << 3);
        }
        // a class count field is nonzero in the OR over the warp iff some lane has that class
        if ((__reduce_or_sync(0xffffffffu, cnt) & 0x00FFFFFFu) == 0u)
          acc_components<0>(cur, key, u, cls, aF);  // every component DOUBLE: nothing to round
        else
          acc_components_tab(cur, key, u, cls, &s_rtab, aF);
        if (tcls) {  // check output only (qdot_trace)
#pragma unroll
          for (int j = 0; j < 8; ++j) tcls[it * kItem + item_offset<LB>(lane, j)] = (uint8_t)cls[j];
        }
      } else {
        const int ub = group_max<L>(cmax);  // the block's largest key (biased)
        {  // one byte per block: u - u_b, saturated at 255 (the gather's per-block check)
          const unsigned du = (unsigned)min(u - ub, 255);
          unsigned long long word = 0;
#pragma unroll
          for (int g = 0; g < Map<LB>::BPI; ++g)
            word |= (unsigned long long)__shfl_sync(0xffffffffu, du, g * L) << (8 * g);
          if (lane == 0) iblk[it] = word;
        }
        const int sg = LB + ub - a;  // the block's score (M_b = B)
        const int cls = sg < 0 ? kPerf : (sg < mh ? kHalf : (sg < ms ? kSingle : kDouble));
        const unsigned prim = cls == kPerf ? 0u : 1u << cls;
        double aH2 = 0.0, aS2 = 0.0;
        acc_lane_mask<LB>(__reduce_or_sync(0xffffffffu, prim), 0u, cur, key, u, prim, aH2, aS2, aF);
        if (!prim) aF = 0.0;  // a perforated block adds nothing
        cnt = 8u << (cls << 3);
        if (tcls) {
#pragma unroll
          for (int j = 0; j < 8; ++j) tcls[it * kItem + item_offset<LB>(lane, j)] = (uint8_t)cls;
        }
      }
      long long v = __double2ll_rz(aF * 4503599627370496.0);  // onto the grid 2^(u - 52)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const unsigned ps = __reduce_add_sync(0xffffffffu, cnt & 0x00FF00FFu);         // PERF, SINGLE
      const unsigned hd = __reduce_add_sync(0xffffffffu, (cnt >> 8) & 0x00FF00FFu);  // HALF, DOUBLE
      slot = v;
      meta = (unsigned long long)u | ((unsigned long long)e_lo << 12) | ((unsigned long long)(hd & 0xFFFFu) << 24) |
             ((unsigned long long)(ps >> 16) << 33) | ((unsigned long long)(hd >> 16) << 42);
      nbins += LOG2B == 0 ? 8 : (sub == 0);  // nonzero components, or non-empty blocks
      emax_l = max(emax_l, u - 2046);
    } else {  // statistics only; the gather recomputes the item
      int wmax = kNone, nz = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint64_t a = cur.x[j], b = cur.y[j];
        const bool in = (cur.vmask >> j) & 1u;
        const bool fin = !(is_nonfinite(a) || is_nonfinite(b));
        bad |= in && !fin;
        const bool z = is_zero(a) || is_zero(b);
        zeros_l += in && fin && z;
        if (in && fin && !z) {
          const int k = exponent_of(a) + exponent_of(b) + 2046;
          ++nz;
          kmin = min(kmin, k);
          wmax = max(wmax, k);
        }
      }
      if (LOG2B == 0) {
        nbins += nz;
      } else {  // non-empty blocks; every lane takes part in the block's shuffles
        const int block_nz = group_sum_i<L>(nz);
        nbins += (sub == 0 && block_nz > 0);
      }
      wmax = __reduce_max_sync(0xffffffffu, wmax);
      track_bound(wmax, lane, iter, erun, e_lo, pending, raised);
      if (wmax != kNone) emax_l = max(emax_l, wmax - 2046);
    }
    if (lane == 0) {
      isum[it] = slot;
      imeta[it] = meta;
    }
    it += nwarps;
    ++iter;
  }
  cp_async_wait<0>();
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


// Gather of item records: an item whose bound e_lo was e_max, and f_spec f, adds
// its record; every other item goes to a list that k_items_redo sums again
// with the final classes.  The CTA takes kGatherPer x 256 records per round,
// kGatherPer per thread with independent loads; the rejected ones of a round
// are appended to the list together (one atomic per CTA and round).  The
// CTA's partial goes to parts[blockIdx.x]; k_items_redo adds the partials.
constexpr int kGatherPer = 4;

template <int LOG2B>
__global__ void __launch_bounds__(256, 2) k_op_gather_items(const long long* __restrict__ isum,
                                                     const unsigned long long* __restrict__ imeta, long long nitems,
                                                     int f_spec, qdot_selection* __restrict__ sel,
                                                     OpHeader* __restrict__ hdr, OpPart* __restrict__ parts,
                                                     const unsigned long long* __restrict__ iblk,
                                                     long long* __restrict__ redo, long long* __restrict__ fix,
                                                     qdot_trace_unit* __restrict__ trace) {
  __shared__ long long s_qitem[256 * kGatherPer];
  __shared__ int s_nqueue;
  __shared__ unsigned long long s_base;
  if (threadIdx.x == 0) s_nqueue = 0;
  __syncthreads();
  const int lsb = hdr->lsb;
  const bool ok = hdr->status == QDOT_OK;
  const unsigned anchor = (unsigned)(sel->e_max + 2046);  // the bound an exact item recorded
  const bool f_exact = sel->f == f_spec;
  // blocks: score = s_b - a with the anchor a = e_lo + f - 1 (biased keys)
  const int a_true = sel->e_max + 2046 + sel->f - 1;
  const int mh = sel->m_half, ms = sel->m_single;
  unsigned long long acc_lo = 0;
  long long acc_hi = 0;
  unsigned long long c[5] = {0, 0, 0, 0, 0};
  const long long G = gridDim.x;
  const long long T = blockDim.x;
  for (long long q0 = 0; ok && q0 * G + blockIdx.x < nitems; q0 += T * kGatherPer) {
    unsigned long long m[kGatherPer], bws[kGatherPer];
    long long v[kGatherPer];
    long long fx[LOG2B ? kGatherPer * Map<LOG2B ? LOG2B : 8>::BPI : 1];  // this thread's block entries
    int nfx = 0;
#pragma unroll
    for (int k = 0; k < kGatherPer; ++k) {  // independent loads first
      const long long i = (q0 + threadIdx.x + k * T) * G + blockIdx.x;
      m[k] = i < nitems ? imeta[i] : 0ull;
      v[k] = i < nitems ? isum[i] : 0ll;
      bws[k] = (LOG2B > 0 && i < nitems) ? iblk[i] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kGatherPer; ++k) {
      const long long i = (q0 + threadIdx.x + k * T) * G + blockIdx.x;
      if (i >= nitems) continue;
      bool accept = f_exact && !(m[k] & kItemRecompute) && (unsigned)((m[k] >> 12) & 0xFFFu) == anchor;
      unsigned flip = 0;
      if (LOG2B > 0 && !accept && !(m[k] & kItemRecompute)) {
        // blocks: the anchor was stale, but only blocks whose class the final
        // anchor changes matter (a block 255 or more keys below the item's
        // largest is recomputed with the whole item)
        const int a_used = (int)((m[k] >> 12) & 0xFFFu) + f_spec - 1;
        const int ui = (int)(m[k] & 0xFFFu);
        const unsigned long long bw = bws[k];
        bool far = false;
#pragma unroll
        for (int g = 0; g < Map<LOG2B ? LOG2B : 8>::BPI; ++g) {
          const int du = (int)((bw >> (8 * g)) & 0xFFu);
          far |= du == 255;
          const int sb = LOG2B + ui - du;
          flip |= precision_of(sb - a_used, mh, ms) != precision_of(sb - a_true, mh, ms) ? (1u << g) : 0u;
        }
        // the blocks' corrections are added apart from the record, which is exact
        // only while the item's grid 2^(u - 52) is not finer than the sum's
        const bool coarse = ui - 2046 - 52 >= lsb;
        if (far || !coarse) flip = 0;
        accept = !far && coarse;  // with flip != 0: the record now, its changed blocks in k_items_redo
      }
      if (flip) {  // entries: (1 << 62) | u << 50 | e_lo << 38 | block index
        const unsigned long long hi = (1ull << 62) | ((m[k] & 0xFFFull) << 50) | (((m[k] >> 12) & 0xFFFull) << 38);
        const long long b0 = i * Map<LOG2B ? LOG2B : 8>::BPI;
        for (unsigned f2 = flip; f2; f2 &= f2 - 1) fx[nfx++] = (long long)(hi | (unsigned long long)(b0 + __ffs(f2) - 1));
      }
      if (accept) {
        const unsigned nh = (unsigned)(m[k] >> 24) & 0x1FFu, ns = (unsigned)(m[k] >> 33) & 0x1FFu,
                       nd = (unsigned)(m[k] >> 42) & 0x1FFu;
        c[kHalf] += nh;
        c[kSingle] += ns;
        c[kDouble] += nd;
        c[kPerf] += kItem - nh - ns - nd;
        const int sh = (int)(m[k] & 0xFFFu) - 2046 - 52 - lsb;  // <= L - 52
        const int sl = min(max(sh, 0), 63), sr = min(max(-sh, 0), 63);
        const long long wv = v[k] >> sr;
        const unsigned long long lo = (unsigned long long)wv << sl;
        acc_lo += lo;
        acc_hi += ((wv >> 1) >> (63 - sl)) + (acc_lo < lo ? 1 : 0);
        if (trace)
          trace[i] = qdot_trace_unit{v[k], (int)(m[k] & 0xFFFu) - 2046 - 52, 255,
                                     (uint8_t)(flip ? QDOT_TRACE_ITEM_FIXED : QDOT_TRACE_ITEM), 0};
      } else {
        ++c[4];  // at most kGatherPer per thread and round
        s_qitem[atomicAdd(&s_nqueue, 1)] = i;
      }
    }
    if (LOG2B > 0) {  // block entries: one atomic per warp
      const int lane = threadIdx.x & 31;
      int incl = nfx;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      unsigned long long wbase = 0;
      if (lane == 31 && incl) wbase = atomicAdd(&hdr->nfix, (unsigned long long)incl);
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      for (int t = 0; t < nfx; ++t) fix[wbase + incl - nfx + t] = fx[t];
    }
    __syncthreads();
    const int nq = s_nqueue;
    if (threadIdx.x == 0 && nq) s_base = atomicAdd(&hdr->nredo, (unsigned long long)nq);
    __syncthreads();
    for (int t = threadIdx.x; t < nq; t += blockDim.x) redo[s_base + t] = s_qitem[t];
    __syncthreads();
    if (threadIdx.x == 0) s_nqueue = 0;
    __syncthreads();
  }
  const i128 acc = (i128)(((unsigned __int128)(unsigned long long)acc_hi << 64) | acc_lo);
  finish_gather(acc, c, parts, hdr, sel, nullptr, 0, false);
}

// The work the gather listed, summed again at streaming speed.
// 1. Blocks of 32 .. 256 whose class changed under the final anchor in an item
//    whose record the gather kept (its sum was formed with the stale anchor
//    a_used = e_lo + f_spec - 1; the final a_true is larger, so a block's class
//    can only drop): a warp takes 256 / B such blocks at once, B / 8 lanes per
//    block as in the streaming layout.  Each lane forms its chain with the
//    class the streaming kernel used and with the final class, exactly as the
//    streaming kernel forms a chain, and the difference of the truncated lane
//    values (on the item's grid 2^(u - 52), no finer than the sum's, which the
//    gather checked) is added to the sum.
// 2. Items the gather rejected: each summed with the final classes (the
//    selection's table) in the streaming kernel's arithmetic
//    (recompute_loaded_item); the warps take the list in turn and load each
//    item one ahead in registers.
// The gather's partials sit in parts[0 .. gather_grid - 1], this kernel's
// after them; the last CTA to finish adds them all in order and rounds once.
template <int LOG2B>
__global__ void __launch_bounds__(256, 2) k_items_redo(const double* __restrict__ x, const double* __restrict__ y,
                                                long long n, const long long* __restrict__ redo,
                                                const long long* __restrict__ fix, int f_spec,
                                                qdot_selection* __restrict__ sel, OpHeader* __restrict__ hdr,
                                                OpPart* __restrict__ parts, int gather_grid,
                                                qdot_result* __restrict__ out, qdot_trace_unit* __restrict__ trace,
                                                uint8_t* __restrict__ tcls) {
  constexpr int LB = LOG2B ? LOG2B : 8;
  constexpr int L = Map<LB>::L, BPI = Map<LB>::BPI, B = 1 << LB;
  __shared__ __align__(16) uint8_t s_lut[kKeyCount];  // filled as 32-bit words
  for (int i = threadIdx.x; i < kKeyCount / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(s_lut)[i] = reinterpret_cast<const uint32_t*>(sel->cls)[i];
  __syncthreads();
  const int lsb = hdr->lsb;
  const bool ok = hdr->status == QDOT_OK;
  const long long m = ok ? (long long)hdr->nredo : 0ll;
  const int lane = threadIdx.x & 31;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  i128 acc = 0;
  unsigned long long c[5] = {0, 0, 0, 0, 0};
  if (LOG2B > 0) {  // 1. changed blocks
    const long long nf = ok ? (long long)hdr->nfix : 0ll;
    const int a_true = sel->e_max + 2046 + sel->f - 1;
    const int mh = sel->m_half, ms = sel->m_single;
    const int g = lane / L, sub = lane % L;
    for (long long b0 = gwarp * BPI; b0 < nf; b0 += nwarps * BPI) {  // warp-uniform
      const long long idx = b0 + g;
      const bool have = idx < nf;
      const unsigned long long E = have ? (unsigned long long)fix[idx] : 0ull;
      const long long blk = (long long)(E & ((1ull << 38) - 1));
      const int u = (int)((E >> 50) & 0xFFFu), elo = (int)((E >> 38) & 0xFFFu);
      const long long item = blk / BPI;
      const int gi = (int)(blk % BPI);
      Chunk ch;
      ch.vmask = 0xFFu;
      if (have) {  // the block lies in a plain item, inside the vectors
        const long long base = item * kItem + item_offset<LB>(gi * L + sub, 0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double2 av = __ldcs(reinterpret_cast<const double2*>(x + base + 2 * L * j));
          const double2 bv = __ldcs(reinterpret_cast<const double2*>(y + base + 2 * L * j));
          ch.x[2 * j] = (uint64_t)__double_as_longlong(av.x);
          ch.x[2 * j + 1] = (uint64_t)__double_as_longlong(av.y);
          ch.y[2 * j] = (uint64_t)__double_as_longlong(bv.x);
          ch.y[2 * j + 1] = (uint64_t)__double_as_longlong(bv.y);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) ch.x[j] = ch.y[j] = 0ull;
      }
      int key[8];
      int cmax = kNone, kmin = INT_MAX;
      chunk_keys(ch, key, cmax, kmin);
      const int ub = group_max<L>(cmax);  // every lane joins its block's shuffles
      const int c_old = precision_of((long long)LB + ub - (elo + f_spec - 1), mh, ms);
      const int c_new = precision_of((long long)LB + ub - a_true, mh, ms);
      long long d = 0;
      if (have) {
        const unsigned p_old = c_old == kPerf ? 0u : 1u << c_old, p_new = c_new == kPerf ? 0u : 1u << c_new;
        double h = 0.0, sg = 0.0, a0 = 0.0, a1 = 0.0;
        acc_lane<LB, 3, 0u>(ch, key, u, p_old, h, sg, a0);
        acc_lane<LB, 3, 0u>(ch, key, u, p_new, h, sg, a1);
        d = (p_new ? __double2ll_rz(a1 * 4503599627370496.0) : 0ll) -
            (p_old ? __double2ll_rz(a0 * 4503599627370496.0) : 0ll);  // grid 2^(u - 52)
        if (tcls) {
#pragma unroll
          for (int j = 0; j < 8; ++j) tcls[item * kItem + item_offset<LB>(gi * L + sub, j)] = (uint8_t)c_new;
        }
      }
      d = group_sum<L>(d);
      if (have && sub == 0) {
        acc += candidate_to_fixed(d, kSingle, u - 2046, 8, lsb);  // exact: the gather checked the grid
        c[c_old] -= (unsigned long long)B;
        c[c_new] += (unsigned long long)B;
        if (trace) atomicAdd(reinterpret_cast<unsigned long long*>(&trace[item].value), (unsigned long long)d);
      }
    }
  }
  // 2. rejected items
  Chunk cur, nxt;
  long long j = gwarp;
  long long it = j < m ? redo[j] : 0;
  if (j < m) load_item<LB>(x, y, n, it, lane, cur);
  for (; j < m; j += nwarps) {
    const long long jn = j + nwarps;
    const long long itn = jn < m ? redo[jn] : 0;
    if (jn < m) load_item<LB>(x, y, n, itn, lane, nxt);  // in flight while this item is summed
    int u;
    const long long v = recompute_loaded_item<LOG2B>(x, y, n, it, cur, s_lut, lane, &u, c, tcls);
    if (lane == 0 && u != kNone) acc += candidate_to_fixed(v, kSingle, u, 8, lsb);  // grid 2^(u - 52)
    if (lane == 0 && trace)
      trace[it] = qdot_trace_unit{u != kNone ? v : 0ll, u != kNone ? u - 52 : 0, 255,
                                  (uint8_t)QDOT_TRACE_ITEM_RECOMPUTED, 0};
    cur = nxt;
    it = itn;
  }
  c[4] = 0;  // the gather counted the listed items
  finish_gather(acc, c, parts, hdr, sel, out, gather_grid, true);
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
                      char* ws, qdot_result* out, cudaStream_t st, TraceOut tr) {
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
                                                    nblocks, sel, hdr, parts, x, y, n, out, tr.units);
  return cudaGetLastError();
}

template <int LOG2B>
cudaError_t launch_items(const double* x, const double* y, int64_t n, const qdot_params* p, const OnePassPlan& pl,
                         char* ws, qdot_result* out, cudaStream_t st, TraceOut tr) {
  auto* sel = reinterpret_cast<qdot_selection*>(ws + pl.off_sel);
  auto* hdr = reinterpret_cast<OpHeader*>(ws + pl.off_hdr);
  auto* wst = reinterpret_cast<WarpStats*>(ws + pl.off_rec);
  auto* isum = reinterpret_cast<long long*>(ws + pl.off_misc);
  auto* imeta = reinterpret_cast<unsigned long long*>(ws + pl.off_meta);
  auto* parts = reinterpret_cast<OpPart*>(ws + pl.off_sel + align_up(sizeof(qdot_selection), 256) +
                                          align_up(sizeof(OpHeader), 256));
  const long long nitems = (n + kItem - 1) / kItem;
  // f if every block is non-empty (a lower bound of the real f)
  const long long nblocks = LOG2B ? (n + (1ll << LOG2B) - 1) >> LOG2B : n;
  const int f_spec = host_floor_log2_ratio(p->eps, p->split_budget ? (unsigned long long)nblocks : 1ull);
  const int mh = p->mant_reading ? 11 : 10, ms = p->mant_reading ? 24 : 23;
  cudaError_t e = cudaMemsetAsync(&hdr->erun, 0x80, sizeof(int), st);  // very negative
  if (e != cudaSuccess) return e;
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  static bool smem_set = false;
  if (!smem_set) {
    e = cudaFuncSetAttribute(k_onepass_items<LOG2B>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOpSmem);
    if (e != cudaSuccess) return e;
    smem_set = true;
  }
  auto* iblk = LOG2B ? reinterpret_cast<unsigned long long*>(ws + pl.off_slot3) : nullptr;
  k_seed_bound<<<pl.grid, kOpThreads, 0, st>>>(x, y, n, (long long)pl.grid * kOpWarps, &hdr->erun);
  if (ev0) cudaEventRecord(ev0, st);  // the streaming kernel alone
  k_onepass_items<LOG2B><<<pl.grid, kOpThreads, kOpSmem, st>>>(x, y, n, f_spec, mh, ms, &hdr->erun, wst, isum,
                                                                 imeta, iblk, tr.cls);
  if (ev1) cudaEventRecord(ev1, st);
  k_op_select<<<1, 1024, 0, st>>>(wst, pl.grid * kOpWarps, n, *p, sel, hdr);
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int gather_grid = 2 * sms, redo_grid = 2 * sms;  // 2 CTAs per SM each; 4 x sms partial slots
  auto* redo = reinterpret_cast<long long*>(ws + pl.off_slot1);
  auto* fix = LOG2B ? reinterpret_cast<long long*>(ws + pl.off_rec2) : nullptr;
  k_op_gather_items<LOG2B><<<gather_grid, 256, 0, st>>>(isum, imeta, nitems, f_spec, sel, hdr, parts, iblk, redo,
                                                         fix, tr.units);
  k_items_redo<LOG2B><<<redo_grid, 256, 0, st>>>(x, y, n, redo, fix, f_spec, sel, hdr, parts, gather_grid, out,
                                                  tr.units, tr.cls);
  return cudaGetLastError();
}

}  // namespace

bool one_pass_supported(int64_t n, const qdot_params* p, bool aligned16) {
  return aligned16 && n > 0 && (p->block == 1 || (p->block >= 32 && p->block <= 256));
}

// stream, select, gather (+ the item records' seed and redo)
int one_pass_launches(int64_t n, const qdot_params* p) { return plan_one_pass(n, p).items ? 5 : 3; }

const char* one_pass_stream_kernel(int64_t n, const qdot_params* p) {
  return plan_one_pass(n, p).items ? "k_onepass_items" : "k_onepass";
}

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
  pl.items = p->block == 1 || (kItemPathForBlocks && p->block == 32 && n >= kItemPathMinN);
  if (pl.items) {  // one record per item: its sum and its meta word
    const long long nitems = (n + kItem - 1) / kItem;
    pl.off_misc = off;
    off = align_up(off + sizeof(long long) * (size_t)nitems, 256);
    pl.off_meta = off;
    off = align_up(off + sizeof(unsigned long long) * (size_t)nitems, 256);
    pl.off_slot1 = off;  // the list of items the gather rejects (k_items_redo)
    off = align_up(off + sizeof(long long) * (size_t)nitems, 256);
    if (p->block >= 32) {
      pl.off_slot3 = off;  // per item: how far each block's largest key lies below the item's
      off = align_up(off + sizeof(unsigned long long) * (size_t)nitems, 256);
      pl.off_rec2 = off;  // the list of blocks whose class the final selection changed
      off = align_up(off + sizeof(long long) * (size_t)nblocks, 256);
    }
    pl.total = off;
    return pl;
  }
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
                            cudaStream_t stream, TraceOut tr) {
  char* w = static_cast<char*>(ws);
  cudaError_t e;
  switch (plan.log2b) {
    case 0: e = launch_items<0>(x, y, n, p, plan, w, out, stream, tr); break;
    case 5: e = plan.items ? launch_items<5>(x, y, n, p, plan, w, out, stream, tr) : launch_lb<5>(x, y, n, p, plan, w, out, stream, tr); break;
    case 6: e = plan.items ? launch_items<6>(x, y, n, p, plan, w, out, stream, tr) : launch_lb<6>(x, y, n, p, plan, w, out, stream, tr); break;
    case 7: e = plan.items ? launch_items<7>(x, y, n, p, plan, w, out, stream, tr) : launch_lb<7>(x, y, n, p, plan, w, out, stream, tr); break;
    default: e = plan.items ? launch_items<8>(x, y, n, p, plan, w, out, stream, tr) : launch_lb<8>(x, y, n, p, plan, w, out, stream, tr); break;
  }
  if (e != cudaSuccess) return e;
  if (sel) e = cudaMemcpyAsync(sel, w + plan.off_sel, sizeof(qdot_selection), cudaMemcpyDeviceToDevice, stream);
  return e;
}

}  // namespace qd
