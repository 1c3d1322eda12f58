// Batched qdot: many independent pairs (x_j, y_j) of uneven lengths, each a
// full qdot (Algorithm 3 with blocked binning, 32 <= B <= 256), in one
// persistent streaming launch.
//
//   k_bplan    one CTA: per-pair block and work-group counts, exclusive scans,
//              argument checks (16-byte alignment, n >= 0), per-pair state.
//   k_bstream  persistent: the warps split the concatenated warp items (256
//              components each) of all pairs into equal contiguous ranges;
//              every block's candidate sums go to a record as in the one-pass
//              kernel; per-pair statistics are merged with one set of atomics
//              per (warp, pair) run.
//   k_bfinal   one CTA per pair: f = floor(log2(eps / N_bins)) exactly, the
//              class of every block record (eq. bin-score-def and eq.
//              precision-def), exact fixed-point sum, one rounding.
#include <climits>

#include "qdot_chunk.cuh"
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

using namespace chunk;

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;

struct PairStats {
  int e_max;                // max block maximum u_b (kNone if none)
  int e_min;                // min component key
  int status;               // QDOT_OK, QDOT_ERR_ARG or QDOT_ERR_NONFINITE
  int f_spec;               // f if every block of the pair is non-empty (a lower bound of f)
  unsigned long long nbins; // non-empty blocks
  unsigned long long zeros; // ZERO components
  int e_run;                // running lower bound of e_max shared by the warps (biased), for speculation
  int pad2;
  long long pad3;
};

struct BatchHeader {
  long long total_groups;
  long long total_blocks;
  int status;               // QDOT_OK or QDOT_ERR_WORKSPACE
  int pad;
};

__global__ void __launch_bounds__(1024) k_bplan(const double* const* __restrict__ xs,
                                                const double* const* __restrict__ ys,
                                                const long long* __restrict__ ns, int count, int log2b,
                                                double eps, int split_budget,
                                                long long rec_capacity, long long* __restrict__ gpre,
                                                long long* __restrict__ bpre, PairStats* __restrict__ ps,
                                                BatchHeader* __restrict__ hdr) {
  __shared__ long long s_g[1024], s_b[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (count + T - 1) / T;
  const int lo = min(count, t * per), hi = min(count, lo + per);
  long long g = 0, b = 0;
  for (int p = lo; p < hi; ++p) {
    const long long n = ns[p];
    const bool aligned = ((reinterpret_cast<uintptr_t>(xs[p]) | reinterpret_cast<uintptr_t>(ys[p])) & 15u) == 0;
    const bool ok = n >= 0 && (n == 0 || (aligned && xs[p] && ys[p]));
    const long long nb = ok ? ((n + (1ll << log2b) - 1) >> log2b) : 0;
    b += nb;
    g += ok ? (n + kItem - 1) / kItem : 0;
    PairStats s;
    s.e_max = kNone;
    s.e_min = INT_MAX;
    s.status = ok ? QDOT_OK : QDOT_ERR_ARG;
    s.f_spec = nb > 0 ? floor_log2_ratio(eps, split_budget ? (unsigned long long)nb : 1ull) : 0;
    s.nbins = 0;
    s.zeros = 0;
    s.e_run = kNone;
    s.pad2 = 0;
    s.pad3 = 0;
    ps[p] = s;
  }
  s_g[t] = g;
  s_b[t] = b;
  __syncthreads();
  // inclusive scan (Hillis-Steele) of the per-thread sums
  for (int o = 1; o < T; o <<= 1) {
    long long vg = t >= o ? s_g[t - o] : 0, vb = t >= o ? s_b[t - o] : 0;
    __syncthreads();
    s_g[t] += vg;
    s_b[t] += vb;
    __syncthreads();
  }
  long long go = t ? s_g[t - 1] : 0, bo = t ? s_b[t - 1] : 0;
  for (int p = lo; p < hi; ++p) {
    gpre[p] = go;
    bpre[p] = bo;
    const long long n = ns[p];
    const bool ok = ps[p].status == QDOT_OK;
    bo += ok ? ((n + (1ll << log2b) - 1) >> log2b) : 0;
    go += ok ? (n + kItem - 1) / kItem : 0;
  }
  if (t == T - 1) {
    gpre[count] = s_g[T - 1];
    bpre[count] = s_b[T - 1];
    hdr->total_groups = s_g[T - 1];
    hdr->total_blocks = s_b[T - 1];
    hdr->status = s_b[T - 1] > rec_capacity ? QDOT_ERR_WORKSPACE : QDOT_OK;
    hdr->pad = 0;
  }
}

// Largest p with gpre[p] <= gg (pairs with no groups are skipped by the scan).
__device__ __forceinline__ int find_pair(const long long* __restrict__ gpre, int count, long long gg) {
  int lo = 0, hi = count;  // gpre[lo] <= gg < gpre[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (gpre[mid] <= gg)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// THREADS per CTA; STAGED: items staged through shared memory with cp.async
// (one item ahead), else double-buffered in registers.
template <int LOG2B, int THREADS, bool STAGED>
__global__ void __launch_bounds__(THREADS, 768 / THREADS) k_bstream(const double* const* __restrict__ xs,
                                                                  const double* const* __restrict__ ys,
                                                                  const long long* __restrict__ ns, int count,
                                                                  const long long* __restrict__ gpre,
                                                                  const long long* __restrict__ bpre,
                                                                  PairStats* __restrict__ ps,
                                                                  const BatchHeader* __restrict__ hdr,
                                                                  BlockRec* __restrict__ recs, int mh, int ms) {
  constexpr int L = Map<LOG2B>::L, BPI = Map<LOG2B>::BPI;
  if (hdr->status != QDOT_OK) return;
  const int lane = threadIdx.x & 31;
  const int g = lane / L, sub = lane % L;
  const long long total = hdr->total_groups;  // warp items over all pairs
  const long long gwarp = ((long long)blockIdx.x * THREADS + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * THREADS) >> 5;
  const long long per = (total + nwarps - 1) / nwarps;
  const long long g0 = min(total, gwarp * per), g1 = min(total, g0 + per);
  if (g0 >= g1) return;

  // statistics of the current run of items of one pair
  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;
  auto flush = [&](int p) {
    const int emax = __reduce_max_sync(0xffffffffu, emax_l);
    const int km = __reduce_min_sync(0xffffffffu, kmin);
    const int bd = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
    const unsigned long long nb = warp_sum_u64((unsigned long long)nbins);
    const unsigned long long zr = warp_sum_u64((unsigned long long)zeros_l);
    if (lane == 0) {
      if (emax != kNone) atomicMax(&ps[p].e_max, emax);
      if (km != INT_MAX) atomicMin(&ps[p].e_min, km - 2046);
      if (bd) atomicCAS(&ps[p].status, QDOT_OK, QDOT_ERR_NONFINITE);
      if (nb) atomicAdd(&ps[p].nbins, nb);
      if (zr) atomicAdd(&ps[p].zeros, zr);
    }
    nbins = zeros_l = 0;
    emax_l = kNone;
    kmin = INT_MAX;
    bad = 0;
  };

  extern __shared__ uint4 s_bring[];
  uint4* ring = STAGED ? s_bring + (threadIdx.x >> 5) * (2 * kStageWords) : nullptr;
  long long gg = g0;
  int p = find_pair(gpre, count, g0);
  // speculation state of the current pair (see the one-pass kernel): e_lo is
  // a lower bound of the pair's e_max; the first two items of the warp in a
  // pair get every candidate
  int e_lo = kNone, piter = 0;
  Chunk cur, nxt;
  if (STAGED) {
    issue_item<LOG2B>(xs[p], ys[p], ns[p], gg - gpre[p], lane, ring);
    cp_async_commit();
  } else {
    load_item<LOG2B>(xs[p], ys[p], ns[p], gg - gpre[p], lane, cur);
  }
  int stage = 0;
  while (gg < g1) {
    // next item of this warp, possibly in the next pair
    const long long ngg = gg + 1;
    int np = p;
    while (np + 1 < count && ngg >= gpre[np + 1]) ++np;
    if (STAGED) {
      if (ngg < g1) issue_item<LOG2B>(xs[np], ys[np], ns[np], ngg - gpre[np], lane, ring + (stage ^ 1) * kStageWords);
      cp_async_commit();
      cp_async_wait<1>();  // this lane's copies of item gg have landed
      read_item<LOG2B>(ring + stage * kStageWords, ns[p], gg - gpre[p], lane, cur);
      stage ^= 1;
    } else if (ngg < g1) {
      load_item<LOG2B>(xs[np], ys[np], ns[np], ngg - gpre[np], lane, nxt);
    }
    long long aH = 0, aS = 0;
    double aD = 0.0;
    int M = 0, zeros = 0, u;
    int key[8];
    int cmax = kNone;
    unsigned cands = kCandAll, top = kCandD;
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      u = group_max<L>(cmax);
      M = 8;
      int wmax = u;
#pragma unroll
      for (int o = L; o < 32; o <<= 1) wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
      if ((piter & 7) == 1) {  // the pair's shared bound, every 8 items
        int seen = kNone;
        if (lane == 0) seen = *(volatile int*)&ps[p].e_run;
        e_lo = max(e_lo, __shfl_sync(0xffffffffu, seen, 0));
      }
      if (wmax > e_lo) {
        e_lo = wmax;
        if (lane == 0) atomicMax(&ps[p].e_run, wmax);
      }
      unsigned want = kCandAll;
      if (piter >= 4) {  // windows wider than the single call's: a pair's warps see less of it
        const int sig_hi = LOG2B + u - e_lo - ps[p].f_spec + 1;  // >= the block's score
        want = 0;
        if (sig_hi >= ms) want |= kCandD;
        if (sig_hi >= mh && sig_hi - 10 < ms) want |= kCandS;
        if (sig_hi >= 0 && sig_hi - 8 < mh) want |= kCandH;
      }
      cands = __reduce_or_sync(0xffffffffu, want);
      top = cands ? (1u << (31 - __clz((int)cands))) : kCandD;
      acc_fast_mask<LOG2B>(cands, cur, key, u, aH, aS, aD);
    } else {
      u = chunk_general<LOG2B>(cur, aH, aS, aD, M, zeros, kmin, bad);
    }
    int kb, ub, mb;
    const long long word = block_record_word<LOG2B>(aH, aS, aD, M, u, cands, sub, &kb, &ub, &mb, top);
    const long long lb = (gg - gpre[p]) * BPI + g;  // block index within pair p
    const long long nblk_p = bpre[p + 1] - bpre[p];
    zeros_l += zeros;
    if (lb < nblk_p) {
      if (mb > 0) {
        nbins += (sub == 0);
        emax_l = max(emax_l, ub);
      }
      if (sub < 4) reinterpret_cast<long long*>(recs + bpre[p] + lb)[sub] = word;
    }
    if (np != p) {
      flush(p);
      e_lo = kNone;
      piter = 0;
    } else {
      ++piter;
    }
    if (!STAGED) cur = nxt;
    gg = ngg;
    p = np;
  }
  if (STAGED) cp_async_wait<0>();
  flush(p < count ? p : count - 1);
}

// ---------------------------------------------------------------------------
// Blocks of 32: item records per pair (the single call's item path, pair by
// pair).  Every warp item of pair p is summed once with the class its blocks
// get under the pair's running bound e_lo of e_max (one chain per lane, the
// single call's arithmetic) and recorded: its sum on the grid 2^(u - 52), a
// meta word (u, e_lo, class counts, or "recompute"), and each block's
// distance below u.  k_bfinal_items then takes each record as it is, takes it
// and lists the blocks whose class the pair's final anchor changed, or lists
// the whole item; k_bredo sums the listed work again and adds it to the
// pair's sum; k_bfinish rounds each pair once.
// ---------------------------------------------------------------------------
constexpr unsigned long long kBItemRecompute = 1ull << 63;

struct BPairSlot {
  const double* x;
  const double* y;
  long long n, start, end;  // length and item range [start, end) of the pair
};

template <int LOG2B, int THREADS>
__global__ void __launch_bounds__(THREADS, 768 / THREADS) k_bstream_items(
    const double* const* __restrict__ xs, const double* const* __restrict__ ys, const long long* __restrict__ ns,
    int count, const long long* __restrict__ gpre, PairStats* __restrict__ ps, const BatchHeader* __restrict__ hdr,
    long long* __restrict__ isum, unsigned long long* __restrict__ imeta, unsigned long long* __restrict__ iblk,
    int mh, int ms) {
  constexpr int L = Map<LOG2B>::L, BPI = Map<LOG2B>::BPI;
  if (hdr->status != QDOT_OK) return;
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  const long long total = hdr->total_groups;  // warp items over all pairs
  const long long gwarp = ((long long)blockIdx.x * THREADS + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * THREADS) >> 5;
  const long long per = (total + nwarps - 1) / nwarps;
  const long long g0 = min(total, gwarp * per), g1 = min(total, g0 + per);
  if (g0 >= g1) return;

  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;
  auto flush = [&](int p) {
    const int emax = __reduce_max_sync(0xffffffffu, emax_l);
    const int km = __reduce_min_sync(0xffffffffu, kmin);
    const int bd = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
    const unsigned long long nb = warp_sum_u64((unsigned long long)nbins);
    const unsigned long long zr = warp_sum_u64((unsigned long long)zeros_l);
    if (lane == 0) {
      if (emax != kNone) atomicMax(&ps[p].e_max, emax);
      if (km != INT_MAX) atomicMin(&ps[p].e_min, km - 2046);
      if (bd) atomicCAS(&ps[p].status, QDOT_OK, QDOT_ERR_NONFINITE);
      if (nb) atomicAdd(&ps[p].nbins, nb);
      if (zr) atomicAdd(&ps[p].zeros, zr);
    }
    nbins = zeros_l = 0;
    emax_l = kNone;
    kmin = INT_MAX;
    bad = 0;
  };

  extern __shared__ uint4 s_bring[];
  uint4* ring = s_bring + (threadIdx.x >> 5) * (2 * kStageWords);
  // The pair of the next item to load, in a per-warp shared-memory slot that
  // lane 0 rewrites when the stream crosses into a later pair: an item reads
  // it with broadcast shared loads instead of loading the pair's entries of
  // xs, ys, ns and gpre from global memory (those loads stalled every item;
  // registers for them would spill).
  __shared__ BPairSlot s_pair[THREADS / 32];
  BPairSlot* slot = s_pair + (threadIdx.x >> 5);
  long long gg = g0;
  int p = find_pair(gpre, count, g0);
  // the pair's running bound of e_max: this warp's largest key so far, and
  // every 2 items the pair's shared word (read 2 items before it is used)
  int e_lo = kNone, pending = kNone, piter = 0;
  int f_spec = ps[p].f_spec;
  if (lane == 0) *slot = BPairSlot{xs[p], ys[p], ns[p], gpre[p], gpre[p + 1]};
  __syncwarp();
  long long crem = slot->n - (gg - slot->start) * kItem;  // components of item gg and after it in its pair
  issue_item<LOG2B>(slot->x, slot->y, slot->n, gg - slot->start, lane, ring);
  cp_async_commit();
  int stage = 0;
  Chunk cur;
  while (gg < g1) {
    const long long ngg = gg + 1;
    int np = p;
    if (ngg < g1 && ngg >= slot->end) {  // the next item lies in a later pair (empty pairs have no items)
      np = p + 1;
      while (np + 1 < count && ngg >= gpre[np + 1]) ++np;
      __syncwarp();  // every lane has read the slot
      if (lane == 0) *slot = BPairSlot{xs[np], ys[np], ns[np], gpre[np], gpre[np + 1]};
      __syncwarp();
    }
    const BPairSlot nx = *slot;
    if (ngg < g1) issue_item<LOG2B>(nx.x, nx.y, nx.n, ngg - nx.start, lane, ring + (stage ^ 1) * kStageWords);
    cp_async_commit();
    cp_async_wait<1>();  // this lane's copies of item gg have landed
    read_item<LOG2B>(ring + stage * kStageWords, crem, 0, lane, cur);  // item 0 of the rest of its pair
    crem = nx.n - (ngg - nx.start) * kItem;
    stage ^= 1;
    int key[8];
    int cmax = kNone;
    long long slot = 0;
    unsigned long long meta = kBItemRecompute, bw = 0;
    if ((piter & 1) == 1) {  // exchange with the pair's shared word
      const int seen = __shfl_sync(0xffffffffu, pending, 0);
      if (lane == 0) pending = *(volatile int*)&ps[p].e_run;
      e_lo = max(e_lo, seen);
    }
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      const int u = __reduce_max_sync(0xffffffffu, cmax);  // the item's largest key (biased)
      if (u > e_lo) {
        e_lo = u;
        if (lane == 0) atomicMax(&ps[p].e_run, u);
      }
      const int ub = group_max<L>(cmax);  // the block's largest key (biased)
      {
        const unsigned du = (unsigned)min(u - ub, 255);
#pragma unroll
        for (int g = 0; g < BPI; ++g) bw |= (unsigned long long)__shfl_sync(0xffffffffu, du, g * L) << (8 * g);
      }
      const int sg = LOG2B + ub - (e_lo + f_spec - 1);  // the block's score (M_b = B) under the bound
      const int cls = sg < 0 ? kPerf : (sg < mh ? kHalf : (sg < ms ? kSingle : kDouble));
      const unsigned prim = cls == kPerf ? 0u : 1u << cls;
      double aH2 = 0.0, aS2 = 0.0, aF = 0.0;
      acc_lane_mask<LOG2B>(__reduce_or_sync(0xffffffffu, prim), 0u, cur, key, u, prim, aH2, aS2, aF);
      if (!prim) aF = 0.0;  // a perforated block adds nothing
      const unsigned cnt = 8u << (cls << 3);
      long long v = __double2ll_rz(aF * 4503599627370496.0);  // onto the grid 2^(u - 52)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const unsigned pcs = __reduce_add_sync(0xffffffffu, cnt & 0x00FF00FFu);         // PERF, SINGLE
      const unsigned hd = __reduce_add_sync(0xffffffffu, (cnt >> 8) & 0x00FF00FFu);  // HALF, DOUBLE
      slot = v;
      meta = (unsigned long long)u | ((unsigned long long)e_lo << 12) | ((unsigned long long)(hd & 0xFFFFu) << 24) |
             ((unsigned long long)(pcs >> 16) << 33) | ((unsigned long long)(hd >> 16) << 42);
      nbins += (sub == 0);  // a plain item's blocks are all non-empty
      emax_l = max(emax_l, ub - 2046);
    } else {  // statistics only; k_bfinal_items lists the item for recomputation
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
      const int block_nz = group_sum_i<L>(nz);  // every lane takes part in the block's shuffles
      nbins += (sub == 0 && block_nz > 0);
      wmax = __reduce_max_sync(0xffffffffu, wmax);
      if (wmax != kNone) {
        emax_l = max(emax_l, wmax - 2046);
        if (wmax > e_lo) {
          e_lo = wmax;
          if (lane == 0) atomicMax(&ps[p].e_run, wmax);
        }
      }
    }
    if (lane == 0) {
      isum[gg] = slot;
      imeta[gg] = meta;
      iblk[gg] = bw;
    }
    if (np != p) {  // the next item belongs to another pair
      flush(p);
      e_lo = kNone;
      pending = kNone;
      piter = 0;
      f_spec = ps[np].f_spec;
    } else {
      ++piter;
    }
    gg = ngg;
    p = np;
  }
  cp_async_wait<0>();
  flush(p < count ? p : count - 1);
}

// Per pair: the exact sum (128-bit two's complement in two words, so that
// k_bredo can add to it with 64-bit atomics), class counts, the selection,
// and how much work k_bfinal_items listed.
struct PairPart {
  unsigned long long lo, hi;
  unsigned long long cnt[4];
  long long nfix, nredo;
  int e_max, f, lsb, status;
};

__device__ __forceinline__ void atomic_add_i128(unsigned long long* lo, unsigned long long* hi, i128 v) {
  const unsigned long long vl = (unsigned long long)(u128)v, vh = (unsigned long long)((u128)v >> 64);
  const unsigned long long old = atomicAdd(lo, vl);
  atomicAdd(hi, vh + (old + vl < old ? 1ull : 0ull));  // the carry out of the low word
}

// One CTA per pair: f and the pair's final anchor; every item record taken as
// it is, taken with its changed blocks listed (fix[bpre[p] + k]: block index
// within the pair | u << 38 | e_lo << 50), or listed whole (redo[gpre[p] + k]:
// item index within the pair).  The same checks as the single call's gather.
template <int LOG2B>
__global__ void __launch_bounds__(256) k_bfinal_items(const long long* __restrict__ ns,
                                                      const long long* __restrict__ gpre,
                                                      const long long* __restrict__ bpre,
                                                      const PairStats* __restrict__ ps,
                                                      const BatchHeader* __restrict__ hdr,
                                                      const long long* __restrict__ isum,
                                                      const unsigned long long* __restrict__ imeta,
                                                      const unsigned long long* __restrict__ iblk,
                                                      long long* __restrict__ fix, long long* __restrict__ redo,
                                                      PairPart* __restrict__ pp, qdot_params prm) {
  constexpr int BPI = Map<LOG2B>::BPI;
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][4];
  __shared__ int s_nfix, s_nredo;
  const int p = blockIdx.x;
  const PairStats st = ps[p];
  const int status = hdr->status != QDOT_OK ? hdr->status : st.status;
  const long long nb = (long long)st.nbins;
  const int e_max = nb > 0 ? st.e_max : 0;
  const int f = (status == QDOT_OK && nb > 0)
                    ? floor_log2_ratio(prm.eps, prm.split_budget ? (unsigned long long)nb : 1ull)
                    : 0;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  const int lsb = e_max - fixed_point_bits(ns[p] > 0 ? ns[p] : 1);
  const int a_true = e_max + 2046 + f - 1;
  const unsigned anchor = (unsigned)(e_max + 2046);
  const bool f_exact = f == st.f_spec;
  if (threadIdx.x == 0) {
    s_nfix = 0;
    s_nredo = 0;
  }
  __syncthreads();
  unsigned long long acc_lo = 0;
  long long acc_hi = 0;
  unsigned long long c[4] = {0, 0, 0, 0};
  if (status == QDOT_OK) {
    for (long long i = gpre[p] + threadIdx.x; i < gpre[p + 1]; i += blockDim.x) {
      const unsigned long long m = imeta[i];
      const long long v = isum[i];
      bool accept = f_exact && !(m & kBItemRecompute) && (unsigned)((m >> 12) & 0xFFFu) == anchor;
      unsigned flip = 0;
      bool whole = (m & kBItemRecompute) != 0;
      if (!accept && !whole) {
        const int a_used = (int)((m >> 12) & 0xFFFu) + st.f_spec - 1;
        const int ui = (int)(m & 0xFFFu);
        const unsigned long long bw = iblk[i];
        bool far = false;
#pragma unroll
        for (int g = 0; g < BPI; ++g) {
          const int du = (int)((bw >> (8 * g)) & 0xFFu);
          far |= du == 255;
          const int sb = LOG2B + ui - du;
          flip |= precision_of(sb - a_used, mh, ms) != precision_of(sb - a_true, mh, ms) ? (1u << g) : 0u;
        }
        const bool coarse = ui - 2046 - 52 >= lsb;  // corrections added apart are exact
        whole = far || (flip && !coarse);
        accept = !whole;
      }
      if (accept) {
        const unsigned nh = (unsigned)(m >> 24) & 0x1FFu, ns_ = (unsigned)(m >> 33) & 0x1FFu,
                       nd = (unsigned)(m >> 42) & 0x1FFu;
        c[kHalf] += nh;
        c[kSingle] += ns_;
        c[kDouble] += nd;
        c[kPerf] += kItem - nh - ns_ - nd;
        const int sh = (int)(m & 0xFFFu) - 2046 - 52 - lsb;
        const int sl = min(max(sh, 0), 63), sr = min(max(-sh, 0), 63);
        const long long wv = v >> sr;
        const unsigned long long lo = (unsigned long long)wv << sl;
        acc_lo += lo;
        acc_hi += ((wv >> 1) >> (63 - sl)) + (acc_lo < lo ? 1 : 0);
        if (flip) {
          const unsigned long long hi = ((m & 0xFFFull) << 38) | (((m >> 12) & 0xFFFull) << 50);
          const long long lb0 = (i - gpre[p]) * BPI;
          for (unsigned f2 = flip; f2; f2 &= f2 - 1) {
            const int k = atomicAdd(&s_nfix, 1);  // at most the pair's block count
            fix[bpre[p] + k] = (long long)(hi | (unsigned long long)(lb0 + __ffs(f2) - 1));
          }
        }
      } else {
        const int k = atomicAdd(&s_nredo, 1);
        redo[gpre[p] + k] = i - gpre[p];
      }
    }
  }
  i128 acc = (i128)(((unsigned __int128)(unsigned long long)acc_hi << 64) | acc_lo);
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
    PairPart r;
    r.lo = (unsigned long long)(u128)acc;
    r.hi = (unsigned long long)((u128)acc >> 64);
    for (int k = 0; k < 4; ++k) r.cnt[k] = c[k];
    r.nfix = s_nfix;
    r.nredo = s_nredo;
    r.e_max = e_max;
    r.f = f;
    r.lsb = lsb;
    r.status = status;
    pp[p] = r;
  }
}

// One CTA: exclusive scans of the listed blocks and items over the pairs.
__global__ void __launch_bounds__(1024) k_bscan(const PairPart* __restrict__ pp, int count,
                                                long long* __restrict__ fpre, long long* __restrict__ rpre) {
  __shared__ long long s_f[1024], s_r[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int per = (count + T - 1) / T;
  const int lo = min(count, t * per), hi = min(count, lo + per);
  long long a = 0, b = 0;
  for (int p = lo; p < hi; ++p) {
    a += pp[p].nfix;
    b += pp[p].nredo;
  }
  s_f[t] = a;
  s_r[t] = b;
  __syncthreads();
  for (int o = 1; o < T; o <<= 1) {
    const long long va = t >= o ? s_f[t - o] : 0, vb = t >= o ? s_r[t - o] : 0;
    __syncthreads();
    s_f[t] += va;
    s_r[t] += vb;
    __syncthreads();
  }
  long long ra = s_f[t] - a, rb = s_r[t] - b;
  for (int p = lo; p < hi; ++p) {
    fpre[p] = ra;
    rpre[p] = rb;
    ra += pp[p].nfix;
    rb += pp[p].nredo;
  }
  if (t == T - 1) {
    fpre[count] = s_f[T - 1];
    rpre[count] = s_r[T - 1];
  }
}

// The listed work of every pair, added to the pair's sum with 64-bit atomics.
// 1. Listed blocks: a warp takes 256 / B of them at once (B / 8 lanes each)
//    from its contiguous range of the concatenated lists; each lane forms its
//    chain with the class the stream used and with the final one, and the
//    difference on the item's grid (no finer than the pair's sum, which
//    k_bfinal_items checked) goes to the pair's sum.
// 2. Listed items: one per warp, summed whole with the pair's final classes.
template <int LOG2B>
__global__ void __launch_bounds__(256, 2) k_bredo(const double* const* __restrict__ xs,
                                               const double* const* __restrict__ ys,
                                               const long long* __restrict__ ns, int count,
                                               const long long* __restrict__ gpre,
                                               const long long* __restrict__ bpre,
                                               const PairStats* __restrict__ ps,
                                               const long long* __restrict__ fix,
                                               const long long* __restrict__ redo,
                                               const long long* __restrict__ fpre,
                                               const long long* __restrict__ rpre, PairPart* __restrict__ pp,
                                               int mh, int ms) {
  constexpr int L = Map<LOG2B>::L, BPI = Map<LOG2B>::BPI, B = 1 << LOG2B;
  const int lane = threadIdx.x & 31, g = lane / L, sub = lane % L;
  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  // the pair of global entry e in a list with prefix `pre` (pairs move forward)
  auto pair_of = [&](const long long* pre, long long e, int start) {
    int q = start;
    while (q + 1 < count && pre[q + 1] <= e) ++q;
    return q;
  };
  auto first_pair = [&](const long long* pre, long long e) {
    int lo = 0, hi = count - 1;  // last q with pre[q] <= e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  // 1. listed blocks.  The warp reads the entries of 32 / (32 / BPI)
  //    iterations with one load (entry base + lane), and loads the next
  //    iteration's blocks while it sums the current ones.
  {
    const long long nf = fpre[count];
    const long long units = (nf + BPI - 1) / BPI;  // warp iterations
    const long long per = (units + nwarps - 1) / nwarps;
    const long long u0 = gwarp * per, u1 = min(units, u0 + per);
    constexpr int kIters = 32 / BPI;  // iterations whose entries one warp-wide load covers
    int q = u0 < u1 ? first_pair(fpre, u0 * BPI) : 0;
    // lane l: entry e0 + l of the current window, its pair and record word
    long long wbase = -1;
    long long wE = 0;
    int wq = 0;
    auto window = [&](long long it) {  // warp-uniform: the entries of iterations it .. it + kIters - 1
      const long long e0 = it * BPI;
      const long long e = e0 + lane;
      int ql = q;
      unsigned long long E = 0;
      if (e < nf) {
        ql = pair_of(fpre, e, q);
        E = (unsigned long long)fix[bpre[ql] + (e - fpre[ql])];
      }
      wbase = it;
      wE = (long long)E;
      wq = ql;
      q = __shfl_sync(0xffffffffu, ql, 31);
    };
    struct Fetched {
      bool have;
      int pq;
      unsigned long long E;
      Chunk ch;
    };
    auto fetch = [&](long long it, Fetched& fd) {  // warp-uniform
      if (it - wbase >= kIters || wbase < 0) window(it);
      const int src = (int)(it - wbase) * BPI + g;
      fd.E = (unsigned long long)__shfl_sync(0xffffffffu, wE, src);
      fd.pq = __shfl_sync(0xffffffffu, wq, src);
      fd.have = it * BPI + g < nf;
      fd.ch.vmask = 0xFFu;
      if (fd.have) {  // the block lies in a plain item, inside the pair's vectors
        const long long lb = (long long)(fd.E & ((1ull << 38) - 1));
        const long long item = lb / BPI;
        const int gi = (int)(lb % BPI);
        const double* x = xs[fd.pq];
        const double* y = ys[fd.pq];
        const long long base = item * kItem + item_offset<LOG2B>(gi * L + sub, 0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double2 av = __ldcs(reinterpret_cast<const double2*>(x + base + 2 * L * j));
          const double2 bv = __ldcs(reinterpret_cast<const double2*>(y + base + 2 * L * j));
          fd.ch.x[2 * j] = (uint64_t)__double_as_longlong(av.x);
          fd.ch.x[2 * j + 1] = (uint64_t)__double_as_longlong(av.y);
          fd.ch.y[2 * j] = (uint64_t)__double_as_longlong(bv.x);
          fd.ch.y[2 * j + 1] = (uint64_t)__double_as_longlong(bv.y);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) fd.ch.x[j] = fd.ch.y[j] = 0ull;
      }
    };
    Fetched cur, nxt;
    if (u0 < u1) fetch(u0, cur);
    for (long long it = u0; it < u1; ++it) {  // warp-uniform
      if (it + 1 < u1) fetch(it + 1, nxt);
      const int u = (int)((cur.E >> 38) & 0xFFFu), elo = (int)((cur.E >> 50) & 0xFFFu);
      int key[8];
      int cmax = kNone, kmin = INT_MAX;
      chunk_keys(cur.ch, key, cmax, kmin);
      const int ub = group_max<L>(cmax);  // every lane joins its block's shuffles
      int c_old = kPerf, c_new = kPerf;
      long long d = 0;
      if (cur.have) {
        const PairPart& r = pp[cur.pq];
        c_old = precision_of((long long)LOG2B + ub - (elo + ps[cur.pq].f_spec - 1), mh, ms);
        c_new = precision_of((long long)LOG2B + ub - (r.e_max + 2046 + r.f - 1), mh, ms);
        const unsigned p_old = c_old == kPerf ? 0u : 1u << c_old, p_new = c_new == kPerf ? 0u : 1u << c_new;
        double h = 0.0, sg = 0.0, a0 = 0.0, a1 = 0.0;
        acc_lane<LOG2B, 3, 0u>(cur.ch, key, u, p_old, h, sg, a0);
        acc_lane<LOG2B, 3, 0u>(cur.ch, key, u, p_new, h, sg, a1);
        d = (p_new ? __double2ll_rz(a1 * 4503599627370496.0) : 0ll) -
            (p_old ? __double2ll_rz(a0 * 4503599627370496.0) : 0ll);  // grid 2^(u - 52)
      }
      d = group_sum<L>(d);
      if (cur.have && sub == 0) {
        const int pq = cur.pq;
        atomic_add_i128(&pp[pq].lo, &pp[pq].hi, candidate_to_fixed(d, kSingle, u - 2046, 8, pp[pq].lsb));
        atomicAdd(&pp[pq].cnt[c_old], (unsigned long long)(-(long long)B));
        atomicAdd(&pp[pq].cnt[c_new], (unsigned long long)B);
      }
      cur = nxt;
    }
  }
  // 2. listed items
  {
    const long long nr = rpre[count];
    const long long per = (nr + nwarps - 1) / nwarps;
    const long long e0 = gwarp * per, e1 = min(nr, e0 + per);
    int q = e0 < e1 ? first_pair(rpre, e0) : 0;
    for (long long e = e0; e < e1; ++e) {  // warp-uniform
      q = pair_of(rpre, e, q);
      const long long item = redo[gpre[q] + (e - rpre[q])];
      const PairPart& r = pp[q];
      const ClassByAnchor lut{r.e_max, r.f, mh, ms};
      unsigned long long c[5] = {0, 0, 0, 0, 0};
      int u;
      const long long v = recompute_item_fast<LOG2B, ClassByAnchor>(xs[q], ys[q], ns[q], item, lut, lane, &u, c,
                                                                     nullptr);
      for (int k = 0; k < 4; ++k) c[k] = warp_sum_u64(c[k]);
      if (lane == 0) {
        if (u != kNone) atomic_add_i128(&pp[q].lo, &pp[q].hi, candidate_to_fixed(v, kSingle, u, 8, r.lsb));
        for (int k = 0; k < 4; ++k)
          if (c[k]) atomicAdd(&pp[q].cnt[k], c[k]);
      }
    }
  }
}

// One thread per pair: the pair's sum rounded once, and its result.
__global__ void k_bfinish(const PairStats* __restrict__ ps, const PairPart* __restrict__ pp, int count,
                          qdot_result* __restrict__ outs) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const PairPart r = pp[p];
  const PairStats st = ps[p];
  qdot_result o;
  o.status = r.status;
  o.n_bins = (long long)st.nbins;
  o.e_max = r.e_max;
  o.e_min = st.nbins > 0 ? st.e_min : 0;
  o.f = r.f;
  for (int k = 0; k < 4; ++k) o.count[k] = (int64_t)r.cnt[k];
  o.count[4] = (int64_t)st.zeros;
  if (r.status != QDOT_OK) {
    o.value = __longlong_as_double(0x7FF8000000000000ll);
    o.bound = o.value;
  } else {
    o.value = fixed_to_double((i128)(((u128)r.hi << 64) | r.lo), r.lsb);
    o.bound = st.nbins > 0 ? fixed_to_double((i128)st.nbins, r.e_max + r.f) : 0.0;
  }
  outs[p] = o;
}

constexpr int kBatchRepairQueue = 256;

__device__ long long recompute_any(const double* x, const double* y, long long n, long long blk, int u, int cls,
                                   int log2b) {
  switch (log2b) {
    case 5: return recompute_candidate<5>(x, y, n, blk, u, cls);
    case 6: return recompute_candidate<6>(x, y, n, blk, u, cls);
    case 7: return recompute_candidate<7>(x, y, n, blk, u, cls);
    default: return recompute_candidate<8>(x, y, n, blk, u, cls);
  }
}

__device__ long long recompute_any_warp(const double* x, const double* y, long long n, long long blk, int u, int cls,
                                        int log2b, int lane) {
  switch (log2b) {
    case 5: return recompute_candidate_warp<5>(x, y, n, blk, u, cls, lane);
    case 6: return recompute_candidate_warp<6>(x, y, n, blk, u, cls, lane);
    case 7: return recompute_candidate_warp<7>(x, y, n, blk, u, cls, lane);
    default: return recompute_candidate_warp<8>(x, y, n, blk, u, cls, lane);
  }
}

__global__ void __launch_bounds__(256) k_bfinal(const double* const* __restrict__ xs,
                                                const double* const* __restrict__ ys,
                                                const long long* __restrict__ ns, const long long* __restrict__ bpre,
                                                const PairStats* __restrict__ ps, const BatchHeader* __restrict__ hdr,
                                                const BlockRec* __restrict__ recs, int log2b, qdot_params prm,
                                                qdot_result* __restrict__ outs) {
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][4];
  const int p = blockIdx.x;
  const PairStats st = ps[p];
  int status = hdr->status != QDOT_OK ? hdr->status : st.status;
  const long long nb = (long long)st.nbins;
  const int e_max = nb > 0 ? st.e_max : 0;
  const int f = (status == QDOT_OK && nb > 0)
                    ? floor_log2_ratio(prm.eps, prm.split_budget ? (unsigned long long)nb : 1ull)
                    : 0;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  const int L = fixed_point_bits(ns[p] > 0 ? ns[p] : 1);
  const int lsb = e_max - L;
  i128 acc = 0;
  unsigned long long c[4] = {0, 0, 0, 0};
  __shared__ long long s_qblk[kBatchRepairQueue];
  __shared__ int s_qinfo[kBatchRepairQueue];
  __shared__ int s_nq;
  if (threadIdx.x == 0) s_nq = 0;
  __syncthreads();
  const double* xp = xs[p];
  const double* yp = ys[p];
  const long long np_ = ns[p];
  if (status == QDOT_OK) {
    for (long long r = bpre[p] + threadIdx.x; r < bpre[p + 1]; r += blockDim.x) {
      const longlong2 r0 = reinterpret_cast<const longlong2*>(recs + r)[0];
      const longlong2 r1 = reinterpret_cast<const longlong2*>(recs + r)[1];
      const int key = (int)(short)(r1.y & 0xFFFF);
      if (key == kEmptyKey) continue;
      const int u = (int)(short)((r1.y >> 16) & 0xFFFF);
      const unsigned mw = (unsigned)((unsigned long long)r1.y >> 32);
      const unsigned m = rec_count(mw);
      const int cls = precision_of((long long)key - e_max - f + 1, mh, ms);
#pragma unroll
      for (int k = 0; k < 4; ++k) c[k] += (cls == k) ? m : 0u;
      if (cls == kPerf) continue;
      if (rec_cands(mw) & (1u << cls)) {
        acc += record_candidate(r0.x, r0.y, r1.x, u, cls, log2b, lsb);
        continue;
      }
      const int slot = atomicAdd(&s_nq, 1);  // recomputed by the CTA's warps below
      if (slot < kBatchRepairQueue) {
        s_qblk[slot] = r - bpre[p];
        s_qinfo[slot] = (u << 2) | cls;
      } else {
        const long long v = recompute_any(xp, yp, np_, r - bpre[p], u, cls, log2b);
        acc += record_candidate(v, v, v, u, cls, log2b, lsb);
      }
    }
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nq = min(s_nq, kBatchRepairQueue);
    for (int qi = w; qi < nq; qi += (int)(blockDim.x >> 5)) {
      const int cls = s_qinfo[qi] & 3, u = s_qinfo[qi] >> 2;
      const long long v = recompute_any_warp(xp, yp, np_, s_qblk[qi], u, cls, log2b, lane);
      if (lane == 0) acc += record_candidate(v, v, v, u, cls, log2b, lsb);
    }
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
    r.status = status;
    r.n_bins = nb;
    r.e_max = e_max;
    r.e_min = nb > 0 ? st.e_min : 0;
    r.f = f;
    for (int k = 0; k < 4; ++k) r.count[k] = (int64_t)c[k];
    r.count[4] = (int64_t)st.zeros;
    if (status != QDOT_OK) {
      r.value = __longlong_as_double(0x7FF8000000000000ll);
      r.bound = r.value;
    } else {
      r.value = fixed_to_double(acc, lsb);
      r.bound = nb > 0 ? fixed_to_double((i128)nb, e_max + f) : 0.0;
    }
    outs[p] = r;
  }
}

struct BatchLayout {
  size_t off_hdr, off_gpre, off_bpre, off_ps, off_rec, fixed;
};

BatchLayout batch_layout(int count) {
  BatchLayout l;
  size_t off = 0;
  l.off_hdr = off;
  off = align_up(off + sizeof(BatchHeader), 256);
  l.off_gpre = off;
  off = align_up(off + sizeof(long long) * (size_t)(count + 1), 256);
  l.off_bpre = off;
  off = align_up(off + sizeof(long long) * (size_t)(count + 1), 256);
  l.off_ps = off;
  off = align_up(off + sizeof(PairStats) * (size_t)(count > 0 ? count : 1), 256);
  l.off_rec = off;
  l.fixed = off;
  return l;
}

// Workspace of the item-record path (blocks of 32): batch_layout's part, then
// per pair its PairPart and the two list prefixes, then the lists and records
// for up to cap_b blocks (8 B each in the block list) and cap_b / 8 + count + 1
// items (8 B each in the item sums, meta words, block offsets and item list).
struct ItemsLayout {
  size_t off_pp, off_fpre, off_rpre, head;
  size_t off_fix, off_isum, off_imeta, off_iblk, off_redo, total;
  long long cap_b, cap_i;
};

ItemsLayout items_layout(int count, long long cap_b) {
  ItemsLayout l;
  size_t off = batch_layout(count).fixed;
  l.off_pp = off;
  off = align_up(off + sizeof(PairPart) * (size_t)(count > 0 ? count : 1), 256);
  l.off_fpre = off;
  off = align_up(off + sizeof(long long) * (size_t)(count + 1), 256);
  l.off_rpre = off;
  off = align_up(off + sizeof(long long) * (size_t)(count + 1), 256);
  l.head = off;
  l.cap_b = cap_b;
  l.cap_i = cap_b / 8 + count + 1;
  l.off_fix = off;
  off = align_up(off + sizeof(long long) * (size_t)l.cap_b, 256);
  l.off_isum = off;
  off = align_up(off + sizeof(long long) * (size_t)l.cap_i, 256);
  l.off_imeta = off;
  off = align_up(off + sizeof(long long) * (size_t)l.cap_i, 256);
  l.off_iblk = off;
  off = align_up(off + sizeof(long long) * (size_t)l.cap_i, 256);
  l.off_redo = off;
  off = align_up(off + sizeof(long long) * (size_t)l.cap_i, 256);
  l.total = off;
  return l;
}

size_t items_region_bytes(int count, long long blocks) {
  const ItemsLayout l = items_layout(count, blocks);
  return l.total - l.head;
}

// The largest block capacity whose layout fits ws_bytes.
ItemsLayout items_layout_for(int count, size_t ws_bytes) {
  const ItemsLayout h = items_layout(count, 0);
  if (ws_bytes <= h.total) return h;
  long long cap = (long long)((ws_bytes - h.head) / 12);  // 8 B + 4 x 8 B / 8 per block
  ItemsLayout l = items_layout(count, cap);
  while (cap > 0 && l.total > ws_bytes) l = items_layout(count, --cap);
  return l;
}

template <int LOG2B, int THREADS, bool STAGED>
cudaError_t launch_stream(int grid, const double* const* xs, const double* const* ys, const long long* ns, int count,
                          const long long* gpre, const long long* bpre, PairStats* ps, const BatchHeader* hdr,
                          BlockRec* recs, int mh, int ms, cudaStream_t st) {
  const int smem = STAGED ? (THREADS / 32) * 2 * kStageWords * 16 : 0;
  static bool attr_set = false;  // per instantiation
  if (STAGED && !attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_bstream<LOG2B, THREADS, STAGED>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_bstream<LOG2B, THREADS, STAGED><<<grid, THREADS, smem, st>>>(xs, ys, ns, count, gpre, bpre, ps, hdr, recs, mh,
                                                                  ms);
  return cudaGetLastError();
}

template <int THREADS>
cudaError_t launch_stream_items(int grid, const double* const* xs, const double* const* ys, const long long* ns,
                                int count, const long long* gpre, PairStats* ps, const BatchHeader* hdr,
                                long long* isum, unsigned long long* imeta, unsigned long long* iblk, int mh, int ms,
                                cudaStream_t st) {
  const int smem = (THREADS / 32) * 2 * kStageWords * 16;
  static bool attr_set = false;  // per instantiation
  if (!attr_set) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_bstream_items<5, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  k_bstream_items<5, THREADS><<<grid, THREADS, smem, st>>>(xs, ys, ns, count, gpre, ps, hdr, isum, imeta, iblk, mh,
                                                            ms);
  return cudaGetLastError();
}

// Blocks of 32: item records per pair (k_bstream_items, k_bfinal_items,
// k_bscan, k_bredo, k_bfinish).
cudaError_t launch_batched_items(const double* const* xs, const double* const* ys, const long long* ns, int count,
                                 const qdot_params* p, qdot_result* outs, const qdot_batched_tuning& t, char* ws,
                                 size_t ws_bytes, cudaStream_t st) {
  const BatchLayout b = batch_layout(count);
  const ItemsLayout l = items_layout_for(count, ws_bytes);
  auto* hdr = reinterpret_cast<BatchHeader*>(ws + b.off_hdr);
  auto* gpre = reinterpret_cast<long long*>(ws + b.off_gpre);
  auto* bpre = reinterpret_cast<long long*>(ws + b.off_bpre);
  auto* ps = reinterpret_cast<PairStats*>(ws + b.off_ps);
  auto* pp = reinterpret_cast<PairPart*>(ws + l.off_pp);
  auto* fpre = reinterpret_cast<long long*>(ws + l.off_fpre);
  auto* rpre = reinterpret_cast<long long*>(ws + l.off_rpre);
  auto* fix = reinterpret_cast<long long*>(ws + l.off_fix);
  auto* isum = reinterpret_cast<long long*>(ws + l.off_isum);
  auto* imeta = reinterpret_cast<unsigned long long*>(ws + l.off_imeta);
  auto* iblk = reinterpret_cast<unsigned long long*>(ws + l.off_iblk);
  auto* redo = reinterpret_cast<long long*>(ws + l.off_redo);
  // every pair has at most ceil(n / 256) <= blocks / 8 + 1 items, so cap_i >= items
  k_bplan<<<1, 1024, 0, st>>>(xs, ys, ns, count, 5, p->eps, p->split_budget, l.cap_b, gpre, bpre, ps, hdr);
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int grid = t.grid_ctas > 0 ? t.grid_ctas : t.ctas_per_sm * sms;
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  const int mh = p->mant_reading ? 11 : 10, ms = p->mant_reading ? 24 : 23;
  cudaError_t e = t.threads_per_cta == 128
                      ? launch_stream_items<128>(grid, xs, ys, ns, count, gpre, ps, hdr, isum, imeta, iblk, mh, ms, st)
                      : launch_stream_items<256>(grid, xs, ys, ns, count, gpre, ps, hdr, isum, imeta, iblk, mh, ms, st);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, st);
  k_bfinal_items<5><<<count, 256, 0, st>>>(ns, gpre, bpre, ps, hdr, isum, imeta, iblk, fix, redo, pp, *p);
  k_bscan<<<1, 1024, 0, st>>>(pp, count, fpre, rpre);
  k_bredo<5><<<2 * sms, 256, 0, st>>>(xs, ys, ns, count, gpre, bpre, ps, fix, redo, fpre, rpre, pp, mh, ms);
  k_bfinish<<<(count + 255) / 256, 256, 0, st>>>(ps, pp, count, outs);
  return cudaGetLastError();
}

template <int LOG2B>
cudaError_t launch_batched_lb(const double* const* xs, const double* const* ys, const long long* ns, int count,
                              const qdot_params* p, qdot_result* outs, const qdot_batched_tuning& t, char* ws,
                              size_t ws_bytes, cudaStream_t st) {
  if (LOG2B == 5) return launch_batched_items(xs, ys, ns, count, p, outs, t, ws, ws_bytes, st);
  const BatchLayout l = batch_layout(count);
  auto* hdr = reinterpret_cast<BatchHeader*>(ws + l.off_hdr);
  auto* gpre = reinterpret_cast<long long*>(ws + l.off_gpre);
  auto* bpre = reinterpret_cast<long long*>(ws + l.off_bpre);
  auto* ps = reinterpret_cast<PairStats*>(ws + l.off_ps);
  auto* recs = reinterpret_cast<BlockRec*>(ws + l.off_rec);
  const long long capacity = (long long)((ws_bytes - l.fixed) / sizeof(BlockRec));
  k_bplan<<<1, 1024, 0, st>>>(xs, ys, ns, count, LOG2B, p->eps, p->split_budget, capacity, gpre, bpre, ps, hdr);
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int grid = t.grid_ctas > 0 ? t.grid_ctas : t.ctas_per_sm * sms;
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  cudaError_t e;
  const int mh = p->mant_reading ? 11 : 10, ms = p->mant_reading ? 24 : 23;
  if (t.threads_per_cta == 128)
    e = t.staged ? launch_stream<LOG2B, 128, true>(grid, xs, ys, ns, count, gpre, bpre, ps, hdr, recs, mh, ms, st)
                 : launch_stream<LOG2B, 128, false>(grid, xs, ys, ns, count, gpre, bpre, ps, hdr, recs, mh, ms, st);
  else
    e = t.staged ? launch_stream<LOG2B, 256, true>(grid, xs, ys, ns, count, gpre, bpre, ps, hdr, recs, mh, ms, st)
                 : launch_stream<LOG2B, 256, false>(grid, xs, ys, ns, count, gpre, bpre, ps, hdr, recs, mh, ms, st);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, st);
  k_bfinal<<<count, 256, 0, st>>>(xs, ys, ns, bpre, ps, hdr, recs, LOG2B, *p, outs);
  return cudaGetLastError();
}

}  // namespace

size_t batched_ws_bytes(const int64_t* ns_host, int count, const qdot_params* p) {
  long long blocks = 0;
  for (int i = 0; i < count; ++i) blocks += (ns_host[i] + p->block - 1) / p->block;
  if (p->block == 32) return items_layout(count, 0).head + items_region_bytes(count, blocks);
  return batch_layout(count).fixed + align_up(sizeof(chunk::BlockRec) * (size_t)blocks, 256);
}

qdot_batched_tuning default_batched_tuning() { return qdot_batched_tuning{256, 3, 0, 1}; }

cudaError_t launch_qdot_batched(const double* const* xs, const double* const* ys, const long long* ns, int count,
                                const qdot_params* p, qdot_result* outs, int grid_ctas, void* ws, size_t ws_bytes,
                                cudaStream_t st, const qdot_batched_tuning* tuning) {
  qdot_batched_tuning t = tuning ? *tuning : default_batched_tuning();
  if (grid_ctas > 0) t.grid_ctas = grid_ctas;
  int lb = 0;
  while ((1 << lb) < p->block) ++lb;
  char* w = static_cast<char*>(ws);
  switch (lb) {
    case 5: return launch_batched_lb<5>(xs, ys, ns, count, p, outs, t, w, ws_bytes, st);
    case 6: return launch_batched_lb<6>(xs, ys, ns, count, p, outs, t, w, ws_bytes, st);
    case 7: return launch_batched_lb<7>(xs, ys, ns, count, p, outs, t, w, ws_bytes, st);
    default: return launch_batched_lb<8>(xs, ys, ns, count, p, outs, t, w, ws_bytes, st);
  }
}

}  // namespace qd

using namespace qd;

extern "C" {

size_t qdot_batched_workspace_size(const int64_t* ns_host, int32_t count, const qdot_params* p) {
  std::string why;
  if (count < 0 || !p || !valid_params(0, p, &why) || p->block < 32 || p->block > 256) return 0;
  if (count > 0 && !ns_host) return 0;
  for (int i = 0; i < count; ++i)
    if (ns_host[i] < 0) return 0;
  return batched_ws_bytes(ns_host, count, p);
}

qdot_status qdot_batched_tuned(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                               const qdot_params* p, qdot_result* outs, const qdot_batched_tuning* tuning,
                               int32_t grid_ctas, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  std::string why;
  if (!p || !valid_params(0, p, &why)) {
    set_error("qdot_batched: " + (p ? why : std::string("params pointer is NULL")));
    return QDOT_ERR_ARG;
  }
  if (p->block < 32 || p->block > 256) {
    set_error("qdot_batched: block must be a power of two in [32, 256]");
    return QDOT_ERR_ARG;
  }
  if (count < 0 || (count > 0 && (!xs || !ys || !ns || !outs))) {
    set_error("qdot_batched: count must be >= 0 and xs, ys, ns, outs non-NULL device arrays");
    return QDOT_ERR_ARG;
  }
  if (grid_ctas < 0) {
    set_error("qdot_batched: grid_ctas must be >= 0 (0 = default)");
    return QDOT_ERR_ARG;
  }
  if (count == 0) return QDOT_OK;
  const BatchLayout l = batch_layout(count);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < l.fixed) {
    set_error("qdot_batched: workspace missing, misaligned or smaller than qdot_batched_workspace_size()");
    return QDOT_ERR_WORKSPACE;
  }
  if (tuning && !((tuning->threads_per_cta == 128 || tuning->threads_per_cta == 256) &&
                  (tuning->staged == 0 || tuning->staged == 1) && tuning->grid_ctas >= 0 &&
                  (tuning->grid_ctas > 0 || (tuning->ctas_per_sm >= 1 && tuning->ctas_per_sm <= 64)))) {
    set_error("qdot_batched: tuning needs threads_per_cta 128 or 256, staged 0 or 1, and grid_ctas > 0 or "
              "ctas_per_sm in [1, 64]");
    return QDOT_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long* nsl = reinterpret_cast<const long long*>(ns);
  const cudaError_t e = launch_qdot_batched(xs, ys, nsl, count, p, outs, grid_ctas, ws, ws_bytes, st, tuning);
  if (e != cudaSuccess) {
    set_error(std::string("qdot_batched launch: ") + cudaGetErrorString(e));
    return QDOT_ERR_CUDA;
  }
  return QDOT_OK;
}

qdot_status qdot_batched(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                         const qdot_params* p, qdot_result* outs, int32_t grid_ctas, void* ws, size_t ws_bytes,
                         void* stream) {
  return qdot_batched_tuned(xs, ys, ns, count, p, outs, nullptr, grid_ctas, ws, ws_bytes, stream);
}

}  // extern "C"
