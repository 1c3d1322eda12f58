// qdot in one launch for vectors that the resident grid covers in a few
// warp items (the sizes of the solvers' dot products: 2^21 .. 2^23).
//
// At these sizes the multi-kernel paths spend most of their time in launch
// gaps and one-CTA kernels.  Here one cooperative launch does everything:
//   phase 1  every warp streams its items (at most kFusedItems) and keeps, per
//            block, the DOUBLE candidate, the block key and M_b in shared
//            memory (blocked binning, 32 <= B <= 256); per-CTA statistics go
//            to the workspace;
//   sync     grid-wide barrier;
//   phase 2  every CTA reduces the statistics (e_max, N_bins, f exactly), then
//            classes its own blocks (eq. bin-score-def, eq. precision-def):
//            a DOUBLE block adds its kept candidate, a HALF or SINGLE block is
//            summed again from x and y (held in L2 at these sizes) on the
//            chain of its class, a perforated block adds nothing; all of it
//            exactly, in fixed point.  When e_max - e_min <= -f - m_single
//            every block is DOUBLE (Theorem 5), so no class is looked up and
//            nothing is read again;
//   phase 3  the last CTA to finish phase 2 (an arrival counter) adds the
//            per-CTA sums in order and rounds once.
// Every candidate is the one-pass path's (qdot_chunk.cuh: one chain per lane
// of the streaming layout), so both paths return the same bits.
#include <climits>
#include <cooperative_groups.h>

#include "qdot_chunk.cuh"
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

using namespace chunk;
namespace cgrp = cooperative_groups;

constexpr int kFusedThreads = 512;
constexpr int kFusedWarps = kFusedThreads / 32;
constexpr int kFusedItems = 8;    // items per warp at most
constexpr int kFusedCtasPerSm = 1;

struct FusedBlock {  // one block's DOUBLE candidate (in shared memory)
  long long d;
  int key;           // s_b, kEmptyKey when the block has no nonzero component
  unsigned m;        // M_b
};

struct CtaStats {
  int e_max, e_min, bad, pad;
  long long nbins, zeros;
};

struct FusedPart {
  i128 sum;
  unsigned long long cnt[4];
};

// The last phase of both fused kernels: the CTA's part is already in
// parts[blockIdx.x]; the last CTA to arrive (an arrival counter) adds every
// part in CTA order, rounds the fixed-point sum once and writes the result.
// s_sum and s_cnt are the kernel's shared scratch of kFusedWarps entries.
__device__ void fused_finish(const FusedPart* __restrict__ parts, unsigned* __restrict__ arrivals, i128* s_sum,
                             unsigned long long (*s_cnt)[4], int e_max, int e_min, int f, int bad, long long nbins,
                             long long zeros, int lsb, qdot_result* __restrict__ out) {
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's part is visible before its arrival counts
    s_last = atomicAdd(arrivals, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  i128 tot = 0;
  unsigned long long c4[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < (int)gridDim.x; i += kFusedThreads) {
    tot += parts[i].sum;
    for (int c = 0; c < 4; ++c) c4[c] += parts[i].cnt[c];
  }
  tot = warp_sum_i128(tot);
  for (int c = 0; c < 4; ++c) c4[c] = warp_sum_u64(c4[c]);
  __syncthreads();  // s_sum / s_cnt are reused
  if (lane == 0) {
    s_sum[w] = tot;
    for (int c = 0; c < 4; ++c) s_cnt[w][c] = c4[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kFusedWarps; ++i) {
      tot += s_sum[i];
      for (int c = 0; c < 4; ++c) c4[c] += s_cnt[i][c];
    }
    // (tot and c4 in thread 0 already hold warp 0's totals)
    qdot_result r;
    r.status = bad ? QDOT_ERR_NONFINITE : QDOT_OK;
    r.n_bins = nbins;
    r.e_max = e_max;
    r.e_min = e_min;
    r.f = f;
    for (int c = 0; c < 4; ++c) r.count[c] = (int64_t)c4[c];
    r.count[4] = zeros;
    if (r.status != QDOT_OK) {
      r.value = __longlong_as_double(0x7FF8000000000000ll);
      r.bound = r.value;
    } else {
      r.value = fixed_to_double(tot, lsb);
      r.bound = r.n_bins > 0 ? fixed_to_double((i128)r.n_bins, e_max + f) : 0.0;
    }
    *out = r;
  }
}

template <int LOG2B>
__global__ void __launch_bounds__(kFusedThreads, kFusedCtasPerSm)
    k_qdot_fused(const double* __restrict__ x, const double* __restrict__ y, long long n, qdot_params prm,
                 CtaStats* __restrict__ cstats, FusedPart* __restrict__ parts, unsigned* __restrict__ arrivals,
                 qdot_selection* __restrict__ sel, qdot_result* __restrict__ out,
                 qdot_trace_unit* __restrict__ trace) {
  constexpr int L = Map<LOG2B>::L, BPI = Map<LOG2B>::BPI;
  __shared__ FusedBlock s_blk[kFusedWarps][kFusedItems][BPI];
  __shared__ CtaStats s_w[kFusedWarps];
  __shared__ i128 s_sum[kFusedWarps];
  __shared__ unsigned long long s_cnt[kFusedWarps][4];
  __shared__ int s_emax, s_emin, s_bad, s_f;
  __shared__ long long s_nbins, s_zeros;
  cgrp::grid_group grid = cgrp::this_grid();

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane / L, sub = lane % L;
  const long long nblocks = (n + (1ll << LOG2B) - 1) >> LOG2B;
  const long long nitems = (n + kItem - 1) / kItem;
  const long long gwarp = (long long)blockIdx.x * kFusedWarps + w;
  const long long nwarps = (long long)gridDim.x * kFusedWarps;

  // ---- phase 1: stream ----
  if (blockIdx.x == 0 && threadIdx.x == 0) *arrivals = 0;  // ordered before phase 2 by the grid barrier
  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;
  int k = 0;
  Chunk cur, nxt;
  if (gwarp < nitems) load_item<LOG2B>(x, y, n, gwarp, lane, cur);
  for (long long it = gwarp; it < nitems && k < kFusedItems; it += nwarps, ++k) {
    if (it + nwarps < nitems) load_item<LOG2B>(x, y, n, it + nwarps, lane, nxt);
    double aH = 0.0, aS = 0.0, aD = 0.0;
    int M = 0, zeros = 0, u;
    int key[8];
    int cmax = kNone;
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      u = group_max<L>(cmax);
      M = 8;
      acc_lane<LOG2B, 0, 0u>(cur, key, u, kCandD, aH, aS, aD);  // the DOUBLE chain
    } else {
      u = chunk_general_chains<LOG2B, kCandD>(cur, aH, aS, aD, M, zeros, kmin, bad);
    }
    int kb, ub, mb;
    long long dv = 0;
    {
      dv = group_sum<L>(__double2ll_rz(aD * chain_scale<LOG2B>(kDouble)));
      mb = group_sum_i<L>(M);
      ub = u - 2046;
      kb = mb > 0 ? ceil_log2_u32((uint32_t)mb) + ub : (int)kEmptyKey;
    }
    const long long blk = it * BPI + g;
    zeros_l += zeros;
    const bool real = blk < nblocks && mb > 0;
    if (real) {
      nbins += (sub == 0);
      emax_l = max(emax_l, ub);
    }
    if (sub == 0) s_blk[w][k][g] = FusedBlock{dv, real ? kb : (int)kEmptyKey, (unsigned)mb};
    cur = nxt;
  }
  emax_l = __reduce_max_sync(0xffffffffu, emax_l);
  kmin = __reduce_min_sync(0xffffffffu, kmin);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  nbins = (long long)warp_sum_u64((unsigned long long)nbins);
  zeros_l = (long long)warp_sum_u64((unsigned long long)zeros_l);
  if (lane == 0) s_w[w] = CtaStats{emax_l, kmin == INT_MAX ? INT_MAX : kmin - 2046, bad, 0, nbins, zeros_l};
  __syncthreads();
  if (threadIdx.x == 0) {
    CtaStats c = s_w[0];
    for (int i = 1; i < kFusedWarps; ++i) {
      c.e_max = max(c.e_max, s_w[i].e_max);
      c.e_min = min(c.e_min, s_w[i].e_min);
      c.bad |= s_w[i].bad;
      c.nbins += s_w[i].nbins;
      c.zeros += s_w[i].zeros;
    }
    cstats[blockIdx.x] = c;
  }
  grid.sync();

  // ---- phase 2: global statistics, classes, exact sums ----
  {
    int em = kNone, en = INT_MAX, bd = 0;
    long long nb = 0, z = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kFusedThreads) {
      const CtaStats c = cstats[i];
      em = max(em, c.e_max);
      en = min(en, c.e_min);
      bd |= c.bad;
      nb += c.nbins;
      z += c.zeros;
    }
    em = __reduce_max_sync(0xffffffffu, em);
    en = __reduce_min_sync(0xffffffffu, en);
    bd = (int)__reduce_or_sync(0xffffffffu, (unsigned)bd);
    nb = (long long)warp_sum_u64((unsigned long long)nb);
    z = (long long)warp_sum_u64((unsigned long long)z);
    if (lane == 0) s_w[w] = CtaStats{em, en, bd, 0, nb, z};
    __syncthreads();
    if (threadIdx.x == 0) {
      CtaStats c = s_w[0];
      for (int i = 1; i < kFusedWarps; ++i) {
        c.e_max = max(c.e_max, s_w[i].e_max);
        c.e_min = min(c.e_min, s_w[i].e_min);
        c.bad |= s_w[i].bad;
        c.nbins += s_w[i].nbins;
        c.zeros += s_w[i].zeros;
      }
      if (c.nbins == 0) {
        c.e_max = 0;
        c.e_min = 0;
      }
      s_emax = c.e_max;
      s_emin = c.e_min;
      s_bad = c.bad;
      s_nbins = c.nbins;
      s_zeros = c.zeros;
      s_f = c.nbins > 0 ? floor_log2_ratio(prm.eps, prm.split_budget ? (unsigned long long)c.nbins : 1ull) : 0;
    }
    __syncthreads();
  }
  const int e_max = s_emax, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  const int lsb = e_max - fixed_point_bits(n);
  i128 acc = 0;
  unsigned long long cnt[4] = {0, 0, 0, 0};
  // Theorem 5: every score is at least m_single, so every block is DOUBLE
  const bool all_double = (long long)e_max - s_emin <= -(long long)f - ms;
  if (!s_bad) {
    // HALF and SINGLE blocks are summed again from x and y (in L2 at these
    // sizes): a warp loads the next item that has such a block while it sums
    // the current one, so the L2 round trips overlap
    auto block_class = [&](int kk) {
      const FusedBlock b = s_blk[w][kk][g];
      return b.key == (int)kEmptyKey ? kZero
                                     : (all_double ? kDouble : precision_of((long long)b.key - e_max - f + 1, mh, ms));
    };
    auto needs_chain = [&](int kk) {  // warp-uniform
      const int c = block_class(kk);
      return __any_sync(0xffffffffu, c == kHalf || c == kSingle);
    };
    bool need_cur = k > 0 && !all_double && needs_chain(0);
    if (need_cur) load_item<LOG2B>(x, y, n, gwarp, lane, cur);
    for (int kk = 0; kk < k; ++kk) {  // k is the same in every lane of the warp
      const bool need_nxt = kk + 1 < k && !all_double && needs_chain(kk + 1);
      if (need_nxt) load_item<LOG2B>(x, y, n, gwarp + (kk + 1) * nwarps, lane, nxt);
      const FusedBlock b = s_blk[w][kk][g];
      const long long blk = (gwarp + kk * nwarps) * BPI + g;
      const bool empty = b.key == (int)kEmptyKey;
      const int cls = block_class(kk);
      const int u = empty ? 0 : b.key - ceil_log2_u32(b.m);
      // every lane of a HALF or SINGLE block sums its chain (no shuffle
      // inside the branch), then the block's lanes add up
      long long lv = 0;
      if (need_cur && (cls == kHalf || cls == kSingle)) lv = chain_lane_loaded<LOG2B>(cur, u, cls);
      if (!all_double) lv = group_sum<L>(lv);
      if (sub == 0 && !empty) {
#pragma unroll
        for (int c = 0; c < 4; ++c) cnt[c] += (cls == c) ? b.m : 0u;
        const long long v = cls == kDouble ? b.d : lv;
        if (cls != kPerf) acc += candidate_to_fixed(v, cls, u, LOG2B, lsb);
        if (trace)  // check output only (qdot_trace)
          trace[blk] = qdot_trace_unit{cls != kPerf ? v : 0ll, cls != kPerf ? candidate_grid(cls, u, LOG2B) : 0,
                                       (uint8_t)cls, (uint8_t)(cls != kPerf ? QDOT_TRACE_FUSED : QDOT_TRACE_NONE), 0};
      }
      if (sub == 0 && empty && trace && blk < nblocks)
        trace[blk] = qdot_trace_unit{0ll, 0, (uint8_t)kZero, (uint8_t)QDOT_TRACE_NONE, 0};
      cur = nxt;
      need_cur = need_nxt;
    }
  }
  acc = warp_sum_i128(acc);
  for (int c = 0; c < 4; ++c) cnt[c] = warp_sum_u64(cnt[c]);
  if (lane == 0) {
    s_sum[w] = acc;
    for (int c = 0; c < 4; ++c) s_cnt[w][c] = cnt[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    FusedPart p;
    p.sum = 0;
    for (int c = 0; c < 4; ++c) p.cnt[c] = 0;
    for (int i = 0; i < kFusedWarps; ++i) {
      p.sum += s_sum[i];
      for (int c = 0; c < 4; ++c) p.cnt[c] += s_cnt[i][c];
    }
    parts[blockIdx.x] = p;
  }
  if (blockIdx.x == 0 && sel) {  // the parameter selection, for qdot_backward
    for (int kk = threadIdx.x; kk < kKeyCount; kk += kFusedThreads)
      sel->cls[kk] = (uint8_t)precision_of((long long)kKeyMin + kk - e_max - f + 1, mh, ms);
    if (threadIdx.x == 0) {
      sel->e_max = e_max;
      sel->e_min = s_emin;
      sel->f = f;
      sel->status = s_bad ? QDOT_ERR_NONFINITE : QDOT_OK;
      sel->n_bins = s_nbins;
      sel->block = prm.block;
      sel->key_min = kKeyMin;
      sel->m_half = mh;
      sel->m_single = ms;
      sel->reserved[0] = sel->reserved[1] = 0;
    }
  }
  // ---- phase 3: the last CTA to finish phase 2 adds the CTA sums in order ----
  fused_finish(parts, arrivals, s_sum, s_cnt, e_max, s_emin, f, s_bad, s_nbins, s_zeros, lsb, out);
}

// ---------------------------------------------------------------------------
// Exact binning (block 0, Algorithm 2) and blocks of one component (block 1)
// in one cooperative launch, for the sizes k_qdot_fused covers.  Bins are not
// contiguous index ranges here, so no candidate can be formed before the
// classes are known; instead the statistics come from one read of x and y
// (HBM) and the sums from a second read of the same items, which the whole
// working set (at most about 80 MB) leaves in L2:
//   phase 1  every warp reads its items (at most kFusedItems): e_max, e_min,
//            the nonzero count (block 1: N_bins), zeros, non-finite values;
//            with exact binning also the CTA's histogram of the keys
//            e_i = e(x_i) + e(y_i) (shared-memory counters), written out
//            whole to the workspace;
//   sync     grid-wide barrier;
//   phase 2  exact binning only: CTA b adds up its slice of keys over every
//            CTA's histogram (the bin counts M_k) and counts the non-empty
//            ones (N_bins); a second grid-wide barrier;
//   phase 3  every CTA: e_max and N_bins over the grid, f exactly, and the
//            class of every key into a shared table, score
//            ceil(log2 M_k) + e - e_max - f + 1 (M = 1 for blocks of one;
//            eq. bin-score-def, eq. precision-def); each warp reads its items
//            again, quantizes every component to its key's class and sums
//            the item on the grid 2^(u - 52) of its largest key u, the
//            arithmetic of the one-pass item path (recompute_item_fast), so
//            both paths return the same bits; the item sums go into 128-bit
//            fixed point;
//   phase 4  fused_finish.
// ---------------------------------------------------------------------------
template <bool EXACT>
__global__ void __launch_bounds__(kFusedThreads, kFusedCtasPerSm)
    k_qdot_fused_bins(const double* __restrict__ x, const double* __restrict__ y, long long n, qdot_params prm,
                      CtaStats* __restrict__ cstats, FusedPart* __restrict__ parts, unsigned* __restrict__ arrivals,
                      unsigned* __restrict__ hists, unsigned long long* __restrict__ gcount,
                      long long* __restrict__ slice_nb, qdot_selection* __restrict__ sel,
                      qdot_result* __restrict__ out, qdot_trace_unit* __restrict__ trace,
                      uint8_t* __restrict__ tcls) {
  __shared__ unsigned s_hist[EXACT ? kKeyCount : 1];
  __shared__ __align__(16) uint8_t s_lut[kKeyCount];
  __shared__ CtaStats s_w[kFusedWarps];
  __shared__ i128 s_sum[kFusedWarps];
  __shared__ unsigned long long s_cnt[kFusedWarps][4];
  __shared__ long long s_nb[kFusedWarps];
  __shared__ int s_emax, s_emin, s_bad, s_f;
  __shared__ long long s_nbins, s_zeros;
  cgrp::grid_group grid = cgrp::this_grid();

  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nitems = (n + kItem - 1) / kItem;
  const long long gwarp = (long long)blockIdx.x * kFusedWarps + w;
  const long long nwarps = (long long)gridDim.x * kFusedWarps;

  // ---- phase 1: statistics (and the CTA's key histogram) ----
  if (EXACT) {
    for (int i = threadIdx.x; i < kKeyCount; i += kFusedThreads) s_hist[i] = 0u;
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *arrivals = 0;  // ordered before phase 4 by the grid barrier
  long long nz_l = 0, zeros_l = 0;
  int emax_l = kNone, emin_l = INT_MAX, bad = 0;
  int k = 0;
  Chunk cur, nxt;
  if (gwarp < nitems) load_item<8, true>(x, y, n, gwarp, lane, cur);
  for (long long it = gwarp; it < nitems && k < kFusedItems; it += nwarps, ++k) {
    if (it + nwarps < nitems) load_item<8, true>(x, y, n, it + nwarps, lane, nxt);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint64_t a = cur.x[j], b = cur.y[j];
      const bool in = (cur.vmask >> j) & 1u;
      const bool fin = !(is_nonfinite(a) || is_nonfinite(b));
      bad |= in && !fin;
      const bool z = is_zero(a) || is_zero(b);
      zeros_l += in && fin && z;
      if (in && fin && !z) {
        const int e = exponent_of(a) + exponent_of(b);
        ++nz_l;
        emax_l = max(emax_l, e);
        emin_l = min(emin_l, e);
        if (EXACT) atomicAdd(&s_hist[e - kKeyMin], 1u);
      }
    }
    cur = nxt;
  }
  emax_l = __reduce_max_sync(0xffffffffu, emax_l);
  emin_l = __reduce_min_sync(0xffffffffu, emin_l);
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  nz_l = (long long)warp_sum_u64((unsigned long long)nz_l);
  zeros_l = (long long)warp_sum_u64((unsigned long long)zeros_l);
  if (lane == 0) s_w[w] = CtaStats{emax_l, emin_l, bad, 0, nz_l, zeros_l};
  __syncthreads();
  if (threadIdx.x == 0) {
    CtaStats c = s_w[0];
    for (int i = 1; i < kFusedWarps; ++i) {
      c.e_max = max(c.e_max, s_w[i].e_max);
      c.e_min = min(c.e_min, s_w[i].e_min);
      c.bad |= s_w[i].bad;
      c.nbins += s_w[i].nbins;
      c.zeros += s_w[i].zeros;
    }
    cstats[blockIdx.x] = c;
  }
  if (EXACT)
    for (int i = threadIdx.x; i < kKeyCount; i += kFusedThreads)
      hists[(size_t)blockIdx.x * kKeyCount + i] = s_hist[i];
  grid.sync();

  // ---- phase 2 (exact binning): bin counts M_k and N_bins, a slice of keys per CTA ----
  if (EXACT) {
    const int G = (int)gridDim.x;
    const int per = (kKeyCount + G - 1) / G;
    const int k0 = (int)blockIdx.x * per, k1 = min(k0 + per, kKeyCount);
    long long nb = 0;
    for (int kk = k0 + w; kk < k1; kk += kFusedWarps) {  // one warp per key
      unsigned long long m = 0;
      for (int c = lane; c < G; c += 32) m += hists[(size_t)c * kKeyCount + kk];
      m = warp_sum_u64(m);
      if (lane == 0) {
        gcount[kk] = m;
        nb += m != 0ull;
      }
    }
    if (lane == 0) s_nb[w] = nb;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < kFusedWarps; ++i) t += s_nb[i];
      slice_nb[blockIdx.x] = t;
    }
    grid.sync();
  }

  // ---- phase 3: selection, then the items again with the final classes ----
  {
    int em = kNone, en = INT_MAX, bd = 0;
    long long nb = 0, z = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += kFusedThreads) {
      const CtaStats c = cstats[i];
      em = max(em, c.e_max);
      en = min(en, c.e_min);
      bd |= c.bad;
      nb += EXACT ? slice_nb[i] : c.nbins;
      z += c.zeros;
    }
    em = __reduce_max_sync(0xffffffffu, em);
    en = __reduce_min_sync(0xffffffffu, en);
    bd = (int)__reduce_or_sync(0xffffffffu, (unsigned)bd);
    nb = (long long)warp_sum_u64((unsigned long long)nb);
    z = (long long)warp_sum_u64((unsigned long long)z);
    if (lane == 0) s_w[w] = CtaStats{em, en, bd, 0, nb, z};
    __syncthreads();
    if (threadIdx.x == 0) {
      CtaStats c = s_w[0];
      for (int i = 1; i < kFusedWarps; ++i) {
        c.e_max = max(c.e_max, s_w[i].e_max);
        c.e_min = min(c.e_min, s_w[i].e_min);
        c.bad |= s_w[i].bad;
        c.nbins += s_w[i].nbins;
        c.zeros += s_w[i].zeros;
      }
      if (c.nbins == 0) {
        c.e_max = 0;
        c.e_min = 0;
      }
      s_emax = c.e_max;
      s_emin = c.e_min;
      s_bad = c.bad;
      s_nbins = c.nbins;
      s_zeros = c.zeros;
      s_f = c.nbins > 0 ? floor_log2_ratio(prm.eps, prm.split_budget ? (unsigned long long)c.nbins : 1ull) : 0;
    }
    __syncthreads();
  }
  const int e_max = s_emax, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  for (int kk = threadIdx.x; kk < kKeyCount; kk += kFusedThreads) {
    long long sigma = (long long)kKeyMin + kk - e_max - f + 1;
    if (EXACT) {
      const unsigned long long m = gcount[kk];
      sigma = m ? sigma + (m <= 1ull ? 0 : 64 - __clzll((long long)(m - 1ull))) : -1;
    }
    s_lut[kk] = (uint8_t)precision_of(sigma, mh, ms);
  }
  __syncthreads();
  const int lsb = e_max - fixed_point_bits(n);
  i128 acc = 0;
  unsigned long long c5[5] = {0, 0, 0, 0, 0};
  if (!s_bad) {
    for (int kk = 0; kk < k; ++kk) {  // k is the same in every lane of the warp
      const long long it = gwarp + kk * nwarps;
      int u;
      const long long v = recompute_item_fast<0>(x, y, n, it, s_lut, lane, &u, c5, tcls);
      if (lane == 0 && u != kNone) acc += candidate_to_fixed(v, kSingle, u, 8, lsb);  // grid 2^(u - 52)
      if (lane == 0 && trace)  // check output only (qdot_trace)
        trace[it] = qdot_trace_unit{u != kNone ? v : 0ll, u != kNone ? u - 52 : 0, 255,
                                    (uint8_t)(u != kNone ? QDOT_TRACE_FUSED : QDOT_TRACE_NONE), 0};
    }
  }
  acc = warp_sum_i128(acc);
  for (int c = 0; c < 4; ++c) c5[c] = warp_sum_u64(c5[c]);
  if (lane == 0) {
    s_sum[w] = acc;
    for (int c = 0; c < 4; ++c) s_cnt[w][c] = c5[c];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    FusedPart p;
    p.sum = 0;
    for (int c = 0; c < 4; ++c) p.cnt[c] = 0;
    for (int i = 0; i < kFusedWarps; ++i) {
      p.sum += s_sum[i];
      for (int c = 0; c < 4; ++c) p.cnt[c] += s_cnt[i][c];
    }
    parts[blockIdx.x] = p;
  }
  if (blockIdx.x == 0 && sel) {  // the parameter selection, for qdot_backward
    for (int kk = threadIdx.x; kk < kKeyCount; kk += kFusedThreads) sel->cls[kk] = s_lut[kk];
    if (threadIdx.x == 0) {
      sel->e_max = e_max;
      sel->e_min = s_emin;
      sel->f = f;
      sel->status = s_bad ? QDOT_ERR_NONFINITE : QDOT_OK;
      sel->n_bins = s_nbins;
      sel->block = prm.block;
      sel->key_min = kKeyMin;
      sel->m_half = mh;
      sel->m_single = ms;
      sel->reserved[0] = sel->reserved[1] = 0;
    }
  }
  // ---- phase 4 ----
  fused_finish(parts, arrivals, s_sum, s_cnt, e_max, s_emin, f, s_bad, s_nbins, s_zeros, lsb, out);
}

// Grid of the fused launch on this device (co-resident CTAs), 0 if unknown.
template <int LOG2B>
int fused_grid() {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (grid[dev] == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qdot_fused<LOG2B>, kFusedThreads, 0) !=
        cudaSuccess)
      return 0;
    const int sms = device_info().sms > 0 ? device_info().sms : 0;
    grid[dev] = std::min(per_sm, kFusedCtasPerSm) * sms;
  }
  return grid[dev];
}

template <int LOG2B>
cudaError_t launch_fused_lb(const double* x, const double* y, int64_t n, const qdot_params* p, char* ws,
                            qdot_result* out, qdot_selection* sel, cudaStream_t st, qdot_trace_unit* trace) {
  const int grid = fused_grid<LOG2B>();
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  auto* cstats = reinterpret_cast<CtaStats*>(ws);
  auto* parts = reinterpret_cast<FusedPart*>(ws + align_up(sizeof(CtaStats) * (size_t)grid, 256));
  auto* arrivals = reinterpret_cast<unsigned*>(ws + align_up(sizeof(CtaStats) * (size_t)grid, 256) +
                                               align_up(sizeof(FusedPart) * (size_t)grid, 256));
  long long nn = n;
  qdot_params prm = *p;
  void* args[] = {(void*)&x,        (void*)&y,   (void*)&nn,  (void*)&prm,  (void*)&cstats, (void*)&parts,
                  (void*)&arrivals, (void*)&sel, (void*)&out, (void*)&trace};
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_qdot_fused<LOG2B>, dim3(grid),
                                                    dim3(kFusedThreads), args, 0, st);
  if (ev1) cudaEventRecord(ev1, st);
  return e;
}

template <bool EXACT>
int fused_bins_grid() {
  static int grid[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (grid[dev] == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qdot_fused_bins<EXACT>, kFusedThreads, 0) !=
        cudaSuccess)
      return 0;
    const int sms = device_info().sms > 0 ? device_info().sms : 0;
    grid[dev] = std::min(per_sm, kFusedCtasPerSm) * sms;
  }
  return grid[dev];
}

// Exact binning's workspace beyond the common part: per-CTA non-empty key
// counts, the bin counts M_k and every CTA's key histogram.
size_t bins_extra_bytes(size_t grid) {
  return align_up(sizeof(long long) * grid, 256) + align_up(sizeof(unsigned long long) * kKeyCount, 256) +
         align_up(sizeof(unsigned) * kKeyCount * grid, 256);
}

template <bool EXACT>
cudaError_t launch_fused_bins(const double* x, const double* y, int64_t n, const qdot_params* p, char* ws,
                              qdot_result* out, qdot_selection* sel, cudaStream_t st, TraceOut tr) {
  const int grid = fused_bins_grid<EXACT>();
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  size_t off = 0;
  auto* cstats = reinterpret_cast<CtaStats*>(ws + off);
  off += align_up(sizeof(CtaStats) * (size_t)grid, 256);
  auto* parts = reinterpret_cast<FusedPart*>(ws + off);
  off += align_up(sizeof(FusedPart) * (size_t)grid, 256);
  auto* arrivals = reinterpret_cast<unsigned*>(ws + off);
  off += 256;
  long long* slice_nb = nullptr;
  unsigned long long* gcount = nullptr;
  unsigned* hists = nullptr;
  if (EXACT) {
    slice_nb = reinterpret_cast<long long*>(ws + off);
    off += align_up(sizeof(long long) * (size_t)grid, 256);
    gcount = reinterpret_cast<unsigned long long*>(ws + off);
    off += align_up(sizeof(unsigned long long) * kKeyCount, 256);
    hists = reinterpret_cast<unsigned*>(ws + off);
  }
  long long nn = n;
  qdot_params prm = *p;
  qdot_trace_unit* trace = tr.units;
  uint8_t* tcls = tr.cls;
  void* args[] = {(void*)&x,     (void*)&y,      (void*)&nn,       (void*)&prm, (void*)&cstats,
                  (void*)&parts, (void*)&arrivals, (void*)&hists,  (void*)&gcount, (void*)&slice_nb,
                  (void*)&sel,   (void*)&out,    (void*)&trace,    (void*)&tcls};
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_qdot_fused_bins<EXACT>, dim3(grid),
                                                    dim3(kFusedThreads), args, 0, st);
  if (ev1) cudaEventRecord(ev1, st);
  return e;
}

int fused_grid_for(int log2b) {
  switch (log2b) {
    case 5: return fused_grid<5>();
    case 6: return fused_grid<6>();
    case 7: return fused_grid<7>();
    default: return fused_grid<8>();
  }
}

}  // namespace

bool fused_supported(int64_t n, const qdot_params* p, bool aligned16) {
  if (!aligned16 || n <= 0 || p->block > 256 || (p->block > 1 && p->block < 32)) return false;
  int grid;
  if (p->block <= 1) {
    grid = p->block == 0 ? fused_bins_grid<true>() : fused_bins_grid<false>();
  } else {
    int lb = 0;
    while ((1 << lb) < p->block) ++lb;
    grid = fused_grid_for(lb);
  }
  if (grid <= 0) return false;
  const long long nitems = (n + kItem - 1) / kItem;
  return nitems <= (long long)grid * kFusedWarps * kFusedItems;
}

size_t fused_ws_bytes(const qdot_params* p) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const size_t grid = (size_t)sms * kFusedCtasPerSm;
  size_t b = align_up(sizeof(CtaStats) * grid, 256) + align_up(sizeof(FusedPart) * grid, 256) + 256;
  if (p && p->block == 0) b += bins_extra_bytes(grid);
  return b;
}

const char* fused_stream_kernel(const qdot_params* p) {
  return p->block <= 1 ? "k_qdot_fused_bins" : "k_qdot_fused";
}

cudaError_t launch_fused(const double* x, const double* y, int64_t n, const qdot_params* p, void* ws,
                         qdot_result* out, qdot_selection* sel, cudaStream_t st, TraceOut tr) {
  char* w = static_cast<char*>(ws);
  if (p->block == 0) return launch_fused_bins<true>(x, y, n, p, w, out, sel, st, tr);
  if (p->block == 1) return launch_fused_bins<false>(x, y, n, p, w, out, sel, st, tr);
  int lb = 0;
  while ((1 << lb) < p->block) ++lb;
  switch (lb) {
    case 5: return launch_fused_lb<5>(x, y, n, p, w, out, sel, st, tr.units);
    case 6: return launch_fused_lb<6>(x, y, n, p, w, out, sel, st, tr.units);
    case 7: return launch_fused_lb<7>(x, y, n, p, w, out, sel, st, tr.units);
    default: return launch_fused_lb<8>(x, y, n, p, w, out, sel, st, tr.units);
  }
}

}  // namespace qd
