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

template <int LOG2B>
cudaError_t launch_batched_lb(const double* const* xs, const double* const* ys, const long long* ns, int count,
                              const qdot_params* p, qdot_result* outs, const qdot_batched_tuning& t, char* ws,
                              size_t ws_bytes, cudaStream_t st) {
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
