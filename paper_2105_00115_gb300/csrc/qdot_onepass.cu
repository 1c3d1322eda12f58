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
#include <climits>

#include "qdot_chunk.cuh"
#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

using namespace chunk;

constexpr int kOpThreads = 256;
constexpr int kOpWarps = kOpThreads / 32;

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
  int status, pad;
  long long zeros;
};
struct OpPart {
  i128 sum;
  unsigned long long cnt[4];
};


template <int LOG2B>
__global__ void __launch_bounds__(kOpThreads, 2) k_onepass(const double* __restrict__ x,
                                                           const double* __restrict__ y, long long n,
                                                           WarpStats* __restrict__ wstats,
                                                           BlockRec* __restrict__ recs) {
  constexpr long long B = 1ll << LOG2B;
  constexpr int kChunks = (int)(B / 32);
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, sub = lane & 3;
  long long nbins = 0, zeros_l = 0;
  int emax_l = kNone, kmin = INT_MAX, bad = 0;

  const long long nblocks = (n + B - 1) / B;
  const long long ngroups = (nblocks + kBlocksPerWarp - 1) / kBlocksPerWarp;
  const long long gwarp = ((long long)blockIdx.x * kOpThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kOpThreads) >> 5;

  long long grp = gwarp;
  int c = 0;
  Chunk cur, nxt;
  if (grp < ngroups) load_chunk<LOG2B>(x, y, n, grp * kBlocksPerWarp + g, 0, sub, cur);
  int u_run = kNone, M = 0, zeros = 0;
  long long aH = 0, aS = 0;
  double aD = 0.0;
  while (grp < ngroups) {
    // prefetch the next chunk of this warp
    long long ngrp = grp;
    int nc = c + 1;
    if (nc == kChunks) {
      nc = 0;
      ngrp = grp + nwarps;
    }
    if (ngrp < ngroups) load_chunk<LOG2B>(x, y, n, ngrp * kBlocksPerWarp + g, nc, sub, nxt);
    int key[8];
    int cmax = kNone;
    if (__all_sync(0xffffffffu, chunk_keys(cur, key, cmax, kmin))) {
      chunk_fast<LOG2B>(cur, key, cmax, u_run, aH, aS, aD);
      M += 8;
    } else {
      chunk_general<LOG2B>(cur, u_run, aH, aS, aD, M, zeros, kmin, bad);
    }
    if (c == kChunks - 1) {
      int key, u, mb;
      const long long word = block_record_word<LOG2B>(aH, aS, aD, M, u_run, sub, &key, &u, &mb);
      const long long blk = grp * kBlocksPerWarp + g;
      zeros_l += zeros;
      if (blk < nblocks) {
        if (mb > 0) {
          nbins += (sub == 0);
          emax_l = max(emax_l, u);
        }
        reinterpret_cast<long long*>(recs + blk)[sub] = word;
      }
      u_run = kNone;
      M = 0;
      zeros = 0;
      aH = aS = 0;
      aD = 0.0;
    }
    cur = nxt;
    grp = ngrp;
    c = nc;
  }

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
  }
  __syncthreads();
  const int e_max = sel->e_max, f = s_f;
  const int mh = prm.mant_reading ? 11 : 10, ms = prm.mant_reading ? 24 : 23;
  for (int k = threadIdx.x; k < kKeyCount; k += blockDim.x)
    sel->cls[k] = (uint8_t)precision_of((long long)kKeyMin + k - e_max - f + 1, mh, ms);
}

// Deferred selection: per block record pick the candidate of the block's
// class and add it exactly to a fixed-point sum anchored at 2^(e_max - L).
__global__ void __launch_bounds__(256) k_op_gather(const BlockRec* __restrict__ recs, long long nblocks, int log2b,
                                                   const qdot_selection* __restrict__ sel,
                                                   const OpHeader* __restrict__ hdr, OpPart* __restrict__ parts) {
  __shared__ uint8_t s_lut[kKeyCount];
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][4];
  for (int i = threadIdx.x; i < kKeyCount / 4; i += blockDim.x)
    reinterpret_cast<uint32_t*>(s_lut)[i] = reinterpret_cast<const uint32_t*>(sel->cls)[i];
  __syncthreads();
  const int lsb = hdr->lsb;
  const bool ok = hdr->status == QDOT_OK;
  i128 acc = 0;
  unsigned long long c[4] = {0, 0, 0, 0};
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; ok && b < nblocks;
       b += (long long)gridDim.x * blockDim.x) {
    const longlong2 r0 = reinterpret_cast<const longlong2*>(recs + b)[0];
    const longlong2 r1 = reinterpret_cast<const longlong2*>(recs + b)[1];
    const int key = (int)(short)(r1.y & 0xFFFF);
    if (key == kEmptyKey) continue;
    const int u = (int)(short)((r1.y >> 16) & 0xFFFF);
    const unsigned m = (unsigned)((unsigned long long)r1.y >> 32);
    const int cls = s_lut[key - kKeyMin];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] += (cls == k) ? m : 0u;
    acc += record_candidate(r0.x, r0.y, r1.x, u, cls, log2b, lsb);
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
    OpPart p;
    p.sum = 0;
    for (int k = 0; k < 4; ++k) p.cnt[k] = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      p.sum += s_sum[i];
      for (int k = 0; k < 4; ++k) p.cnt[k] += s_cnt[i][k];
    }
    parts[blockIdx.x] = p;
  }
}

__global__ void __launch_bounds__(256) k_op_final(const OpPart* __restrict__ parts, int np,
                                                  const qdot_selection* __restrict__ sel,
                                                  const OpHeader* __restrict__ hdr, qdot_result* __restrict__ out) {
  __shared__ i128 s_sum[8];
  __shared__ unsigned long long s_cnt[8][4];
  i128 acc = 0;
  unsigned long long c[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    acc += parts[i].sum;
    for (int k = 0; k < 4; ++k) c[k] += parts[i].cnt[k];
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

template <int LOG2B>
cudaError_t launch_lb(const double* x, const double* y, int64_t n, const qdot_params* p, const OnePassPlan& pl,
                      char* ws, qdot_result* out, cudaStream_t st) {
  auto* sel = reinterpret_cast<qdot_selection*>(ws + pl.off_sel);
  auto* hdr = reinterpret_cast<OpHeader*>(ws + pl.off_hdr);
  auto* wst = reinterpret_cast<WarpStats*>(ws + pl.off_rec);
  auto* recs = reinterpret_cast<BlockRec*>(ws + pl.off_misc);
  auto* parts = reinterpret_cast<OpPart*>(ws + pl.off_sel + align_up(sizeof(qdot_selection), 256) +
                                          align_up(sizeof(OpHeader), 256));
  cudaEvent_t ev0, ev1;
  kernel_events(&ev0, &ev1);
  if (ev0) cudaEventRecord(ev0, st);
  k_onepass<LOG2B><<<pl.grid, kOpThreads, 0, st>>>(x, y, n, wst, recs);
  if (ev1) cudaEventRecord(ev1, st);
  const int nw = pl.grid * kOpWarps;
  k_op_select<<<1, 1024, 0, st>>>(wst, nw, n, *p, sel, hdr);
  const int gather_grid = 4 * (device_info().sms > 0 ? device_info().sms : 152);
  const long long nblocks = (n + (1ll << LOG2B) - 1) >> LOG2B;
  k_op_gather<<<gather_grid, 256, 0, st>>>(recs, nblocks, LOG2B, sel, hdr, parts);
  k_op_final<<<1, 256, 0, st>>>(parts, gather_grid, sel, hdr, out);
  return cudaGetLastError();
}

}  // namespace

bool one_pass_supported(int64_t n, const qdot_params* p, bool aligned16) {
  return aligned16 && n > 0 && p->block >= 32 && p->block <= 256;
}

int one_pass_launches(int64_t, const qdot_params*) { return 4; }

OnePassPlan plan_one_pass(int64_t n, const qdot_params* p) {
  OnePassPlan pl;
  int lb = 0;
  while ((1 << lb) < p->block) ++lb;
  pl.log2b = lb;
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  pl.grid = sms * 2;
  const long long nblocks = (n + p->block - 1) / p->block;
  size_t off = 0;
  pl.off_sel = off;
  off = align_up(off + sizeof(qdot_selection), 256);
  pl.off_hdr = off;
  off = align_up(off + sizeof(OpHeader), 256);
  off = align_up(off + sizeof(OpPart) * 4 * sms, 256);  // gather partials
  pl.off_rec = off;
  off = align_up(off + sizeof(WarpStats) * pl.grid * kOpWarps, 256);
  pl.off_misc = off;
  off = align_up(off + sizeof(BlockRec) * (size_t)nblocks, 256);
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
