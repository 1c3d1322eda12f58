// The paper's two applications, with every dot product a qdot:
//   ACG (Algorithm 4): conjugate gradients, qdot for p.q and r.r; the loop
//        runs while sqrt(c_k) / ||b|| > tau (the residual norm the algorithm
//        holds, relative to ||b||, which is computed exactly).
//   APM (Algorithm 5): power method, qdot for the Rayleigh quotient x.(Ax)
//        (||x|| = 1) and for ||Ax||^2; x <- Ax / sqrt(c).
// Scalars (alpha, beta, c, lambda) stay on the device.  A batch of iterations
// is recorded once as a CUDA graph and replayed until a device flag reports
// convergence; kernels of iterations past convergence return at once.
// Vector updates use fused multiply-adds in the same order as the oracle, and
// SpMV sums each CSR row in storage order with fused multiply-adds.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

constexpr int kIterPerGraph = 16;

struct SolverState {
  double c, pq, alpha, beta, bnorm, lam, lam_prev, s, tol, tau;
  int k, done, status, max_it;
  int active;  // 1 when the current iteration runs (read by the vector kernels)
  int pad;
  long long counts[5];
};

__global__ void k_spmv(const long long* __restrict__ rowptr, const int* __restrict__ col,
                       const double* __restrict__ val, long long n, const double* __restrict__ xin,
                       double* __restrict__ yout, const SolverState* __restrict__ st) {
  if (st && st->done) return;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (long long k = rowptr[r]; k < rowptr[r + 1]; ++k) s = fma(val[k], __ldg(xin + col[k]), s);
    yout[r] = s;
  }
}

__device__ __forceinline__ void add_counts(SolverState* st, const qdot_result& r, long long* hist_slot) {
  for (int c = 0; c < 5; ++c) {
    st->counts[c] += r.count[c];
    if (hist_slot) hist_slot[c] = r.count[c];
  }
  if (r.status != QDOT_OK) {
    st->status = r.status;
    st->done = 1;
  }
}

// ---- ACG ----
__global__ void k_cg_init_vectors(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r,
                                  double* __restrict__ p, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = b[i] - ax[i];
    r[i] = v;
    p[i] = v;
  }
}

__global__ void k_cg_init_state(SolverState* st, const qdot_result* __restrict__ rr, const qdot_result* __restrict__ bb,
                                double tol, int max_it) {
  SolverState s = {};
  s.tol = tol;
  s.max_it = max_it;
  s.status = QDOT_OK;
  s.c = rr->value;
  s.bnorm = sqrt(bb->value);
  s.k = 0;
  *st = s;
  add_counts(st, *rr, nullptr);
  if (bb->status != QDOT_OK) st->status = bb->status;
  st->done = (st->status != QDOT_OK) || !(0 < max_it && sqrt(st->c) / st->bnorm > tol);
}

__global__ void k_cg_alpha(SolverState* st, const qdot_result* __restrict__ pq, long long* __restrict__ hist) {
  if (st->done) {
    st->active = 0;
    return;
  }
  st->active = 1;
  add_counts(st, *pq, hist ? hist + (long long)st->k * 10 : nullptr);
  st->pq = pq->value;
  st->alpha = st->c / st->pq;
}

__global__ void k_cg_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                            const double* __restrict__ q, long long n, const SolverState* __restrict__ st) {
  if (!st->active || st->done) return;
  const double a = st->alpha;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

__global__ void k_cg_beta(SolverState* st, const qdot_result* __restrict__ rr, long long* __restrict__ hist) {
  if (!st->active || st->done) {
    st->active = 0;
    return;
  }
  add_counts(st, *rr, hist ? hist + (long long)st->k * 10 + 5 : nullptr);
  const double c_new = rr->value;
  st->beta = c_new / st->c;
  st->c = c_new;
  st->k += 1;
  if (!(st->k < st->max_it && sqrt(st->c) / st->bnorm > st->tol)) st->done = 1;
}

__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ r, long long n,
                       const SolverState* __restrict__ st) {
  if (!st->active) return;
  const double be = st->beta;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(be, p[i], r[i]);
}

__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ res,
                           long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    res[i] = b[i] - ax[i];
}

__global__ void k_cg_finish(const SolverState* __restrict__ st, const qdot_result* __restrict__ true_rr,
                            qdot_cg_info* __restrict__ info) {
  qdot_cg_info o;
  o.iters = st->k;
  o.status = st->status != QDOT_OK ? st->status : (sqrt(st->c) / st->bnorm > st->tol ? QDOT_ERR_NOCONV : QDOT_OK);
  o.relres = sqrt(st->c) / st->bnorm;
  o.true_relres = sqrt(true_rr->value) / st->bnorm;
  for (int c = 0; c < 5; ++c) o.counts[c] = st->counts[c];
  *info = o;
}

// ---- APM ----
__global__ void k_pm_init_state(SolverState* st, int iters, double tau) {
  SolverState s = {};
  s.max_it = iters;
  s.tau = tau;
  s.status = QDOT_OK;
  s.done = iters <= 0;
  *st = s;
}

__global__ void k_pm_step(SolverState* st, const qdot_result* __restrict__ lam, const qdot_result* __restrict__ cc,
                          long long* __restrict__ hist) {
  if (st->done) {
    st->active = 0;
    return;
  }
  st->active = 1;
  add_counts(st, *lam, hist ? hist + (long long)st->k * 10 : nullptr);
  add_counts(st, *cc, hist ? hist + (long long)st->k * 10 + 5 : nullptr);
  st->lam = lam->value;
  st->s = 1.0 / sqrt(cc->value);
  const bool conv = st->tau > 0.0 && st->k > 0 && fabs(st->lam - st->lam_prev) <= st->tau;
  st->k += 1;
  if (conv || st->k >= st->max_it) st->done = 1;
  st->lam_prev = st->lam;
}

__global__ void k_pm_scale(double* __restrict__ x, const double* __restrict__ w, long long n,
                           const SolverState* __restrict__ st) {
  if (!st->active) return;
  const double s = st->s;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = w[i] * s;
}

__global__ void k_pm_finish(const SolverState* __restrict__ st, qdot_power_info* __restrict__ info) {
  qdot_power_info o;
  o.iters = st->k;
  o.status = st->status;
  o.lambda = st->lam;
  for (int c = 0; c < 5; ++c) o.counts[c] = st->counts[c];
  *info = o;
}

// ||b|| and the final true residual of ACG: qdot with every component in the
// double class (eps = 1e-300 puts every bin score above m_single).
constexpr qdot_params kDoubleClass = {1e-300, 0, 1, 0, QDOT_PATH_AUTO};

struct SolverLayout {
  size_t off_state, off_res, off_vec, off_qws, total;
};

SolverLayout solver_layout(int64_t n, int nvec, const qdot_params* p) {
  SolverLayout l;
  size_t off = 0;
  l.off_state = off;
  off = align_up(off + sizeof(SolverState), 256);
  l.off_res = off;
  off = align_up(off + 4 * sizeof(qdot_result), 256);
  l.off_vec = off;
  off = align_up(off + (size_t)nvec * sizeof(double) * (size_t)n, 256);
  l.off_qws = off;
  off = align_up(off + std::max({qdot_ws_bytes(n, p), qdot_ws_bytes(n, &kDoubleClass), dot_fp64_workspace()}), 256);
  l.total = off;
  return l;
}

int vec_grid(long long n) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  long long g = (n + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(g, (long long)sms * 8));
}

cudaStream_t capture_stream(cudaError_t* err) {
  static std::mutex mu;
  static cudaStream_t streams[64] = {nullptr};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!streams[dev]) *err = cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking);
  return streams[dev];
}

// Record `iters` iterations produced by `body` into a graph.
template <typename Body>
cudaError_t record_graph(Body body, int iters, cudaGraphExec_t* exec) {
  cudaError_t e;
  cudaStream_t cs = capture_stream(&e);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t be = cudaSuccess;
  for (int i = 0; i < iters && be == cudaSuccess; ++i) be = body(cs);
  e = cudaStreamEndCapture(cs, &g);
  if (be != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return be;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Replay the graph until the device flag says done (checked once per replay).
cudaError_t run_until_done(cudaGraphExec_t exec, const int* done_flag, int max_replays, cudaStream_t stream) {
  for (int r = 0; r < max_replays; ++r) {
    cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return e;
    int done = 0;
    e = cudaMemcpyAsync(&done, done_flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    if (done) break;
  }
  return cudaSuccess;
}

// Parameters the solver's qdot calls use: `p` with QDOT_PATH_FP64_DOT mapped
// to QDOT_PATH_AUTO (the plain-dot switch is read separately).
bool solver_params(const qdot_csr* A, const qdot_params* p, qdot_params* qp, bool* plain, const char* who) {
  std::string why;
  if (!p) {
    set_error(std::string(who) + ": params pointer is NULL");
    return false;
  }
  *qp = *p;
  *plain = p->path == QDOT_PATH_FP64_DOT;
  if (*plain) *qp = qdot_params{1e-16, 0, 1, 0, QDOT_PATH_AUTO};
  if (!valid_params(A ? A->n : 0, qp, &why)) {
    set_error(std::string(who) + ": " + why);
    return false;
  }
  return true;
}

// One dot product of a solver iteration into res (value; counts and status
// too for qdot).  The plain dot leaves the other fields as zeroed at start.
cudaError_t solver_dot(bool plain, const double* a, const double* b, long long n, const qdot_params* qp, void* qws,
                       qdot_result* res, cudaStream_t s) {
  if (plain) return launch_dot_fp64(a, b, n, &res->value, qws, s);
  return launch_qdot_auto(a, b, n, qp, qws, res, s);
}

qdot_status check_csr(const qdot_csr* A, const char* who) {
  if (!A || A->n < 0 || (A->n > 0 && (!A->rowptr || !A->col || !A->val))) {
    set_error(std::string(who) + ": invalid CSR matrix");
    return QDOT_ERR_ARG;
  }
  return QDOT_OK;
}

qdot_status fail(const char* who, cudaError_t e) {
  set_error(std::string(who) + ": " + cudaGetErrorString(e));
  return QDOT_ERR_CUDA;
}


// ---------------------------------------------------------------------------
// Batched ACG: `count` independent SPD systems (the diagonal blocks of one
// block-diagonal CSR matrix) solved together, every kernel of an iteration
// covering all systems: one SpMV launch, one batched qdot launch per dot
// product, one launch per vector update.  Each system keeps its own scalars
// and stops on its own; a stopped system's rows are skipped and its dot
// products get length 0.  Internal vectors use padded offsets so that every
// system's slice starts on a 16-byte boundary (the batched qdot needs it).
// Work over rows is split into tiles of 256 rows of one system.
// ---------------------------------------------------------------------------
constexpr int kTileRows = 256;

struct BatchSys {
  double c, bnorm;
  double alpha, beta;
  int k, active, status, pad;
  long long counts[5];
};

struct RowTile {
  int sys, nrows;
  long long row0;  // first row (global, unpadded)
};

struct BatchView {
  const long long* off;   // [count + 1] row offsets of the systems
  const long long* poff;  // [count + 1] padded offsets of their internal slices
  const RowTile* tiles;
  long long ntiles;
  int count;
};

__device__ __forceinline__ long long padded(const BatchView& v, int s, long long r) {
  return r - v.off[s] + v.poff[s];
}

// dst_pad = A src (src padded, or the caller's unpadded x), rows of active
// systems only when `sys` is given.  A column outside its row's system is
// skipped and flags *bad.
__global__ void k_bcg_spmv(const long long* __restrict__ rowptr, const int* __restrict__ col,
                           const double* __restrict__ val, BatchView v, const double* __restrict__ src,
                           int src_padded, double* __restrict__ dst, const BatchSys* __restrict__ sys,
                           int* __restrict__ bad) {
  for (long long t = blockIdx.x; t < v.ntiles; t += gridDim.x) {
    const RowTile tile = v.tiles[t];
    if (sys && !sys[tile.sys].active) continue;
    if ((int)threadIdx.x >= tile.nrows) continue;
    const int s = tile.sys;
    const long long r = tile.row0 + threadIdx.x;
    const long long lo = v.off[s], hi = v.off[s + 1], shift = v.poff[s] - lo;
    double acc = 0.0;
    for (long long k = rowptr[r]; k < rowptr[r + 1]; ++k) {
      const long long c = col[k];
      if (c < lo || c >= hi) {
        *bad = 1;
        continue;
      }
      acc = fma(val[k], __ldg(src + (src_padded ? c + shift : c)), acc);
    }
    dst[r + shift] = acc;
  }
}

__global__ void k_bcg_init_vectors(BatchView v, const double* __restrict__ b, const double* __restrict__ ax,
                                   double* __restrict__ r, double* __restrict__ p, double* __restrict__ bp) {
  for (long long t = blockIdx.x; t < v.ntiles; t += gridDim.x) {
    const RowTile tile = v.tiles[t];
    if ((int)threadIdx.x >= tile.nrows) continue;
    const long long row = tile.row0 + threadIdx.x;
    const long long i = padded(v, tile.sys, row);
    const double d = b[row] - ax[i];
    r[i] = d;
    p[i] = d;
    bp[i] = b[row];
  }
}

__global__ void k_bcg_init_state(BatchSys* __restrict__ sys, const qdot_result* __restrict__ rr,
                                 const qdot_result* __restrict__ bb, long long* __restrict__ ns_dot, int count,
                                 double tol, int max_it, int* __restrict__ remaining) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;  // *remaining and *all_done start at 0
  if (s >= count) return;
  BatchSys st = {};
  st.c = rr[s].value;
  st.bnorm = sqrt(bb[s].value);
  st.status = rr[s].status != QDOT_OK ? rr[s].status : bb[s].status;
  for (int k = 0; k < 5; ++k) st.counts[k] = rr[s].count[k];
  st.active = st.status == QDOT_OK && 0 < max_it && sqrt(st.c) / st.bnorm > tol;
  sys[s] = st;
  if (!st.active) ns_dot[s] = 0;
  if (st.active) atomicAdd(remaining, 1);
}

__global__ void k_bcg_all_done(const int* __restrict__ remaining, int* __restrict__ all_done) {
  *all_done = *remaining == 0;
}

__global__ void k_bcg_alpha(BatchSys* __restrict__ sys, const qdot_result* __restrict__ pq, int count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count || !sys[s].active) return;
  for (int k = 0; k < 5; ++k) sys[s].counts[k] += pq[s].count[k];
  if (pq[s].status != QDOT_OK) sys[s].status = pq[s].status;
  sys[s].alpha = sys[s].c / pq[s].value;
}

__global__ void k_bcg_update(BatchView v, double* __restrict__ x, double* __restrict__ r,
                             const double* __restrict__ p, const double* __restrict__ q,
                             const BatchSys* __restrict__ sys) {
  for (long long t = blockIdx.x; t < v.ntiles; t += gridDim.x) {
    const RowTile tile = v.tiles[t];
    const BatchSys& st = sys[tile.sys];
    if (!st.active || (int)threadIdx.x >= tile.nrows) continue;
    const long long row = tile.row0 + threadIdx.x;
    const long long i = padded(v, tile.sys, row);
    const double a = st.alpha;
    x[row] = fma(a, p[i], x[row]);
    r[i] = fma(-a, q[i], r[i]);
  }
}

__global__ void k_bcg_beta(BatchSys* __restrict__ sys, const qdot_result* __restrict__ rr, int count, double tol,
                           int max_it, long long* __restrict__ ns_dot, int* __restrict__ remaining) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < count && sys[s].active) {
    BatchSys& st = sys[s];
    for (int k = 0; k < 5; ++k) st.counts[k] += rr[s].count[k];
    if (rr[s].status != QDOT_OK) st.status = rr[s].status;
    const double c_new = rr[s].value;
    st.beta = c_new / st.c;
    st.c = c_new;
    st.k += 1;
    if (st.status != QDOT_OK || !(st.k < max_it && sqrt(st.c) / st.bnorm > tol)) {
      st.active = 0;  // p is still updated once below; nothing reads it afterwards
      ns_dot[s] = 0;
      atomicSub(remaining, 1);
    }
  }
}

__global__ void k_bcg_p(BatchView v, double* __restrict__ p, const double* __restrict__ r,
                        const BatchSys* __restrict__ sys) {
  for (long long t = blockIdx.x; t < v.ntiles; t += gridDim.x) {
    const RowTile tile = v.tiles[t];
    const BatchSys& st = sys[tile.sys];
    if (!st.active || (int)threadIdx.x >= tile.nrows) continue;
    const long long i = padded(v, tile.sys, tile.row0 + threadIdx.x);
    p[i] = fma(st.beta, p[i], r[i]);
  }
}

__global__ void k_bcg_residual(BatchView v, const double* __restrict__ bp, const double* __restrict__ ax,
                               double* __restrict__ res) {
  for (long long t = blockIdx.x; t < v.ntiles; t += gridDim.x) {
    const RowTile tile = v.tiles[t];
    if ((int)threadIdx.x >= tile.nrows) continue;
    const long long i = padded(v, tile.sys, tile.row0 + threadIdx.x);
    res[i] = bp[i] - ax[i];
  }
}

__global__ void k_bcg_finish(const BatchSys* __restrict__ sys, const qdot_result* __restrict__ true_rr, int count,
                             double tol, const int* __restrict__ bad, qdot_cg_info* __restrict__ infos) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= count) return;
  const BatchSys st = sys[s];
  qdot_cg_info o;
  o.iters = st.k;
  o.relres = sqrt(st.c) / st.bnorm;
  o.status = *bad ? QDOT_ERR_ARG
                  : (st.status != QDOT_OK ? st.status : (o.relres > tol ? QDOT_ERR_NOCONV : QDOT_OK));
  o.true_relres = sqrt(true_rr[s].value) / st.bnorm;
  for (int k = 0; k < 5; ++k) o.counts[k] = st.counts[k];
  infos[s] = o;
}

// Plain FP64 dot per system (the comparator): one warp per tile (8 rows per
// lane, one fused multiply-add chain each), per-tile partial sums, then one
// warp per system adds its tiles in order (deterministic).
__global__ void k_bcg_dot_tiles(BatchView v, const double* __restrict__ a, const double* __restrict__ b,
                                double* __restrict__ part, const long long* __restrict__ ns_dot) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < v.ntiles; t += nwarps) {
    const RowTile tile = v.tiles[t];
    double acc = 0.0;
    if (ns_dot[tile.sys] > 0) {
      const long long i0 = padded(v, tile.sys, tile.row0);
      for (int r = lane; r < tile.nrows; r += 32) acc = fma(a[i0 + r], b[i0 + r], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part[t] = acc;
  }
}

__global__ void k_bcg_dot_final(const double* __restrict__ part, const long long* __restrict__ tile_start, int count,
                                qdot_result* __restrict__ out) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= count) return;
  double acc = 0.0;
  for (long long t = tile_start[s] + lane; t < tile_start[s + 1]; t += 32) acc += part[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    qdot_result r = {};
    r.value = acc;
    r.status = QDOT_OK;
    out[s] = r;
  }
}

struct BatchLayoutCg {
  size_t off_sys, off_res, off_nsd, off_nsf, off_off, off_poff, off_tiles, off_tstart, off_part, off_ptr, off_flags,
      off_vec, off_qws, total;
  long long ntiles, total_pad;
  size_t qws_bytes;
};

BatchLayoutCg batch_cg_layout(const int64_t* row_off, int count, const qdot_params* qp) {
  BatchLayoutCg l;
  long long ntiles = 0, pad = 0;
  std::vector<int64_t> ns(count);
  for (int s = 0; s < count; ++s) {
    const long long m = row_off[s + 1] - row_off[s];
    ns[s] = m;
    ntiles += (m + kTileRows - 1) / kTileRows;
    pad += (m + 1) & ~1ll;  // slices of an even number of doubles: 16-byte aligned starts
  }
  l.ntiles = ntiles;
  l.total_pad = pad;
  const qdot_params exact = {1e-300, 32, 1, 0, QDOT_PATH_AUTO};
  l.qws_bytes = std::max(batched_ws_bytes(ns.data(), count, qp), batched_ws_bytes(ns.data(), count, &exact));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  l.off_sys = take(sizeof(BatchSys) * count);
  l.off_res = take(sizeof(qdot_result) * 3 * count);
  l.off_nsd = take(sizeof(long long) * count);
  l.off_nsf = take(sizeof(long long) * count);
  l.off_off = take(sizeof(long long) * (count + 1));
  l.off_poff = take(sizeof(long long) * (count + 1));
  l.off_tiles = take(sizeof(RowTile) * (ntiles > 0 ? ntiles : 1));
  l.off_tstart = take(sizeof(long long) * (count + 1));
  l.off_part = take(sizeof(double) * (ntiles > 0 ? ntiles : 1));
  l.off_ptr = take(sizeof(double*) * 4 * count);
  l.off_flags = take(sizeof(int) * 4);
  l.off_vec = take(sizeof(double) * 4 * (size_t)pad);
  l.off_qws = take(l.qws_bytes);
  l.total = off;
  return l;
}

}  // namespace
}  // namespace qd

using namespace qd;

extern "C" {

size_t qdot_cg_workspace_size(int64_t n, const qdot_params* p) {
  qdot_csr shape = {n, 0, nullptr, nullptr, nullptr};
  qdot_params qp;
  bool plain;
  if (!solver_params(&shape, p, &qp, &plain, "qdot_cg_workspace_size")) return 0;
  return solver_layout(n, 3, &qp).total;
}

qdot_status qdot_cg(const qdot_csr* A, const double* b, double* x, double rel_tol, int32_t max_it,
                    const qdot_params* p, qdot_cg_info* info, int64_t* class_hist, void* ws, size_t ws_bytes,
                    void* stream) {
  clear_error();
  qdot_params qp;
  bool plain = false;
  if (!solver_params(A, p, &qp, &plain, "qdot_cg")) return QDOT_ERR_ARG;
  if (check_csr(A, "qdot_cg") != QDOT_OK) return QDOT_ERR_ARG;
  const long long n = A->n;
  if (n == 0 || !b || !x || !info || max_it < 0 || !(rel_tol >= 0.0)) {
    set_error("qdot_cg: need n > 0, device b, x, info, max_it >= 0 and rel_tol >= 0");
    return QDOT_ERR_ARG;
  }
  const SolverLayout l = solver_layout(n, 3, &qp);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < l.total) {
    set_error("qdot_cg: workspace missing, misaligned or smaller than qdot_cg_workspace_size()");
    return QDOT_ERR_WORKSPACE;
  }
  char* w = static_cast<char*>(ws);
  auto* st = reinterpret_cast<SolverState*>(w + l.off_state);
  auto* res = reinterpret_cast<qdot_result*>(w + l.off_res);  // [0] p.q, [1] r.r, [2] b.b / true r.r
  double* r = reinterpret_cast<double*>(w + l.off_vec);
  double* pv = r + n;
  double* q = pv + n;
  void* qws = w + l.off_qws;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = vec_grid(n);
  const long long* rowptr = reinterpret_cast<const long long*>(A->rowptr);
  long long* hist = reinterpret_cast<long long*>(class_hist);
  cudaError_t e;
  if ((e = cudaMemsetAsync(res, 0, 4 * sizeof(qdot_result), s)) != cudaSuccess) return fail("qdot_cg", e);
  // r0 = b - A x0, p0 = r0, c0 = qdot(r0, r0), ||b|| exact
  k_spmv<<<grid, 256, 0, s>>>(rowptr, A->col, A->val, n, x, q, nullptr);
  k_cg_init_vectors<<<grid, 256, 0, s>>>(b, q, r, pv, n);
  if ((e = solver_dot(plain, r, r, n, &qp, qws, res + 1, s)) != cudaSuccess) return fail("qdot_cg", e);
  if ((e = launch_qdot_auto(b, b, n, &kDoubleClass, qws, res + 2, s)) != cudaSuccess) return fail("qdot_cg", e);
  k_cg_init_state<<<1, 1, 0, s>>>(st, res + 1, res + 2, rel_tol, max_it);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_cg", e);
  auto body = [&](cudaStream_t cs) -> cudaError_t {
    k_spmv<<<grid, 256, 0, cs>>>(rowptr, A->col, A->val, n, pv, q, st);
    cudaError_t ee = solver_dot(plain, pv, q, n, &qp, qws, res + 0, cs);
    if (ee != cudaSuccess) return ee;
    k_cg_alpha<<<1, 1, 0, cs>>>(st, res + 0, hist);
    k_cg_update<<<grid, 256, 0, cs>>>(x, r, pv, q, n, st);
    ee = solver_dot(plain, r, r, n, &qp, qws, res + 1, cs);
    if (ee != cudaSuccess) return ee;
    k_cg_beta<<<1, 1, 0, cs>>>(st, res + 1, hist);
    k_cg_p<<<grid, 256, 0, cs>>>(pv, r, n, st);
    return cudaGetLastError();
  };
  cudaGraphExec_t exec = nullptr;
  if ((e = record_graph(body, kIterPerGraph, &exec)) != cudaSuccess) return fail("qdot_cg: graph", e);
  e = run_until_done(exec, &st->done, max_it / kIterPerGraph + 2, s);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail("qdot_cg", e);
  // true residual ||b - A x|| / ||b|| (exact dot)
  k_spmv<<<grid, 256, 0, s>>>(rowptr, A->col, A->val, n, x, q, nullptr);
  k_residual<<<grid, 256, 0, s>>>(b, q, r, n);
  if ((e = launch_qdot_auto(r, r, n, &kDoubleClass, qws, res + 2, s)) != cudaSuccess) return fail("qdot_cg", e);
  k_cg_finish<<<1, 1, 0, s>>>(st, res + 2, info);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_cg", e);
  return QDOT_OK;
}

size_t qdot_power_workspace_size(int64_t n, const qdot_params* p) {
  qdot_csr shape = {n, 0, nullptr, nullptr, nullptr};
  qdot_params qp;
  bool plain;
  if (!solver_params(&shape, p, &qp, &plain, "qdot_power_workspace_size")) return 0;
  return solver_layout(n, 1, &qp).total;
}

qdot_status qdot_power(const qdot_csr* A, double* x, int32_t iters, double tau, const qdot_params* p,
                       qdot_power_info* info, int64_t* class_hist, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  qdot_params qp;
  bool plain = false;
  if (!solver_params(A, p, &qp, &plain, "qdot_power")) return QDOT_ERR_ARG;
  if (check_csr(A, "qdot_power") != QDOT_OK) return QDOT_ERR_ARG;
  const long long n = A->n;
  if (n == 0 || !x || !info || iters < 0 || !(tau >= 0.0)) {
    set_error("qdot_power: need n > 0, device x and info, iters >= 0 and tau >= 0");
    return QDOT_ERR_ARG;
  }
  const SolverLayout l = solver_layout(n, 1, &qp);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < l.total) {
    set_error("qdot_power: workspace missing, misaligned or smaller than qdot_power_workspace_size()");
    return QDOT_ERR_WORKSPACE;
  }
  char* w = static_cast<char*>(ws);
  auto* st = reinterpret_cast<SolverState*>(w + l.off_state);
  auto* res = reinterpret_cast<qdot_result*>(w + l.off_res);  // [0] x.(Ax), [1] (Ax).(Ax)
  double* wv = reinterpret_cast<double*>(w + l.off_vec);
  void* qws = w + l.off_qws;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = vec_grid(n);
  const long long* rowptr = reinterpret_cast<const long long*>(A->rowptr);
  long long* hist = reinterpret_cast<long long*>(class_hist);
  cudaError_t e;
  if ((e = cudaMemsetAsync(res, 0, 4 * sizeof(qdot_result), s)) != cudaSuccess) return fail("qdot_power", e);
  k_pm_init_state<<<1, 1, 0, s>>>(st, iters, tau);
  auto body = [&](cudaStream_t cs) -> cudaError_t {
    k_spmv<<<grid, 256, 0, cs>>>(rowptr, A->col, A->val, n, x, wv, st);
    cudaError_t ee = solver_dot(plain, x, wv, n, &qp, qws, res + 0, cs);
    if (ee != cudaSuccess) return ee;
    ee = solver_dot(plain, wv, wv, n, &qp, qws, res + 1, cs);
    if (ee != cudaSuccess) return ee;
    k_pm_step<<<1, 1, 0, cs>>>(st, res + 0, res + 1, hist);
    k_pm_scale<<<grid, 256, 0, cs>>>(x, wv, n, st);
    return cudaGetLastError();
  };
  cudaGraphExec_t exec = nullptr;
  if ((e = record_graph(body, kIterPerGraph, &exec)) != cudaSuccess) return fail("qdot_power: graph", e);
  e = run_until_done(exec, &st->done, iters / kIterPerGraph + 2, s);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail("qdot_power", e);
  k_pm_finish<<<1, 1, 0, s>>>(st, info);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_power", e);
  return QDOT_OK;
}


size_t qdot_cg_batched_workspace_size(const int64_t* row_off_host, int32_t count, const qdot_params* p) {
  if (!row_off_host || count <= 0 || !p) return 0;
  for (int s = 0; s < count; ++s)
    if (row_off_host[s + 1] < row_off_host[s] || row_off_host[0] != 0) return 0;
  qdot_params qp = *p;
  if (qp.path == QDOT_PATH_FP64_DOT) qp = qdot_params{1e-16, 32, 1, 0, QDOT_PATH_AUTO};
  std::string why;
  if (!valid_params(0, &qp, &why) || qp.block < 32 || qp.block > 256) return 0;
  return batch_cg_layout(row_off_host, count, &qp).total;
}

qdot_status qdot_cg_batched(const qdot_csr* A, const int64_t* row_off_host, int32_t count, const double* b,
                            double* x, double rel_tol, int32_t max_it, const qdot_params* p, qdot_cg_info* infos,
                            void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  if (!p) {
    set_error("qdot_cg_batched: params pointer is NULL");
    return QDOT_ERR_ARG;
  }
  const bool plain = p->path == QDOT_PATH_FP64_DOT;
  qdot_params qp = plain ? qdot_params{1e-16, 32, 1, 0, QDOT_PATH_AUTO} : *p;
  std::string why;
  if (!valid_params(0, &qp, &why) || qp.block < 32 || qp.block > 256) {
    set_error("qdot_cg_batched: " + (why.empty() ? std::string("block must be a power of two in [32, 256]") : why));
    return QDOT_ERR_ARG;
  }
  if (check_csr(A, "qdot_cg_batched") != QDOT_OK) return QDOT_ERR_ARG;
  if (!row_off_host || count <= 0 || row_off_host[0] != 0 || row_off_host[count] != A->n || !b || !x || !infos ||
      max_it < 0 || !(rel_tol >= 0.0)) {
    set_error("qdot_cg_batched: need count > 0 host row offsets from 0 to A->n, device b, x, infos, max_it >= 0 "
              "and rel_tol >= 0");
    return QDOT_ERR_ARG;
  }
  for (int s = 0; s < count; ++s)
    if (row_off_host[s + 1] < row_off_host[s]) {
      set_error("qdot_cg_batched: row offsets must not decrease");
      return QDOT_ERR_ARG;
    }
  const BatchLayoutCg l = batch_cg_layout(row_off_host, count, &qp);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < l.total) {
    set_error("qdot_cg_batched: workspace missing, misaligned or smaller than qdot_cg_batched_workspace_size()");
    return QDOT_ERR_WORKSPACE;
  }
  char* w = static_cast<char*>(ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  auto* sys = reinterpret_cast<BatchSys*>(w + l.off_sys);
  auto* res = reinterpret_cast<qdot_result*>(w + l.off_res);  // [0, count) p.q, [count, 2 count) r.r, then b.b
  qdot_result* res_pq = res;
  qdot_result* res_rr = res + count;
  qdot_result* res_bb = res + 2 * count;
  auto* ns_dot = reinterpret_cast<long long*>(w + l.off_nsd);
  auto* ns_full = reinterpret_cast<long long*>(w + l.off_nsf);
  auto* d_off = reinterpret_cast<long long*>(w + l.off_off);
  auto* d_poff = reinterpret_cast<long long*>(w + l.off_poff);
  auto* d_tiles = reinterpret_cast<RowTile*>(w + l.off_tiles);
  auto* d_tstart = reinterpret_cast<long long*>(w + l.off_tstart);
  auto* d_part = reinterpret_cast<double*>(w + l.off_part);
  auto* d_ptr = reinterpret_cast<const double**>(w + l.off_ptr);  // p, q, r, b-copy slices
  auto* flags = reinterpret_cast<int*>(w + l.off_flags);            // remaining, all_done, bad
  double* r = reinterpret_cast<double*>(w + l.off_vec);
  double* pv = r + l.total_pad;
  double* q = pv + l.total_pad;
  double* bp = q + l.total_pad;
  void* qws = w + l.off_qws;
  // host-built tables, copied once
  std::vector<long long> h_off(count + 1), h_poff(count + 1), h_tstart(count + 1), h_ns(count);
  std::vector<RowTile> h_tiles;
  h_tiles.reserve((size_t)l.ntiles);
  std::vector<const double*> h_ptr(4 * (size_t)count);
  long long pad = 0;
  for (int s = 0; s < count; ++s) {
    const long long m = row_off_host[s + 1] - row_off_host[s];
    h_off[s] = row_off_host[s];
    h_poff[s] = pad;
    h_ns[s] = m;
    h_tstart[s] = (long long)h_tiles.size();
    for (long long t0 = 0; t0 < m; t0 += kTileRows)
      h_tiles.push_back(RowTile{s, (int)std::min<long long>(kTileRows, m - t0), row_off_host[s] + t0});
    h_ptr[s] = pv + pad;
    h_ptr[count + s] = q + pad;
    h_ptr[2 * count + s] = r + pad;
    h_ptr[3 * count + s] = bp + pad;
    pad += (m + 1) & ~1ll;
  }
  h_off[count] = row_off_host[count];
  h_poff[count] = pad;
  h_tstart[count] = (long long)h_tiles.size();
  cudaError_t e;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  };
  if ((e = up(d_off, h_off.data(), sizeof(long long) * (count + 1))) != cudaSuccess ||
      (e = up(d_poff, h_poff.data(), sizeof(long long) * (count + 1))) != cudaSuccess ||
      (e = up(d_tstart, h_tstart.data(), sizeof(long long) * (count + 1))) != cudaSuccess ||
      (e = up(d_tiles, h_tiles.data(), sizeof(RowTile) * h_tiles.size())) != cudaSuccess ||
      (e = up(d_ptr, h_ptr.data(), sizeof(double*) * h_ptr.size())) != cudaSuccess ||
      (e = up(ns_dot, h_ns.data(), sizeof(long long) * count)) != cudaSuccess ||
      (e = up(ns_full, h_ns.data(), sizeof(long long) * count)) != cudaSuccess ||
      (e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), st)) != cudaSuccess ||
      (e = cudaMemsetAsync(res, 0, 3 * sizeof(qdot_result) * count, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(r, 0, 4 * sizeof(double) * (size_t)l.total_pad, st)) != cudaSuccess)
    return fail("qdot_cg_batched: setup", e);
  // the host tables must outlive the copies
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail("qdot_cg_batched: setup", e);

  const BatchView v = {d_off, d_poff, d_tiles, l.ntiles, count};
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int tgrid = (int)std::max<long long>(1, std::min<long long>(l.ntiles, (long long)sms * 8));
  const int sgrid = (count + 255) / 256;
  const long long* rowptr = reinterpret_cast<const long long*>(A->rowptr);
  const qdot_params exact = {1e-300, 32, 1, 0, QDOT_PATH_AUTO};
  const double* const* P = d_ptr;
  const double* const* Q = d_ptr + count;
  const double* const* R = d_ptr + 2 * count;
  const double* const* BP = d_ptr + 3 * count;
  auto dots = [&](const double* const* xs, const double* const* ys, const double* xa, const double* ya,
                  const long long* ns, const qdot_params* prm, bool use_plain, qdot_result* out,
                  cudaStream_t cs) -> cudaError_t {
    if (use_plain) {
      k_bcg_dot_tiles<<<tgrid, kTileRows, 0, cs>>>(v, xa, ya, d_part, ns);
      k_bcg_dot_final<<<(count + 7) / 8, 256, 0, cs>>>(d_part, d_tstart, count, out);
      return cudaGetLastError();
    }
    return launch_qdot_batched(xs, ys, ns, count, prm, out, 0, qws, l.qws_bytes, cs);
  };
  // r0 = b - A x0, p0 = r0, c0 = r0.r0, ||b|| (double class)
  k_bcg_spmv<<<tgrid, kTileRows, 0, st>>>(rowptr, A->col, A->val, v, x, 0, q, nullptr, flags + 2);
  k_bcg_init_vectors<<<tgrid, kTileRows, 0, st>>>(v, b, q, r, pv, bp);
  if ((e = dots(R, R, r, r, ns_dot, &qp, plain, res_rr, st)) != cudaSuccess) return fail("qdot_cg_batched", e);
  if ((e = dots(BP, BP, bp, bp, ns_full, &exact, false, res_bb, st)) != cudaSuccess)
    return fail("qdot_cg_batched", e);
  k_bcg_init_state<<<sgrid, 256, 0, st>>>(sys, res_rr, res_bb, ns_dot, count, rel_tol, max_it, flags);
  k_bcg_all_done<<<1, 1, 0, st>>>(flags, flags + 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_cg_batched", e);
  auto body = [&](cudaStream_t cs) -> cudaError_t {
    k_bcg_spmv<<<tgrid, kTileRows, 0, cs>>>(rowptr, A->col, A->val, v, pv, 1, q, sys, flags + 2);
    cudaError_t ee = dots(P, Q, pv, q, ns_dot, &qp, plain, res_pq, cs);
    if (ee != cudaSuccess) return ee;
    k_bcg_alpha<<<sgrid, 256, 0, cs>>>(sys, res_pq, count);
    k_bcg_update<<<tgrid, kTileRows, 0, cs>>>(v, x, r, pv, q, sys);
    ee = dots(R, R, r, r, ns_dot, &qp, plain, res_rr, cs);
    if (ee != cudaSuccess) return ee;
    k_bcg_beta<<<sgrid, 256, 0, cs>>>(sys, res_rr, count, rel_tol, max_it, ns_dot, flags);
    k_bcg_p<<<tgrid, kTileRows, 0, cs>>>(v, pv, r, sys);
    k_bcg_all_done<<<1, 1, 0, cs>>>(flags, flags + 1);
    return cudaGetLastError();
  };
  cudaGraphExec_t exec = nullptr;
  if ((e = record_graph(body, kIterPerGraph, &exec)) != cudaSuccess) return fail("qdot_cg_batched: graph", e);
  e = run_until_done(exec, flags + 1, max_it / kIterPerGraph + 2, st);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail("qdot_cg_batched", e);
  // true residuals ||b - A x|| / ||b|| (double class)
  k_bcg_spmv<<<tgrid, kTileRows, 0, st>>>(rowptr, A->col, A->val, v, x, 0, q, nullptr, flags + 2);
  k_bcg_residual<<<tgrid, kTileRows, 0, st>>>(v, bp, q, r);
  if ((e = dots(R, R, r, r, ns_full, &exact, false, res_pq, st)) != cudaSuccess) return fail("qdot_cg_batched", e);
  k_bcg_finish<<<sgrid, 256, 0, st>>>(sys, res_pq, count, rel_tol, flags + 2, infos);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_cg_batched", e);
  return QDOT_OK;
}

}  // extern "C"
