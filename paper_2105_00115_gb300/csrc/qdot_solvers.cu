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
cudaError_t run_until_done(cudaGraphExec_t exec, const SolverState* st, int max_replays, cudaStream_t stream) {
  for (int r = 0; r < max_replays; ++r) {
    cudaError_t e = cudaGraphLaunch(exec, stream);
    if (e != cudaSuccess) return e;
    int done = 0;
    e = cudaMemcpyAsync(&done, &st->done, sizeof(int), cudaMemcpyDeviceToHost, stream);
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
  e = run_until_done(exec, st, max_it / kIterPerGraph + 2, s);
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
  e = run_until_done(exec, st, iters / kIterPerGraph + 2, s);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail("qdot_power", e);
  k_pm_finish<<<1, 1, 0, s>>>(st, info);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail("qdot_power", e);
  return QDOT_OK;
}

}  // extern "C"
