// C ABI of libqdot.so: argument checks, workspace planning, path choice.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {

static thread_local std::string g_error;
static thread_local cudaEvent_t g_ev_begin = nullptr, g_ev_end = nullptr;
void set_error(const std::string& msg) { g_error = msg; }
void clear_error() { g_error.clear(); }
void kernel_events(cudaEvent_t* begin, cudaEvent_t* end) {
  *begin = g_ev_begin;
  *end = g_ev_end;
}

const DeviceInfo& device_info() {
  static std::mutex mu;
  static DeviceInfo cache[64];
  static bool filled[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    static DeviceInfo none;
    return none;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!filled[dev]) {
    DeviceInfo di;
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) di.sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess)
      di.max_smem_optin = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) == cudaSuccess) di.l2_bytes = (size_t)v;
    cudaGetLastError();
    cache[dev] = di;
    filled[dev] = true;
  }
  return cache[dev];
}

bool valid_params(int64_t n, const qdot_params* p, std::string* why) {
  if (!p) {
    *why = "params pointer is NULL";
    return false;
  }
  if (n < 0) {
    *why = "n must be >= 0";
    return false;
  }
  if (!(p->eps > 0.0) || !std::isfinite(p->eps)) {
    *why = "eps must be a finite number > 0";
    return false;
  }
  if (p->block < 0 || p->block > (1 << 20) || (p->block & (p->block - 1)) != 0) {
    *why = "block must be 0 (exact binning) or a power of two in [1, 2^20]";
    return false;
  }
  if (p->split_budget != 0 && p->split_budget != 1) {
    *why = "split_budget must be 0 or 1";
    return false;
  }
  if (p->mant_reading != 0 && p->mant_reading != 1) {
    *why = "mant_reading must be 0 or 1";
    return false;
  }
  if (p->path < QDOT_PATH_AUTO || p->path > QDOT_PATH_FUSED || p->path == QDOT_PATH_FP64_DOT) {
    *why = "path must be QDOT_PATH_AUTO, QDOT_PATH_TWO_PASS, QDOT_PATH_ONE_PASS or QDOT_PATH_FUSED";
    return false;
  }
  return true;
}

static bool aligned16(const void* a, const void* b) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15u) == 0;
}

}  // namespace qd

using namespace qd;

namespace {

enum PathChoice { kTwoPass, kOnePass, kFused };

// Smallest n for which QDOT_PATH_AUTO takes the one-pass path with blocks of
// one component.
constexpr int64_t kOnePassMinN1 = 1ll << 24;

PathChoice choose_path(int64_t n, const qdot_params* p, bool al16) {
  if (p->path == QDOT_PATH_TWO_PASS) return kTwoPass;
  bool one = one_pass_supported(n, p, al16);
  if (p->path == QDOT_PATH_ONE_PASS) return one ? kOnePass : kTwoPass;
  // blocks of one component: one pass only where a warp has enough items
  // for its bound of e_max to settle early (otherwise most items are read
  // twice anyway)
  if (p->block == 1 && n < kOnePassMinN1) one = false;
  const bool fused = fused_supported(n, p, al16);
  if (p->path == QDOT_PATH_FUSED) return fused ? kFused : (one ? kOnePass : kTwoPass);
  // exact binning and blocks of one: the fused launch reads HBM once, but its
  // grid barriers cost more than the two-pass path's second read, which L2
  // serves at these sizes (measured per call in CUDA graphs, n = 2^16 .. 2^22:
  // 13.5 / 28 / 45 us fused against 13.7 / 23 / 33 us two-pass for blocks of
  // one; 20 / 36 / 53 against 17 / 27 / 37 for exact binning), so AUTO keeps
  // the two passes there and QDOT_PATH_FUSED selects the fused launch
  if (p->block <= 1) return one ? kOnePass : kTwoPass;
  return fused ? kFused : (one ? kOnePass : kTwoPass);
}

size_t workspace_for(int64_t n, const qdot_params* p, bool al16, PathChoice* choice) {
  PathChoice c = choose_path(n, p, al16);
  if (choice) *choice = c;
  if (c == kFused) return fused_ws_bytes(p);
  if (c == kOnePass) return plan_one_pass(n, p).total;
  return plan_two_pass(n, p, al16).total;
}

qdot_status check_common(const double* x, const double* y, int64_t n, const qdot_params* p, const void* out,
                         const void* ws) {
  std::string why;
  if (!valid_params(n, p, &why)) {
    set_error("qdot: " + why);
    return QDOT_ERR_ARG;
  }
  if (n > 0 && (!x || !y)) {
    set_error("qdot: x and y must be non-NULL when n > 0");
    return QDOT_ERR_ARG;
  }
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 7u) != 0) {
    set_error("qdot: x and y must be 8-byte aligned");
    return QDOT_ERR_ARG;
  }
  if (!out) {
    set_error("qdot: out must be a device pointer to a qdot_result");
    return QDOT_ERR_ARG;
  }
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    set_error("qdot: workspace must be non-NULL and 256-byte aligned");
    return QDOT_ERR_WORKSPACE;
  }
  return QDOT_OK;
}

qdot_status cuda_fail(const char* what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return QDOT_ERR_CUDA;
}

// Device address of a page-locked host buffer mapped into the device's
// address space, or NULL (pageable or unknown memory, or any error).
const double* mapped_host_pointer(const double* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error state of the query
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<const double*>(a.devicePointer);
}

// Streams and events for the host-to-device copies of qdot_from_host, one
// set per device, created on first use and kept for the process.
constexpr int kCopyStreams = 4;
struct CopyStreams {
  cudaStream_t s[kCopyStreams];
  cudaEvent_t start, done[kCopyStreams];
};

CopyStreams* copy_streams(cudaError_t* err) {
  static std::mutex mu;
  static CopyStreams* sets[64] = {nullptr};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!sets[dev]) {
    auto* c = new CopyStreams();
    for (int i = 0; i < kCopyStreams && *err == cudaSuccess; ++i) {
      *err = cudaStreamCreateWithFlags(&c->s[i], cudaStreamNonBlocking);
      if (*err == cudaSuccess) *err = cudaEventCreateWithFlags(&c->done[i], cudaEventDisableTiming);
    }
    if (*err == cudaSuccess) *err = cudaEventCreateWithFlags(&c->start, cudaEventDisableTiming);
    if (*err != cudaSuccess) return nullptr;
    sets[dev] = c;
  }
  return sets[dev];
}

}  // namespace

namespace qd {
size_t qdot_ws_bytes(int64_t n, const qdot_params* p) {
  return std::max(workspace_for(n, p, true, nullptr), workspace_for(n, p, false, nullptr));
}
cudaError_t launch_qdot_auto(const double* x, const double* y, int64_t n, const qdot_params* p, void* ws,
                             qdot_result* out, cudaStream_t st) {
  const bool al16 = aligned16(x, y);
  PathChoice c = choose_path(n, p, al16);
  if (c == kFused) return launch_fused(x, y, n, p, ws, out, nullptr, st);
  if (c == kOnePass) return launch_one_pass(x, y, n, p, plan_one_pass(n, p), ws, out, nullptr, st);
  return launch_two_pass(x, y, n, p, plan_two_pass(n, p, al16), ws, out, nullptr, nullptr, nullptr, nullptr, st);
}
}  // namespace qd

extern "C" {

size_t qdot_workspace_size(int64_t n, const qdot_params* p) {
  std::string why;
  if (!valid_params(n, p, &why)) return 0;
  // Size for the larger of the two alignment cases so any pointer fits.
  return std::max(workspace_for(n, p, true, nullptr), workspace_for(n, p, false, nullptr));
}

qdot_status qdot(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                 qdot_selection* sel, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  qdot_status s = check_common(x, y, n, p, out, ws);
  if (s != QDOT_OK) return s;
  const bool al16 = aligned16(x, y);
  PathChoice c;
  size_t need = workspace_for(n, p, al16, &c);
  if (ws_bytes < need) {
    set_error("qdot: workspace too small (" + std::to_string(ws_bytes) + " < " + std::to_string(need) + ")");
    return QDOT_ERR_WORKSPACE;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (c == kFused)
    e = launch_fused(x, y, n, p, ws, out, sel, st);
  else if (c == kOnePass)
    e = launch_one_pass(x, y, n, p, plan_one_pass(n, p), ws, out, sel, st);
  else
    e = launch_two_pass(x, y, n, p, plan_two_pass(n, p, al16), ws, out, sel, nullptr, nullptr, nullptr, st);
  if (e != cudaSuccess) return cuda_fail("qdot launch", e);
  return QDOT_OK;
}

qdot_status qdot_explain(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                         uint8_t* cls, double* qx, double* qy, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  qdot_status s = check_common(x, y, n, p, out, ws);
  if (s != QDOT_OK) return s;
  const bool al16 = aligned16(x, y);
  TwoPassPlan pl = plan_two_pass(n, p, al16);
  if (ws_bytes < pl.total) {
    set_error("qdot_explain: workspace too small (" + std::to_string(ws_bytes) + " < " + std::to_string(pl.total) +
              ")");
    return QDOT_ERR_WORKSPACE;
  }
  // The explain kernel writes every valid component; a NULL output is skipped.
  cudaError_t e = launch_two_pass(x, y, n, p, pl, ws, out, nullptr, cls, qx, qy, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail("qdot_explain launch", e);
  return QDOT_OK;
}

int64_t qdot_trace_units(int64_t n, const qdot_params* p, int32_t al16, int32_t* unit_components) {
  std::string why;
  if (unit_components) *unit_components = 0;
  if (!valid_params(n, p, &why)) return 0;
  const PathChoice c = choose_path(n, p, al16 != 0);
  if (c == kTwoPass) return 0;
  // item units: the one-pass item records, and the fused kernel for exact
  // binning and blocks of one
  const bool items = (c == kOnePass && plan_one_pass(n, p).items) || (c == kFused && p->block <= 1);
  const int64_t per = items ? 256 : p->block;
  if (unit_components) *unit_components = (int32_t)per;
  return (n + per - 1) / per;
}

qdot_status qdot_trace(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                       qdot_trace_unit* units, int64_t units_len, uint8_t* cls, void* ws, size_t ws_bytes,
                       void* stream) {
  clear_error();
  qdot_status s = check_common(x, y, n, p, out, ws);
  if (s != QDOT_OK) return s;
  const bool al16 = aligned16(x, y);
  PathChoice c;
  const size_t need = workspace_for(n, p, al16, &c);
  if (ws_bytes < need) {
    set_error("qdot_trace: workspace too small (" + std::to_string(ws_bytes) + " < " + std::to_string(need) + ")");
    return QDOT_ERR_WORKSPACE;
  }
  if (c == kTwoPass) {
    set_error("qdot_trace: these arguments take the two-pass path; its per-component view is qdot_explain");
    return QDOT_ERR_ARG;
  }
  const int64_t need_units = qdot_trace_units(n, p, al16 ? 1 : 0, nullptr);
  if (n > 0 && (!units || units_len < need_units)) {
    set_error("qdot_trace: units must hold " + std::to_string(need_units) + " records");
    return QDOT_ERR_ARG;
  }
  TraceOut tr;
  tr.units = units;
  tr.cls = cls;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaError_t e = c == kFused ? launch_fused(x, y, n, p, ws, out, nullptr, st, tr)
                                    : launch_one_pass(x, y, n, p, plan_one_pass(n, p), ws, out, nullptr, st, tr);
  if (e != cudaSuccess) return cuda_fail("qdot_trace launch", e);
  return QDOT_OK;
}

size_t qdot_dot_fp64_workspace_size(void) { return dot_fp64_workspace(); }

qdot_status qdot_dot_fp64(const double* x, const double* y, int64_t n, double* out, void* ws, size_t ws_bytes,
                          void* stream) {
  clear_error();
  if (n < 0 || (n > 0 && (!x || !y)) || !out) {
    set_error("qdot_dot_fp64: invalid arguments");
    return QDOT_ERR_ARG;
  }
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 7u) != 0) {
    set_error("qdot_dot_fp64: x and y must be 8-byte aligned");
    return QDOT_ERR_ARG;
  }
  if (!ws || ws_bytes < dot_fp64_workspace() || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) {
    set_error("qdot_dot_fp64: workspace missing, misaligned or too small");
    return QDOT_ERR_WORKSPACE;
  }
  cudaError_t e = launch_dot_fp64(x, y, n, out, ws, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail("qdot_dot_fp64 launch", e);
  return QDOT_OK;
}

qdot_status qdot_from_host(const double* x_host, const double* y_host, int64_t n, const qdot_params* p,
                           qdot_result* out_host, double* x_dev, double* y_dev, qdot_result* out_dev, void* ws,
                           size_t ws_bytes, void* stream) {
  clear_error();
  if (n > 0 && (!x_host || !y_host)) {
    set_error("qdot_from_host: host buffers must be non-NULL when n > 0");
    return QDOT_ERR_ARG;
  }
  if (!out_host) {
    set_error("qdot_from_host: out_host must be non-NULL");
    return QDOT_ERR_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (n > 0) {
    // Page-locked host buffers are read in place by the kernels, over the
    // host link, in the same single pass (no staging copy).
    const double* xd = mapped_host_pointer(x_host);
    const double* yd = mapped_host_pointer(y_host);
    if (xd && yd) {
      qdot_status s = qdot(xd, yd, n, p, out_dev, nullptr, ws, ws_bytes, stream);
      if (s != QDOT_OK) return s;
      e = cudaMemcpyAsync(out_host, out_dev, sizeof(qdot_result), cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return cuda_fail("qdot_from_host: copy of the result", e);
      e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail("qdot_from_host: synchronize", e);
      return QDOT_OK;
    }
    // Otherwise the two vectors go up in chunks spread over the library's copy streams
    // (several copy engines in flight), ordered after the caller's stream.
    CopyStreams* cs = copy_streams(&e);
    if (!cs) return cuda_fail("qdot_from_host: copy streams", e);
    if ((e = cudaEventRecord(cs->start, st)) != cudaSuccess) return cuda_fail("qdot_from_host: event", e);
    const size_t bytes = sizeof(double) * (size_t)n;
    const size_t chunk = std::max<size_t>(bytes / (2 * kCopyStreams), 1u << 20);
    int k = 0;
    for (int v = 0; v < 2; ++v) {
      const char* src = reinterpret_cast<const char*>(v ? y_host : x_host);
      char* dst = reinterpret_cast<char*>(v ? y_dev : x_dev);
      for (size_t off = 0; off < bytes; off += chunk, ++k) {
        cudaStream_t cst = cs->s[k % kCopyStreams];
        if (k < kCopyStreams && (e = cudaStreamWaitEvent(cst, cs->start, 0)) != cudaSuccess)
          return cuda_fail("qdot_from_host: wait", e);
        e = cudaMemcpyAsync(dst + off, src + off, std::min(chunk, bytes - off), cudaMemcpyHostToDevice, cst);
        if (e != cudaSuccess) return cuda_fail("qdot_from_host: copy of x / y", e);
      }
    }
    for (int i = 0; i < std::min(k, kCopyStreams); ++i) {
      if ((e = cudaEventRecord(cs->done[i], cs->s[i])) != cudaSuccess ||
          (e = cudaStreamWaitEvent(st, cs->done[i], 0)) != cudaSuccess)
        return cuda_fail("qdot_from_host: join", e);
    }
  }
  qdot_status s = qdot(x_dev, y_dev, n, p, out_dev, nullptr, ws, ws_bytes, stream);
  if (s != QDOT_OK) return s;
  e = cudaMemcpyAsync(out_host, out_dev, sizeof(qdot_result), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail("qdot_from_host: copy of the result", e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail("qdot_from_host: synchronize", e);
  return QDOT_OK;
}

int32_t qdot_kernel_launches(int64_t n, const qdot_params* p, int32_t al16) {
  std::string why;
  if (!valid_params(n, p, &why)) return 0;
  PathChoice c = choose_path(n, p, al16 != 0);
  if (c == kFused) return 1;
  if (c == kOnePass) return one_pass_launches(n, p);
  return 4;  // stats, select, apply, final
}

int32_t qdot_select_path(int64_t n, const qdot_params* p, int32_t al16) {
  std::string why;
  if (!valid_params(n, p, &why)) return 0;
  const PathChoice c = choose_path(n, p, al16 != 0);
  return c == kFused ? QDOT_PATH_FUSED : (c == kOnePass ? QDOT_PATH_ONE_PASS : QDOT_PATH_TWO_PASS);
}

const char* qdot_stream_kernel(int64_t n, const qdot_params* p, int32_t al16) {
  std::string why;
  if (!valid_params(n, p, &why)) return "";
  const PathChoice c = choose_path(n, p, al16 != 0);
  if (c == kFused) return fused_stream_kernel(p);
  if (c == kOnePass) return one_pass_stream_kernel(n, p);
  return "k_apply_fast";
}

void qdot_set_kernel_events(void* begin, void* end) {
  g_ev_begin = (begin && end) ? static_cast<cudaEvent_t>(begin) : nullptr;
  g_ev_end = (begin && end) ? static_cast<cudaEvent_t>(end) : nullptr;
}

const char* qdot_last_error(void) { return g_error.c_str(); }

const char* qdot_version(void) { return "qdot-gb300 0.1 (sm_103a)"; }

}  // extern "C"
