// qdot for callers that cannot hand the library a workspace.
//
// Some callers have no way to allocate device memory: code that runs inside a
// host application which owns the whole device allocator (all memory reserved
// up front by a framework, a memory pool with no free slot, a plug-in API that
// only passes tensors in and out), or deployments that forbid allocation after
// start-up.  For them qdot_static_scratch() runs the two-pass path on a
// scratch array that lives in the library itself, a file-scope __device__
// array of QDOT_STATIC_SCRATCH_BYTES.  Every GPU that loads the library holds
// that array until the process exits.
#include <mutex>
#include <string>

#include "qdot_common.cuh"
#include "qdot_internal.h"

namespace qd {
namespace {

constexpr size_t kStaticScratchBytes = QDOT_STATIC_SCRATCH_BYTES;

// The scratch itself.  In host code this name only stands for the symbol; its
// device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Identity of the calling thread's current CUDA context (0 if there is none
// or the driver cannot tell), through driver entry points the runtime hands
// out, so the library needs no link to the driver library.  The runtime
// destroys a device's context on cudaDeviceReset() and makes a new one on
// the next call; the array's address is only valid in the context it was
// looked up in.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
    cudaGetLastError();
  });
  if (!get_current || !get_id) return 0;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return 0;
  unsigned long long id = 0;
  return get_id(ctx, &id) == 0 ? id : 0;
}

// Device address of g_static_scratch on the current device, looked up with
// that device current and cached per device together with the context it
// belongs to: a call in another context (after a device reset) looks it up
// again.
cudaError_t static_scratch_address(void** out) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  static unsigned long long ctx_of[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long ctx = current_context_id();
  if (!addr[dev] || ctx == 0 || ctx != ctx_of[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    addr[dev] = p;
    ctx_of[dev] = current_context_id();  // the context the lookup ran in
  }
  *out = addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace qd

using namespace qd;

extern "C" qdot_status qdot_static_scratch(const double* x, const double* y, int64_t n, const qdot_params* p,
                                           qdot_result* out, void* stream) {
  clear_error();
  std::string why;
  if (!valid_params(n, p, &why)) {
    set_error("qdot_static_scratch: " + why);
    return QDOT_ERR_ARG;
  }
  if (n > 0 && (!x || !y)) {
    set_error("qdot_static_scratch: x and y must be non-NULL when n > 0");
    return QDOT_ERR_ARG;
  }
  if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 7u) != 0) {
    set_error("qdot_static_scratch: x and y must be 8-byte aligned");
    return QDOT_ERR_ARG;
  }
  if (!out) {
    set_error("qdot_static_scratch: out must be a device pointer to a qdot_result");
    return QDOT_ERR_ARG;
  }
  const bool al16 = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15u) == 0;
  const TwoPassPlan plan = plan_two_pass(n, p, al16);
  if (plan.total > kStaticScratchBytes) {
    set_error("qdot_static_scratch: these arguments need " + std::to_string(plan.total) +
              " bytes of scratch, more than the library's fixed " + std::to_string(kStaticScratchBytes) +
              " (blocks of more than 64 components, or of more than 32 with 8-byte aligned x, y, keep 2 bytes "
              "per block); use qdot() with a workspace instead");
    return QDOT_ERR_WORKSPACE;
  }
  void* ws = nullptr;
  cudaError_t e = static_scratch_address(&ws);
  if (e != cudaSuccess) {
    set_error(std::string("qdot_static_scratch: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return QDOT_ERR_CUDA;
  }
  // The two-pass sequence rewrites every scratch word it later reads (the
  // exact-binning histogram is cleared by a memset at its start), so a call
  // never depends on what an earlier call left in the array.
  e = launch_two_pass(x, y, n, p, plan, ws, out, nullptr, nullptr, nullptr, nullptr,
                      static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) {
    set_error(std::string("qdot_static_scratch launch: ") + cudaGetErrorString(e));
    return QDOT_ERR_CUDA;
  }
  return QDOT_OK;
}
