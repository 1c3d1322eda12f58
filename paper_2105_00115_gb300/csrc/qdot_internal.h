// Host-side plumbing shared by the translation units of libqdot.so.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "qdot.h"

namespace qd {

// Thread-local error message behind qdot_last_error().
void set_error(const std::string& msg);
void clear_error();

// Events of qdot_set_kernel_events() for the calling thread (may be null).
void kernel_events(cudaEvent_t* begin, cudaEvent_t* end);

// Device facts cached per device ordinal.
struct DeviceInfo {
  int sms = 0;
  int max_smem_optin = 0;
  size_t l2_bytes = 0;
};
const DeviceInfo& device_info();

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Optional check outputs of qdot_trace(); both null on the timed path.
struct TraceOut {
  qdot_trace_unit* units = nullptr;  // per block or per item
  uint8_t* cls = nullptr;            // per component (item paths)
};

// Execution modes of the two-pass path.
enum Mode { kModeExact = 0, kModeBlock1 = 1, kModeBlockSmall = 2, kModeBlockLarge = 3 };

// Workspace plan of the two-pass path for one call.
struct TwoPassPlan {
  int mode = 0;
  int vec = 2;          // 2: 128-bit loads (16-byte aligned x, y), 1: 64-bit loads
  int log2b = 0;        // log2(block) for block >= 1
  int grid_stats = 0;
  int grid_apply = 0;
  long long nblocks = 0;
  size_t off_sel = 0, off_hdr = 0, off_stats = 0, off_apply = 0, off_hist = 0, off_keys = 0;
  size_t total = 0;
};

bool valid_params(int64_t n, const qdot_params* p, std::string* why);
TwoPassPlan plan_two_pass(int64_t n, const qdot_params* p, bool aligned16);

// Launch the two-pass sequence (stats -> select -> apply [or explain] ->
// final).  Returns cudaSuccess or the first launch error.
cudaError_t launch_two_pass(const double* x, const double* y, int64_t n, const qdot_params* p,
                            const TwoPassPlan& plan, void* ws, qdot_result* out, qdot_selection* sel,
                            uint8_t* cls, double* qx, double* qy, cudaStream_t stream);

// One-pass (deferred selection) path for 32 <= block <= 256.
struct OnePassPlan {
  int log2b = 0;
  int grid = 0;
  int window = 0;         // keys kept per record
  long long units = 0;    // work units (each produces one record)
  long long unit_blocks = 0;
  bool items = false;  // item records (one per 256 components) instead of block records
  size_t off_sel = 0, off_hdr = 0, off_rec = 0, off_misc = 0, off_slot1 = 0, off_meta = 0, off_slot3 = 0;
  size_t off_rec2 = 0;
  size_t rec_bytes = 0;
  size_t total = 0;
};
bool one_pass_supported(int64_t n, const qdot_params* p, bool aligned16);
OnePassPlan plan_one_pass(int64_t n, const qdot_params* p);
const char* one_pass_stream_kernel(int64_t n, const qdot_params* p);
int one_pass_launches(int64_t n, const qdot_params* p);
cudaError_t launch_one_pass(const double* x, const double* y, int64_t n, const qdot_params* p,
                            const OnePassPlan& plan, void* ws, qdot_result* out, qdot_selection* sel,
                            cudaStream_t stream, TraceOut trace = TraceOut());

// One-launch qdot for vectors the resident grid covers in a few items
// (cooperative launch with grid-wide barriers).
bool fused_supported(int64_t n, const qdot_params* p, bool aligned16);
size_t fused_ws_bytes(const qdot_params* p);
const char* fused_stream_kernel(const qdot_params* p);
cudaError_t launch_fused(const double* x, const double* y, int64_t n, const qdot_params* p, void* ws,
                         qdot_result* out, qdot_selection* sel, cudaStream_t stream, TraceOut trace = TraceOut());

// qdot() on device buffers with the path qdot() would choose (no checks);
// ws must hold qdot_workspace_size(n, p) bytes.
size_t qdot_ws_bytes(int64_t n, const qdot_params* p);
cudaError_t launch_qdot_auto(const double* x, const double* y, int64_t n, const qdot_params* p, void* ws,
                             qdot_result* out, cudaStream_t stream);

// Batched qdot on device arrays (no argument checks; 32 <= p->block <= 256).
size_t batched_ws_bytes(const int64_t* ns_host, int count, const qdot_params* p);
cudaError_t launch_qdot_batched(const double* const* xs, const double* const* ys, const long long* ns, int count,
                                const qdot_params* p, qdot_result* outs, int grid_ctas, void* ws, size_t ws_bytes,
                                cudaStream_t stream, const qdot_batched_tuning* tuning = nullptr);

// Plain FP64 dot.
cudaError_t launch_dot_fp64(const double* x, const double* y, int64_t n, double* out, void* ws,
                            cudaStream_t stream);
size_t dot_fp64_workspace();

}  // namespace qd
