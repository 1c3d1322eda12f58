/*
 * qdot -- error-bounded quantized dot product on one NVIDIA GB300 (sm_103a).
 *
 * C ABI of libqdot.so.  Every entry point takes plain pointers and sizes; the
 * caller owns all memory (device buffers, workspace, streams) and the library
 * allocates nothing on any path below.  Device results are written to device
 * memory, asynchronously on the caller's stream, so calls can be recorded in
 * CUDA graphs; a host wrapper copies them back when it needs them.
 *
 * The method is that of Diffenderfer, Osei-Kuffuor and Menon, "Qdot:
 * Quantized Dot Product Kernel for Approximate High Performance Computing"
 * (arXiv 2105.00115): Algorithm 2 (parameter selection: exponent keys, bins,
 * bin scores eq. bin-score-def, precisions eq. precision-def) followed by
 * Algorithm 1 (computation phase), i.e. Algorithm 3.
 *
 * Definitions used throughout (the paper's notation):
 *   e(v)      unbiased IEEE exponent of a finite nonzero double v (floor(log2|v|),
 *             subnormals with their true exponent) -- Sec. 1.1 flexp.
 *   e_i       e(x_i) + e(y_i), the key of component i -- Algorithm 2, exponent
 *             preprocessing.  Components with x_i == 0 or y_i == 0 are class ZERO:
 *             they belong to no bin and contribute exactly 0.
 *   bins      block == 0: exact binning, one bin per distinct key (Sec. 3.2);
 *             block == B: the non-ZERO components of each index block
 *             [bB, (b+1)B), u_b = max key, M_b = count (Sec. 5, the blocked approach of the conclusion).
 *   f         floor(log2(eps / N_bins)) (split_budget = 1, Sec. 4.1) or
 *             floor(log2 eps) (split_budget = 0), computed exactly.
 *   sigma_k   ceil(log2 M_k) + u_k - e_max - f + 1 (eq. bin-score-def).
 *   class     sigma < 0: PERF; < m_half: HALF; < m_single: SINGLE; else DOUBLE
 *             (eq. precision-def; m_half, m_single = 10, 23, or 11, 24 when
 *             mant_reading = 1).
 *   q(v)      v with its significand rounded to 11 (HALF) or 24 (SINGLE) bits,
 *             ties to even, exponent unbounded (Sec. 3.2 scale / cast / rescale);
 *             q(v) = v for DOUBLE, 0 for PERF and ZERO.
 *   z         sum_i q(x_i) q(y_i), evaluated with exact integer arithmetic and
 *             rounded once to the nearest double (exact up to a truncation of at
 *             most n 2^(e_max - L), L = min(104, 124 - ceil(log2 n)), plus, on the
 *             one-pass path, a relative 2^-45 per block; see qdot()).
 *
 * Errors: every entry point returns a qdot_status.  Argument errors are
 * detected on the host before anything is launched (nothing is written).  Data
 * errors found on the device (a NaN or Inf component) are reported in the
 * `status` field of the device result; the host call still returns QDOT_OK.
 * qdot_last_error() gives a message for the last failing call on this thread.
 */
#ifndef QDOT_H
#define QDOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QDOT_OK = 0,
  QDOT_ERR_ARG = 1,        /* invalid argument (checked on the host) */
  QDOT_ERR_NONFINITE = 2,  /* a component of x or y is NaN or Inf (device status) */
  QDOT_ERR_CUDA = 3,       /* a CUDA runtime call failed; see qdot_last_error() */
  QDOT_ERR_TIMEOUT = 4,    /* a bounded device wait expired (device status) */
  QDOT_ERR_WORKSPACE = 5,  /* workspace missing, misaligned or too small */
  QDOT_ERR_NOCONV = 6      /* an iterative solver hit its iteration cap */
} qdot_status;

enum { QDOT_PERF = 0, QDOT_HALF = 1, QDOT_SINGLE = 2, QDOT_DOUBLE = 3, QDOT_ZERO = 4 };

/* Key range: every e_i and every block key ceil(log2 M_b) + u_b lies in
 * [QDOT_KEY_MIN, QDOT_KEY_MIN + QDOT_KEY_COUNT). */
#define QDOT_KEY_MIN (-2148)
#define QDOT_KEY_COUNT 4224

/* Execution path for qdot(): chosen automatically unless forced. */
enum { QDOT_PATH_AUTO = 0, QDOT_PATH_TWO_PASS = 1, QDOT_PATH_ONE_PASS = 2,
       /* qdot_cg / qdot_power only: every dot product a plain FP64 dot (the
        * comparator); eps, block, split_budget and mant_reading are ignored */
       QDOT_PATH_FP64_DOT = 3,
       /* one cooperative launch (32 <= B <= 256, 16-byte aligned, n up to
        * 16 warps x 8 items x 256 per SM, about 5 million on a 152-SM GPU);
        * AUTO takes it when it applies */
       QDOT_PATH_FUSED = 4 };

typedef struct {
  double eps;           /* qdot tolerance eps > 0, finite (Algorithm 3 input) */
  int32_t block;        /* 0: exact binning; else B, a power of two in [1, 2^20] */
  int32_t split_budget; /* 1: eps / N_bins (default, Sec. 4.1); 0: eps (eq. bin-score-def) */
  int32_t mant_reading; /* 0: m_half, m_single = 10, 23 (default); 1: 11, 24 */
  int32_t path;         /* QDOT_PATH_*; the one-pass and fused paths need 32 <= B <= 256 */
} qdot_params;

/* Device-side result of one qdot (80 bytes). */
typedef struct {
  double value;     /* z */
  double bound;     /* a-priori absolute error bound N_bins 2^(e_max + f) (<= eps 2^e_max) */
  int64_t n_bins;   /* number of non-empty bins N_bins */
  int64_t count[5]; /* components per class PERF, HALF, SINGLE, DOUBLE, ZERO */
  int32_t e_max;    /* max key over non-ZERO components (0 if none) */
  int32_t e_min;    /* min key over non-ZERO components (0 if none) */
  int32_t f;        /* floor(log2 eps_eff) used in the scores */
  int32_t status;   /* QDOT_OK or QDOT_ERR_NONFINITE */
} qdot_result;

/* The parameter selection of one call (Algorithm 2 output), compact form:
 * the class of every key.  For block == 0 the key is e_i; for block == B it
 * is the block key ceil(log2 M_b) + u_b.  4272 bytes. */
typedef struct {
  int32_t e_max, e_min, f, status;
  int64_t n_bins;
  int32_t block, key_min;               /* key_min == QDOT_KEY_MIN */
  int32_t m_half, m_single;
  int32_t reserved[2];
  uint8_t cls[QDOT_KEY_COUNT];          /* class per key, index key - key_min */
} qdot_selection;

/* CSR matrix in device memory (rows sorted, int64 row pointers). */
typedef struct {
  int64_t n;              /* rows == columns */
  int64_t nnz;
  const int64_t* rowptr;  /* [n + 1] */
  const int32_t* col;     /* [nnz] */
  const double* val;      /* [nnz] */
} qdot_csr;

/* Device-side summary of a qdot_cg() run (64 bytes). */
typedef struct {
  int32_t iters;        /* CG iterations taken (k at exit) */
  int32_t status;       /* QDOT_OK, QDOT_ERR_NOCONV or QDOT_ERR_NONFINITE */
  double relres;        /* sqrt(c_k) / ||b||, the residual the algorithm holds */
  double true_relres;   /* ||b - A x|| / ||b|| recomputed at exit (exact dot) */
  int64_t counts[5];    /* components per class over every qdot of the run */
} qdot_cg_info;

/* Device-side summary of a qdot_power() run (56 bytes). */
typedef struct {
  int32_t iters;        /* iterations taken */
  int32_t status;       /* QDOT_OK or QDOT_ERR_NONFINITE */
  double lambda;        /* last eigenvalue estimate */
  int64_t counts[5];    /* components per class over every qdot of the run */
} qdot_power_info;

/* ------------------------------------------------------------------------ */

/* Bytes of device workspace qdot() / qdot_explain() need for n components
 * with parameters p (0 on invalid arguments).  The workspace is scratch: its
 * contents on entry are ignored and on exit undefined. */
size_t qdot_workspace_size(int64_t n, const qdot_params* p);

/* z = qdot(x, y, eps) -- Algorithm 3 of the paper.
 *   x, y     device pointers to n doubles (8-byte aligned; 16-byte alignment
 *            selects 128-bit loads).  May be NULL when n == 0.
 *   p        host pointer to the parameters (read during the call).
 *   out      device pointer to one qdot_result (written asynchronously).
 *   sel      optional device pointer to a qdot_selection receiving the
 *            parameter selection (for qdot_backward); NULL to skip.
 *   ws       device workspace of at least qdot_workspace_size(n, p) bytes,
 *            256-byte aligned.
 *   stream   cudaStream_t (NULL = legacy default stream).
 * Returns QDOT_ERR_ARG / QDOT_ERR_WORKSPACE on bad arguments (nothing is
 * launched), QDOT_ERR_CUDA if a launch fails, else QDOT_OK. */
qdot_status qdot(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                 qdot_selection* sel, void* ws, size_t ws_bytes, void* stream);

/* qdot() that also writes, per component i, its class (cls[i], uint8) and
 * the quantized values q(x_i), q(y_i) (0 for PERF and ZERO; a quantized value
 * that overflows double is written as +-Inf).  Any of cls, qx, qy may be
 * NULL.  Uses the two-pass path. */
qdot_status qdot_explain(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                         uint8_t* cls, double* qx, double* qy, void* ws, size_t ws_bytes, void* stream);

/* Batched qdot: `count` independent problems z_j = qdot(x_j, y_j, eps) of
 * uneven lengths n_j, blocked binning with 32 <= block <= 256, computed in
 * one persistent streaming launch (plus a planning and a per-problem
 * finishing kernel).  Each z_j is exactly what qdot() returns for that pair.
 *   xs, ys   device arrays of `count` device pointers (each 16-byte aligned,
 *            or the problem's status is QDOT_ERR_ARG).
 *   ns       device array of `count` lengths (int64, >= 0).
 *   outs     device array of `count` qdot_result.
 *   grid_ctas  CTAs of the streaming kernel (0 = three per SM); see also
 *            qdot_batched_tuned().
 *   ws       workspace of qdot_batched_workspace_size(ns_host, count, p)
 *            bytes, computed from the same lengths on the host; if it is too
 *            small every problem reports QDOT_ERR_WORKSPACE.
 * Nothing synchronises with the host, so the call can be recorded in a CUDA
 * graph and replayed. */
size_t qdot_batched_workspace_size(const int64_t* ns_host, int32_t count, const qdot_params* p);

/* Launch shape of the batched streaming kernel (the one persistent launch).
 * Every lane always handles 8 components of a warp item of 256 (the
 * block-to-lane mapping needs it); the tunable parts are the CTA size, how
 * many CTAs (and so how many warps split the concatenated items of all pairs)
 * and whether items are staged through shared memory. */
typedef struct {
  int32_t threads_per_cta;  /* 128 or 256 */
  int32_t ctas_per_sm;      /* grid = ctas_per_sm * SMs when grid_ctas == 0; 1..64 */
  int32_t grid_ctas;        /* explicit grid size, or 0 */
  int32_t staged;           /* 1: cp.async staging through shared memory; 0: register double buffering */
} qdot_batched_tuning;

/* qdot_batched() with an explicit launch shape (tuning == NULL: 256 threads,
 * 3 CTAs per SM, staged); grid_ctas > 0 overrides the tuning's grid. */
qdot_status qdot_batched_tuned(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                               const qdot_params* p, qdot_result* outs, const qdot_batched_tuning* tuning,
                               int32_t grid_ctas, void* ws, size_t ws_bytes, void* stream);
qdot_status qdot_batched(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                         const qdot_params* p, qdot_result* outs, int32_t grid_ctas, void* ws, size_t ws_bytes,
                         void* stream);

/* ACG, Algorithm 4 of the paper: conjugate gradients for an SPD matrix A with
 * both dot products per iteration (p.q and r.r) computed by qdot with
 * parameters p.  x holds x0 on entry and the iterate on exit.  The loop runs
 * while k < max_it and sqrt(c_k) / ||b|| > rel_tol, c_k = qdot(r_k, r_k)
 * (the residual norm the algorithm holds; ||b|| is computed exactly).
 * info (device) receives the summary; class_hist (device, optional) receives
 * per iteration k the class counts of qdot(p, q) at [10k, 10k + 5) and of
 * qdot(r, r) at [10k + 5, 10k + 10) (max_it * 10 int64).  The call
 * synchronises the stream once per 16 iterations to test convergence.
 * Workspace: qdot_cg_workspace_size(A->n, p). */
size_t qdot_cg_workspace_size(int64_t n, const qdot_params* p);
qdot_status qdot_cg(const qdot_csr* A, const double* b, double* x, double rel_tol, int32_t max_it,
                    const qdot_params* p, qdot_cg_info* info, int64_t* class_hist, void* ws, size_t ws_bytes,
                    void* stream);

/* Batched ACG: `count` independent SPD systems solved together, each by
 * Algorithm 4 with its own scalars and stopping test (as in qdot_cg).  A is
 * one block-diagonal CSR matrix: system s owns rows (and columns)
 * [row_off_host[s], row_off_host[s + 1]); a column outside its row's system
 * is not used and makes every info[s].status QDOT_ERR_ARG.  b, x: device
 * vectors of A->n doubles (x holds x0 on entry).  Each iteration is one SpMV
 * launch, one batched-qdot launch per dot product and one launch per vector
 * update over all systems; 16 iterations are replayed as one CUDA graph until
 * every system has stopped.  p->block must lie in [32, 256] (the batched
 * qdot); QDOT_PATH_FP64_DOT runs the plain-FP64-dot comparator.  infos:
 * device array of `count` qdot_cg_info.  row_off_host is read during the call
 * only.  Workspace: qdot_cg_batched_workspace_size(row_off_host, count, p). */
size_t qdot_cg_batched_workspace_size(const int64_t* row_off_host, int32_t count, const qdot_params* p);
qdot_status qdot_cg_batched(const qdot_csr* A, const int64_t* row_off_host, int32_t count, const double* b,
                            double* x, double rel_tol, int32_t max_it, const qdot_params* p, qdot_cg_info* infos,
                            void* ws, size_t ws_bytes, void* stream);

/* APM, Algorithm 5 of the paper, with the eigenvalue estimate read as the
 * Rayleigh quotient: for k = 0, 1, ...: w = A x_k; lambda_k = qdot(x_k, w);
 * c = qdot(w, w); x_{k+1} = w * (1 / sqrt(c)); stop after `iters` iterations
 * or, when tau > 0, once |lambda_k - lambda_{k-1}| <= tau.  x holds a unit
 * start vector on entry and the last iterate on exit.  class_hist as for
 * qdot_cg (x.w counts, then w.w counts).  Workspace:
 * qdot_power_workspace_size(A->n, p). */
size_t qdot_power_workspace_size(int64_t n, const qdot_params* p);
qdot_status qdot_power(const qdot_csr* A, double* x, int32_t iters, double tau, const qdot_params* p,
                       qdot_power_info* info, int64_t* class_hist, void* ws, size_t ws_bytes, void* stream);

/* Backward of z = qdot(x, y) with the forward's class map held fixed (the
 * classes of Algorithm 2, read straight-through): gx_i = g * q_c(y_i),
 * gy_i = g * q_c(x_i) for components of class HALF / SINGLE / DOUBLE, +0 for
 * PERF and ZERO.  The paper defines no derivative; this is the gradient of the
 * frozen-class surrogate sum_i q_c(x_i) q_c(y_i) with each quantizer's
 * derivative taken as 1.
 *   x, y, n, p  the forward's operands and parameters (device, unchanged).
 *   sel         device qdot_selection the forward qdot() wrote for them; each
 *               component's class is re-derived from it and x, y.
 *   g           device pointer to the upstream gradient dL/dz (one double).
 *   gx, gy      device outputs of n doubles; either may be NULL.
 * All device pointers 8-byte aligned (16 for 128-bit access).  Asynchronous;
 * nothing is allocated. */
qdot_status qdot_backward(const double* x, const double* y, int64_t n, const qdot_params* p,
                          const qdot_selection* sel, const double* g, double* gx, double* gy, void* stream);

/* Batched backward for qdot_batched() (blocked binning, 32 <= block <= 256):
 * problem j's classes come from its forward result outs[j] (e_max, f) and
 * x_j, y_j; gs[j] is dL/dz_j.  gxs / gys are device arrays of `count` device
 * output pointers (either array may be NULL).  A problem whose forward status
 * is not QDOT_OK gets NaN gradients.  Workspace:
 * qdot_batched_backward_workspace_size(count) bytes, 256-byte aligned.
 * grid_ctas: CTAs of the streaming kernel (0 = four per SM). */
size_t qdot_batched_backward_workspace_size(int32_t count);
qdot_status qdot_batched_backward(const double* const* xs, const double* const* ys, const int64_t* ns, int32_t count,
                                  const qdot_params* p, const qdot_result* outs, const double* gs, double* const* gxs,
                                  double* const* gys, int32_t grid_ctas, void* ws, size_t ws_bytes, void* stream);

/* Plain FP64 dot product x.y (the comparator of the paper's speedup metric,
 * eq. approx-speedup): fused multiply-adds in a fixed order, written to
 * *out (device).  Workspace: qdot_dot_fp64_workspace_size(). */
size_t qdot_dot_fp64_workspace_size(void);
qdot_status qdot_dot_fp64(const double* x, const double* y, int64_t n, double* out, void* ws, size_t ws_bytes,
                          void* stream);

/* End-to-end call from host buffers x_host, y_host (n doubles each); the
 * result lands in *out_host and the stream is synchronised before returning.
 * Page-locked buffers that are mapped into the device's address space
 * (cudaHostAlloc, cudaHostRegister; all of them on a unified-address system)
 * are read in place by the kernels over the host link, in the same single
 * pass, and x_dev, y_dev are left untouched.  Other host memory is first
 * copied into the caller's device buffers x_dev, y_dev, in chunks over
 * several streams. */
qdot_status qdot_from_host(const double* x_host, const double* y_host, int64_t n, const qdot_params* p,
                           qdot_result* out_host, double* x_dev, double* y_dev, qdot_result* out_dev, void* ws,
                           size_t ws_bytes, void* stream);

/* Size of the library-owned scratch array used by qdot_static_scratch(). */
#define QDOT_STATIC_SCRATCH_BYTES (1u << 20)

/* qdot() without a workspace argument, for callers that cannot allocate
 * device memory: code running under a host application that owns the whole
 * device allocator (memory reserved up front, a pool with no room left, a
 * plug-in interface that only passes inputs and outputs) or a deployment that
 * forbids allocation after start-up.  The paper has no counterpart: this is a
 * packaging of the same computation.
 *   x, y, n, p, out, stream  as for qdot(); always the two-pass path.
 * Scratch: a fixed array of QDOT_STATIC_SCRATCH_BYTES inside the library,
 * held by every GPU that loads the library until the process exits.  It
 * fits any n for exact binning, blocks of one component, and blocks of up to
 * 64 components when x and y are 16-byte aligned (up to 32 when they are
 * only 8-byte aligned); larger blocks need 2 bytes per block on top of a
 * fixed ~90 KB, so n is limited to about B * 480000.  Arguments that do not
 * fit return QDOT_ERR_WORKSPACE with a message, before anything is launched.
 * Nothing is allocated: no cudaMalloc, cudaFree or allocating library call.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The address is cached per device with the
 * context it belongs to, and looked up again in a new context (after
 * cudaDeviceReset()).  All calls share the one array, which keeps the last
 * call's contents; each call clears what it needs cleared, but calls whose
 * executions overlap on the GPU (for example on two streams) race on the
 * array and must be serialised by the caller. */
qdot_status qdot_static_scratch(const double* x, const double* y, int64_t n, const qdot_params* p,
                                qdot_result* out, void* stream);

/* Per-unit record of qdot_trace() (16 bytes): what the selection decided for
 * one unit of work of the streaming kernels and what the final sum took from
 * it.  A unit is a block of B components (blocked binning with block records)
 * or a warp item of 256 consecutive components (item records: blocks of one
 * component, and blocks of 32 where the library keeps item records). */
typedef struct {
  int64_t value;     /* the unit's contribution is value * 2^grid, exactly; the
                        final fixed-point sum truncates it to its own grid
                        2^(e_max - L) (see z above) */
  int32_t grid;
  uint8_t cls;       /* block units: the block's class (QDOT_PERF .. QDOT_DOUBLE),
                        QDOT_ZERO for a block without a nonzero component;
                        item units: 255 (the per-component classes go to `cls`
                        of qdot_trace) */
  uint8_t source;    /* QDOT_TRACE_* */
  uint16_t reserved;
} qdot_trace_unit;

enum {
  QDOT_TRACE_NONE = 0,             /* nothing added: perforated or empty block */
  QDOT_TRACE_SLOT0 = 1,            /* the block's first kept candidate (streaming kernel) */
  QDOT_TRACE_SLOT1 = 2,            /* its second kept candidate */
  QDOT_TRACE_SLOT3 = 3,            /* its third kept candidate (HALF, early items) */
  QDOT_TRACE_RECOMPUTED = 4,       /* the candidate was not kept; recomputed from x, y */
  QDOT_TRACE_FUSED = 5,            /* the fused kernel's candidate of the block's class */
  QDOT_TRACE_ITEM = 6,             /* the item's record, accepted */
  QDOT_TRACE_ITEM_RECOMPUTED = 7,  /* the item recomputed with the final classes */
  QDOT_TRACE_ITEM_FIXED = 8        /* blocks of 32 .. 256 on item records: the record, with the
                                      blocks whose class the final selection changed summed
                                      again from x, y and swapped in */
};

/* Number of qdot_trace_unit records qdot_trace() writes for these arguments,
 * with the components per unit in *unit_components (B or 256); 0 when qdot()
 * takes the two-pass path (whose per-component view is qdot_explain) or on
 * invalid parameters.  `aligned16` tells whether x and y are 16-byte aligned. */
int64_t qdot_trace_units(int64_t n, const qdot_params* p, int32_t aligned16, int32_t* unit_components);

/* qdot() on the fused or one-pass path, exactly as qdot() runs it (same
 * kernels, launch shapes and result), that also reports what its kernels
 * decided, for checking the timed path component by component against an
 * independent implementation of Algorithm 3.
 *   units     device array of at least qdot_trace_units(...) records: per
 *             unit its class (block units) and the exact value the final sum
 *             took from it (qdot_trace_unit).
 *   cls       optional device array of n bytes (item units only): the class
 *             each component was summed with (QDOT_ZERO for zero components);
 *             left untouched on block paths.  NULL to skip.
 *   units_len length of `units` in records.
 * Everything else as for qdot().  Returns QDOT_ERR_ARG when qdot() would take
 * the two-pass path or `units` is too short. */
qdot_status qdot_trace(const double* x, const double* y, int64_t n, const qdot_params* p, qdot_result* out,
                       qdot_trace_unit* units, int64_t units_len, uint8_t* cls, void* ws, size_t ws_bytes,
                       void* stream);

/* Number of kernels one qdot() call with these arguments launches (0 on
 * invalid parameters); `aligned16` tells whether x and y are 16-byte aligned. */
int32_t qdot_kernel_launches(int64_t n, const qdot_params* p, int32_t aligned16);

/* The path qdot() takes for these arguments: QDOT_PATH_FUSED,
 * QDOT_PATH_ONE_PASS or QDOT_PATH_TWO_PASS (0 on invalid parameters). */
int32_t qdot_select_path(int64_t n, const qdot_params* p, int32_t aligned16);

/* Name of the streaming kernel qdot() runs for these arguments (the one the
 * measurement hook below times): "k_qdot_fused", "k_onepass" (block
 * records), "k_onepass_items" (item records: blocks of one component) or
 * "k_apply_fast" (two-pass); "" on invalid parameters.
 * A static string. */
const char* qdot_stream_kernel(int64_t n, const qdot_params* p, int32_t aligned16);

/* Measurement hook.  When begin and end are both non-NULL (cudaEvent_t
 * handles created by the caller), every later qdot() on the calling thread
 * records `begin` on the call's stream right before its main streaming kernel
 * (the one-pass kernel, or the second pass of the two-pass path) and `end`
 * right after it, so the caller can time that kernel alone.  Pass NULL, NULL
 * to stop.  Not part of the method. */
void qdot_set_kernel_events(void* begin, void* end);

/* Message for the last failing call on the calling thread ("" if none). */
const char* qdot_last_error(void);

/* Library version string. */
const char* qdot_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QDOT_H */
