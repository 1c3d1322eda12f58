/*
 * qdot CPU oracle -- TEST INFRASTRUCTURE ONLY (private header of oracle/).
 * See qdot_oracle.c for the readings of the paper this code takes.
 */
#ifndef QDOT_ORACLE_H
#define QDOT_ORACLE_H
#include <stdint.h>

enum { ORC_PERF = 0, ORC_HALF = 1, ORC_SINGLE = 2, ORC_DOUBLE = 3, ORC_ZERO = 4 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NONFINITE = 2 };

typedef struct {
  double eps;           /* qdot tolerance, > 0 */
  int32_t block;        /* 0: exact binning; B >= 1: index blocks of B */
  int32_t split_budget; /* 1: eps / N_bins (Sec. 4.1); 0: eps */
  int32_t mant_reading; /* 0: m_half, m_single = 10, 23; 1: 11, 24 */
  int32_t pad;
} orc_params;

typedef struct {
  double value;         /* z, the exact sum of quantized products rounded once */
  double value_ld;      /* the same sum accumulated in long double */
  double class_sum[4];  /* [0] exact sum of the perforated x_i y_i; [1..3] exact
                           HALF / SINGLE / DOUBLE partial sums; each rounded once */
  double bound_elem;    /* sum of element-wise error bounds */
  double bound_bins;    /* sum over bins of M_k 2^(u_k + 2 - p_k) */
  double bound_apriori; /* N_bins 2^(e_max + f) */
  int32_t e_max, e_min; /* over non-ZERO keys; 0 when there are none */
  int64_t n_bins;
  int32_t f;            /* floor(log2(eps_eff)) */
  int32_t status;
  int64_t count[5];     /* components per class PERF, HALF, SINGLE, DOUBLE, ZERO */
} orc_result;

int orc_qdot(const double* x, const double* y, int64_t n, const orc_params* prm, uint8_t* cls_out,
             double* qx_out, double* qy_out, orc_result* res);
double orc_quantize(double v, int cls);
int orc_floor_log2_ratio(double eps, int64_t N);
int orc_unit_sums(const double* x, const double* y, int64_t n, const orc_params* prm, int64_t unit, double* sums,
                  double* abs_sums);
double orc_dot_exact(const double* x, const double* y, int64_t n);
double orc_abs_dot_exact(const double* x, const double* y, int64_t n);
double orc_sum_exact(const double* v, int64_t n);
void orc_spmv(int64_t nrows, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
              double* y);
int orc_cg(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
           double rel_tol, int32_t max_it, const orc_params* prm, int32_t* iters, double* relres,
           int64_t* class_counts);
int orc_power(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, double* x, int32_t iters,
              double tau, const orc_params* prm, double* lambda, int32_t* done_iters, int64_t* class_counts);
int orc_qdot_threads(const double* x, const double* y, int64_t n, const orc_params* prm, int nthreads,
                     orc_result* res);
double orc_dot_fp64(const double* x, const double* y, int64_t n, int nthreads);
int orc_max_threads(void);
void orc_backward(const double* x, const double* y, const uint8_t* cls, int64_t n, double g, double* gx,
                  double* gy);

#endif
