/*
 * qdot CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct C implementation of the quantized dot product
 * "qdot" (Diffenderfer, Osei-Kuffuor, Menon, arXiv 2105.00115) and of the two
 * applications the paper runs it in (approximate CG, approximate power method).
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  The GPU library shares no code, header or
 * table with it.
 *
 * Every floating-point result here is computed exactly (integer significands
 * and a fixed-point "Kulisch" accumulator wide enough for any sum of products
 * of doubles) and rounded once, to nearest-even, at the end.
 *
 * Readings of the paper taken here (each one is listed in the design notes):
 *  - exponent of a component: the unbiased IEEE exponent ilogb(v)
 *    (Sec. 1.1 says flexp is the unbiased exponent; Sec. 3.2 extracts it by
 *    bitmask), subnormals with their true exponent;
 *  - component key e_i = ilogb(x_i) + ilogb(y_i) (Algorithm 2, exponent
 *    preprocessing); a component with x_i = 0 or y_i = 0 is class ZERO:
 *    excluded from every bin, contributes exactly 0;
 *  - bins: exact binning (Sec. 3.2 / Algorithm 3) when block == 0, else
 *    contiguous index blocks of `block` components (the blocked approach of
 *    Sec. 5) with u_b = max key, M_b = number of non-ZERO components;
 *  - f = floor(log2(eps / N_bins)) computed exactly (Sec. 4.1 uses
 *    eps / N_bins in the bin score); split_budget = 0 selects raw eps;
 *  - bin score (eq. bin-score-def) and precision function (eq. precision-def)
 *    with m_half, m_single = 10, 23 stored mantissa bits (mant_reading = 0)
 *    or 11, 24 (mant_reading = 1); a score >= m_single is DOUBLE (the quad
 *    line of eq. precision-def is commented out in the paper);
 *  - quantizing to half / single = rounding the 53-bit significand to 11 / 24
 *    bits, ties to even, exponent unbounded (the scale-to-exponent-0, cast,
 *    rescale-by-2^u procedure of Sec. 3.2);
 *  - the computation phase (Algorithm 1) sums the quantized products exactly
 *    and rounds once.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "qdot_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Exact fixed-point accumulator.  Word 0 bit 0 has weight 2^KLSB.  Two's      */
/* complement over KW 64-bit words.  Range covers every product of two finite */
/* doubles (2^-2252 .. 2^2050) plus 2^40 summands of headroom.               */
/* ------------------------------------------------------------------------- */
#define KW 72
#define KLSB (-2304)

typedef struct {
  uint64_t w[KW];
} kacc;

static void kacc_zero(kacc* a) { memset(a->w, 0, sizeof(a->w)); }

/* a += (-1)^neg * mag * 2^exp2, with exp2 >= KLSB and mag < 2^120. */
static void kacc_add(kacc* a, unsigned __int128 mag, int exp2, int neg) {
  if (mag == 0) return;
  int pos = exp2 - KLSB;
  int wi = pos >> 6, sh = pos & 63;
  uint64_t lo = (uint64_t)mag, hi = (uint64_t)(mag >> 64);
  uint64_t part[3];
  if (sh == 0) {
    part[0] = lo;
    part[1] = hi;
    part[2] = 0;
  } else {
    part[0] = lo << sh;
    part[1] = (lo >> (64 - sh)) | (hi << sh);
    part[2] = hi >> (64 - sh);
  }
  if (!neg) {
    uint64_t carry = 0;
    for (int j = 0; wi + j < KW; ++j) {
      uint64_t add = (j < 3) ? part[j] : 0;
      if (j >= 3 && carry == 0) break;
      uint64_t s = a->w[wi + j] + add;
      uint64_t c1 = (s < add);
      uint64_t s2 = s + carry;
      uint64_t c2 = (s2 < carry);
      a->w[wi + j] = s2;
      carry = c1 | c2;
    }
  } else {
    uint64_t borrow = 0;
    for (int j = 0; wi + j < KW; ++j) {
      uint64_t sub = (j < 3) ? part[j] : 0;
      if (j >= 3 && borrow == 0) break;
      uint64_t old = a->w[wi + j];
      uint64_t d = old - sub;
      uint64_t b1 = (old < sub);
      uint64_t d2 = d - borrow;
      uint64_t b2 = (d < borrow);
      a->w[wi + j] = d2;
      borrow = b1 | b2;
    }
  }
}

static int kacc_bit(const kacc* a, int i) { return (int)((a->w[i >> 6] >> (i & 63)) & 1u); }

/* Round the exact value to the nearest double, ties to even. */
static double kacc_to_double(const kacc* acc) {
  kacc m = *acc;
  int neg = (int)((m.w[KW - 1] >> 63) & 1u);
  if (neg) {
    uint64_t carry = 1;
    for (int j = 0; j < KW; ++j) {
      uint64_t v = ~m.w[j];
      uint64_t s = v + carry;
      carry = (s < carry);
      m.w[j] = s;
    }
  }
  int h = -1;
  for (int j = KW - 1; j >= 0; --j) {
    if (m.w[j]) {
      h = j * 64 + 63 - __builtin_clzll(m.w[j]);
      break;
    }
  }
  if (h < 0) return 0.0;
  int top_exp = h + KLSB;
  if (top_exp >= 1024) return neg ? -INFINITY : INFINITY;
  int r = h - 52;               /* bit index of the result's last place */
  int rmin = -1074 - KLSB;      /* last place of a subnormal */
  if (r < rmin) r = rmin;
  uint64_t mi = 0;
  for (int i = h; i >= r; --i) mi = (mi << 1) | (uint64_t)kacc_bit(&m, i);
  int round_bit = (r - 1 >= 0) ? kacc_bit(&m, r - 1) : 0;
  int sticky = 0;
  for (int i = r - 2; i >= 0 && !sticky; --i) sticky = kacc_bit(&m, i);
  if (round_bit && (sticky || (mi & 1u))) mi += 1;
  double v = ldexp((double)mi, r + KLSB);
  return neg ? -v : v;
}

/* ------------------------------------------------------------------------- */
/* Significands and quantization                                             */
/* ------------------------------------------------------------------------- */

/* |v| = M * 2^E with 2^52 <= M < 2^53 (v finite, nonzero; subnormals
 * normalised). */
static void decompose(double v, uint64_t* M, int* E) {
  int k;
  double m = frexp(fabs(v), &k); /* |v| = m 2^k, 0.5 <= m < 1 */
  *M = (uint64_t)ldexp(m, 53);
  *E = k - 53;
}

/* Round the 53-bit significand M to p bits, ties to even, with an unbounded
 * exponent: M * 2^E ~= Mq * 2^Eq, Mq <= 2^p. */
static void round_significand(uint64_t M, int E, int p, uint64_t* Mq, int* Eq) {
  if (p >= 53) {
    *Mq = M;
    *Eq = E;
    return;
  }
  int k = 53 - p;
  uint64_t q = M >> k;
  uint64_t rem = M & ((1ull << k) - 1ull);
  uint64_t half = 1ull << (k - 1);
  if (rem > half || (rem == half && (q & 1u))) q += 1;
  *Mq = q;
  *Eq = E + k;
}

static int class_bits(int cls) {
  switch (cls) {
    case ORC_HALF: return 11;
    case ORC_SINGLE: return 24;
    default: return 53;
  }
}

double orc_quantize(double v, int cls) {
  if (cls == ORC_PERF || cls == ORC_ZERO || v == 0.0) return 0.0;
  uint64_t M, Mq;
  int E, Eq;
  decompose(v, &M, &E);
  round_significand(M, E, class_bits(cls), &Mq, &Eq);
  double q = ldexp((double)Mq, Eq);
  return v < 0 ? -q : q;
}

/* ------------------------------------------------------------------------- */
/* Parameter selection (Algorithm 2)                                         */
/* ------------------------------------------------------------------------- */

static int ceil_log2_u64(uint64_t m) {
  int c = 0;
  while (c < 64 && (1ull << c) < m) c++;
  return c;
}

/* N * 2^k <= eps, exactly (eps > 0 finite, N >= 1). */
static int scaled_count_le(int64_t N, int k, double eps) {
  uint64_t Me;
  int Ee;
  decompose(eps, &Me, &Ee); /* eps = Me * 2^Ee */
  int d = k - Ee;           /* compare N * 2^d with Me */
  unsigned __int128 lhs = (unsigned __int128)(uint64_t)N;
  unsigned __int128 rhs = (unsigned __int128)Me;
  if (d >= 0) {
    if (d >= 64) return 0; /* N * 2^d >= 2^64 > Me */
    lhs <<= d;
  } else {
    if (-d >= 64) return 1; /* Me * 2^-d >= 2^116 > N */
    rhs <<= -d;
  }
  return lhs <= rhs;
}

int orc_floor_log2_ratio(double eps, int64_t N) {
  int k = ilogb(eps) - ceil_log2_u64((uint64_t)N);
  while (scaled_count_le(N, k + 1, eps)) k++;
  while (!scaled_count_le(N, k, eps)) k--;
  return k;
}

/* Precision function, eq. (precision-def), with the reading that a score at or
 * above m_single stays at the input precision (double). */
static int precision_of_score(int64_t sigma, int m_half, int m_single) {
  if (sigma < 0) return ORC_PERF;
  if (sigma < m_half) return ORC_HALF;
  if (sigma < m_single) return ORC_SINGLE;
  return ORC_DOUBLE;
}

typedef struct {
  int64_t M;    /* cardinality M_k */
  int32_t u;    /* upper end u_k of the bin's key range */
  int32_t cls;  /* precision pi_k */
} orc_bin;

/* ------------------------------------------------------------------------- */
/* qdot = Algorithm 2 (parameter selection) then Algorithm 1 (computation)   */
/* ------------------------------------------------------------------------- */
int orc_qdot(const double* x, const double* y, int64_t n, const orc_params* prm, uint8_t* cls_out,
             double* qx_out, double* qy_out, orc_result* res) {
  memset(res, 0, sizeof(*res));
  if (n < 0 || !(prm->eps > 0.0) || !isfinite(prm->eps) || prm->block < 0) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  for (int64_t i = 0; i < n; ++i) {
    if (!isfinite(x[i]) || !isfinite(y[i])) {
      res->status = ORC_ERR_NONFINITE;
      return ORC_ERR_NONFINITE;
    }
  }
  const int m_half = prm->mant_reading ? 11 : 10;
  const int m_single = prm->mant_reading ? 24 : 23;

  /* Algorithm 2, exponent preprocessing: e = flexp(x) + flexp(y). */
  int32_t* e = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* is_zero = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  int64_t nonzero = 0;
  for (int64_t i = 0; i < n; ++i) {
    is_zero[i] = (x[i] == 0.0 || y[i] == 0.0);
    e[i] = is_zero[i] ? 0 : ilogb(x[i]) + ilogb(y[i]);
    nonzero += !is_zero[i];
  }

  /* Algorithm 2: e_min and e_max over the non-ZERO components. */
  int32_t e_min = 0, e_max = 0;
  int first = 1;
  for (int64_t i = 0; i < n; ++i) {
    if (is_zero[i]) continue;
    if (first || e[i] > e_max) e_max = e[i];
    if (first || e[i] < e_min) e_min = e[i];
    first = 0;
  }

  /* Algorithm 2: bins B_k with cardinality M_k and upper key u_k, and for each
   * component the bin it belongs to (bin_of[i], -1 for ZERO). */
  int64_t* bin_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  orc_bin* bins = NULL;
  int64_t n_bins = 0;
  if (prm->block == 0) {
    /* Exact binning via counting sort of e over [e_min, e_max]: cumulative
     * counts delimit the singleton bins (u_k - 1, u_k]. */
    int64_t range = nonzero ? (int64_t)e_max - e_min + 1 : 0;
    /* count[k] = number of components with key e_min + k */
    int64_t* count = (int64_t*)calloc((size_t)(range + 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i)
      if (!is_zero[i]) count[e[i] - e_min] += 1;
    /* start[k] = number of components with key < e_min + k (cumulative counts) */
    int64_t* start = (int64_t*)calloc((size_t)(range + 1), sizeof(int64_t));
    for (int64_t k = 0; k < range; ++k) start[k + 1] = start[k] + count[k];
    int64_t* sorted = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nonzero > 0 ? nonzero : 1));
    int64_t* fill = (int64_t*)calloc((size_t)(range + 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
      if (is_zero[i]) continue;
      int64_t k = e[i] - e_min;
      sorted[start[k] + fill[k]] = i;
      fill[k] += 1;
    }
    /* Each non-empty run of equal keys in sorted order is one bin. */
    int64_t* bin_id_of_key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(range > 0 ? range : 1));
    for (int64_t k = 0; k < range; ++k) {
      bin_id_of_key[k] = -1;
      if (count[k] > 0) n_bins++;
    }
    bins = (orc_bin*)calloc((size_t)(n_bins > 0 ? n_bins : 1), sizeof(orc_bin));
    int64_t b = 0;
    for (int64_t k = 0; k < range; ++k) {
      if (count[k] == 0) continue;
      bins[b].M = count[k];
      bins[b].u = (int32_t)(e_min + k);
      bin_id_of_key[k] = b;
      b++;
    }
    for (int64_t i = 0; i < n; ++i) bin_of[i] = -1;
    for (int64_t s = 0; s < nonzero; ++s) {
      int64_t i = sorted[s];
      bin_of[i] = bin_id_of_key[e[i] - e_min];
    }
    free(count);
    free(start);
    free(sorted);
    free(fill);
    free(bin_id_of_key);
  } else {
    /* Blocked binning: bin b holds the non-ZERO components of the index block
     * [b*B, (b+1)*B); its upper key is the block maximum. */
    int64_t B = prm->block;
    int64_t nblk = (n + B - 1) / B;
    int64_t* blk_bin = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nblk > 0 ? nblk : 1));
    for (int64_t blk = 0; blk < nblk; ++blk) {
      int64_t M = 0;
      for (int64_t i = blk * B; i < n && i < (blk + 1) * B; ++i) M += !is_zero[i];
      blk_bin[blk] = M > 0 ? n_bins++ : -1;
    }
    bins = (orc_bin*)calloc((size_t)(n_bins > 0 ? n_bins : 1), sizeof(orc_bin));
    for (int64_t blk = 0; blk < nblk; ++blk) {
      int64_t b = blk_bin[blk];
      if (b < 0) continue;
      int32_t u = 0;
      int64_t M = 0;
      for (int64_t i = blk * B; i < n && i < (blk + 1) * B; ++i) {
        if (is_zero[i]) continue;
        if (M == 0 || e[i] > u) u = e[i];
        M++;
      }
      bins[b].M = M;
      bins[b].u = u;
    }
    for (int64_t i = 0; i < n; ++i) bin_of[i] = is_zero[i] ? -1 : blk_bin[i / B];
    free(blk_bin);
  }

  /* Algorithm 2: bin scores (eq. bin-score-def) with floor(log2(eps_eff)),
   * eps_eff = eps / N_bins (Sec. 4.1) or eps, then precisions (eq.
   * precision-def). */
  int32_t f = 0;
  if (n_bins > 0) f = orc_floor_log2_ratio(prm->eps, prm->split_budget ? n_bins : 1);
  for (int64_t b = 0; b < n_bins; ++b) {
    int64_t sigma = (int64_t)ceil_log2_u64((uint64_t)bins[b].M) + bins[b].u - e_max - f + 1;
    bins[b].cls = precision_of_score(sigma, m_half, m_single);
  }

  /* Algorithm 1: for each bin cast the sub-vectors to pi_k, take their dot
   * product, and accumulate.  Every product is exact and summed exactly. */
  kacc total, cls_acc[4];
  kacc_zero(&total);
  for (int c = 0; c < 4; ++c) kacc_zero(&cls_acc[c]);
  long double ld = 0.0L;
  kacc bound_elem;
  kacc_zero(&bound_elem);
  for (int64_t i = 0; i < n; ++i) {
    int cls = bin_of[i] < 0 ? ORC_ZERO : bins[bin_of[i]].cls;
    res->count[cls] += 1;
    if (cls_out) cls_out[i] = (uint8_t)cls;
    double qxi = 0.0, qyi = 0.0;
    if (cls != ORC_ZERO) {
      uint64_t Mx, My, Mqx, Mqy;
      int Ex, Ey, Eqx, Eqy;
      decompose(x[i], &Mx, &Ex);
      decompose(y[i], &My, &Ey);
      int neg = (x[i] < 0) != (y[i] < 0);
      if (cls == ORC_PERF) {
        /* dropped mass: exact x_i y_i (reported as the PERF partial sum) */
        kacc_add(&cls_acc[ORC_PERF], (unsigned __int128)Mx * My, Ex + Ey, neg);
        /* element-wise bound |x_i y_i| < 2^(e_i + 2) */
        kacc_add(&bound_elem, 1, e[i] + 2, 0);
      } else {
        int p = class_bits(cls);
        round_significand(Mx, Ex, p, &Mqx, &Eqx);
        round_significand(My, Ey, p, &Mqy, &Eqy);
        unsigned __int128 prod = (unsigned __int128)Mqx * Mqy;
        kacc_add(&total, prod, Eqx + Eqy, neg);
        kacc_add(&cls_acc[cls], prod, Eqx + Eqy, neg);
        qxi = ldexp((double)Mqx, Eqx);
        qyi = ldexp((double)Mqy, Eqy);
        if (x[i] < 0) qxi = -qxi;
        if (y[i] < 0) qyi = -qyi;
        ld += (long double)qxi * (long double)qyi;
        /* element-wise bound |q(x)q(y) - xy| <= 2^(e_i + 2 - p) */
        if (cls != ORC_DOUBLE) kacc_add(&bound_elem, 1, e[i] + 2 - p, 0);
      }
    }
    if (qx_out) qx_out[i] = qxi;
    if (qy_out) qy_out[i] = qyi;
  }

  /* Bin-wise bound sum_k M_k 2^(u_k + 2 - p_k) (PERF: p = 0, DOUBLE: 0). */
  kacc bound_bins;
  kacc_zero(&bound_bins);
  for (int64_t b = 0; b < n_bins; ++b) {
    if (bins[b].cls == ORC_DOUBLE) continue;
    int p = bins[b].cls == ORC_PERF ? 0 : class_bits(bins[b].cls);
    kacc_add(&bound_bins, (unsigned __int128)(uint64_t)bins[b].M, bins[b].u + 2 - p, 0);
  }

  res->value = kacc_to_double(&total);
  res->value_ld = (double)ld;
  for (int c = 0; c < 4; ++c) res->class_sum[c] = kacc_to_double(&cls_acc[c]);
  res->bound_elem = kacc_to_double(&bound_elem);
  res->bound_bins = kacc_to_double(&bound_bins);
  res->bound_apriori = n_bins > 0 ? ldexp((double)n_bins, e_max + f) : 0.0;
  res->e_max = e_max;
  res->e_min = e_min;
  res->n_bins = (int64_t)n_bins;
  res->f = f;
  res->status = ORC_OK;
  free(e);
  free(is_zero);
  free(bin_of);
  free(bins);
  return ORC_OK;
}

/* Partial sums of Algorithm 1 over index ranges: for every range
 * [k*unit, (k+1)*unit) of the components, the exact sum of the quantized
 * products q(x_i) q(y_i) of its components (classes from Algorithm 2 on the
 * whole vectors, as orc_qdot assigns them) and the exact sum of |x_i y_i|,
 * each rounded once.  sums and abs_sums hold ceil(n / unit) doubles.
 * Returns the status of orc_qdot. */
int orc_unit_sums(const double* x, const double* y, int64_t n, const orc_params* prm, int64_t unit, double* sums,
                  double* abs_sums) {
  if (unit < 1) return ORC_ERR_ARG;
  uint8_t* cls = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  orc_result r;
  int st = orc_qdot(x, y, n, prm, cls, NULL, NULL, &r);
  if (st != ORC_OK) {
    free(cls);
    return st;
  }
  for (int64_t lo = 0; lo < n; lo += unit) {
    kacc q, a;
    kacc_zero(&q);
    kacc_zero(&a);
    for (int64_t i = lo; i < n && i < lo + unit; ++i) {
      if (cls[i] == ORC_ZERO) continue;
      uint64_t Mx, My, Mqx, Mqy;
      int Ex, Ey, Eqx, Eqy;
      decompose(x[i], &Mx, &Ex);
      decompose(y[i], &My, &Ey);
      int neg = (x[i] < 0) != (y[i] < 0);
      kacc_add(&a, (unsigned __int128)Mx * My, Ex + Ey, 0);
      if (cls[i] == ORC_PERF) continue;
      int p = class_bits(cls[i]);
      round_significand(Mx, Ex, p, &Mqx, &Eqx);
      round_significand(My, Ey, p, &Mqy, &Eqy);
      kacc_add(&q, (unsigned __int128)Mqx * Mqy, Eqx + Eqy, neg);
    }
    sums[lo / unit] = kacc_to_double(&q);
    abs_sums[lo / unit] = kacc_to_double(&a);
  }
  free(cls);
  return ORC_OK;
}

/* Exact x.y rounded once (every component at input precision). */
double orc_dot_exact(const double* x, const double* y, int64_t n) {
  kacc a;
  kacc_zero(&a);
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] == 0.0 || y[i] == 0.0) continue;
    uint64_t Mx, My;
    int Ex, Ey;
    decompose(x[i], &Mx, &Ex);
    decompose(y[i], &My, &Ey);
    kacc_add(&a, (unsigned __int128)Mx * My, Ex + Ey, (x[i] < 0) != (y[i] < 0));
  }
  return kacc_to_double(&a);
}

/* Exact sum of |x_i y_i| rounded once. */
double orc_abs_dot_exact(const double* x, const double* y, int64_t n) {
  kacc a;
  kacc_zero(&a);
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] == 0.0 || y[i] == 0.0) continue;
    uint64_t Mx, My;
    int Ex, Ey;
    decompose(x[i], &Mx, &Ex);
    decompose(y[i], &My, &Ey);
    kacc_add(&a, (unsigned __int128)Mx * My, Ex + Ey, 0);
  }
  return kacc_to_double(&a);
}

/* Sum of a list of doubles, exactly, rounded once (used by tests to combine
 * exact partials). */
double orc_sum_exact(const double* v, int64_t n) {
  kacc a;
  kacc_zero(&a);
  for (int64_t i = 0; i < n; ++i) {
    if (v[i] == 0.0) continue;
    uint64_t M;
    int E;
    decompose(v[i], &M, &E);
    kacc_add(&a, (unsigned __int128)M, E, v[i] < 0);
  }
  return kacc_to_double(&a);
}

/* ------------------------------------------------------------------------- */
/* Applications: CSR SpMV, approximate CG (Algorithm 4), approximate power    */
/* method (Algorithm 5), backward of qdot.                                    */
/* ------------------------------------------------------------------------- */

/* y = A x, row sums in CSR order with fused multiply-add. */
void orc_spmv(int64_t nrows, const int64_t* rowptr, const int32_t* col, const double* val, const double* x,
              double* y) {
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s = fma(val[k], x[col[k]], s);
    y[r] = s;
  }
}

static double orc_qdot_value(const double* a, const double* b, int64_t n, const orc_params* prm, int* status,
                             int64_t count[5]) {
  orc_result r;
  int st = orc_qdot(a, b, n, prm, NULL, NULL, NULL, &r);
  if (st != ORC_OK) *status = st;
  if (count)
    for (int c = 0; c < 5; ++c) count[c] += r.count[c];
  return r.value;
}

/* Algorithm 4 (ACG).  x holds x0 on entry and the solution on exit.  The loop
 * test uses ||r_k|| = sqrt(c_k) relative to ||b|| (exact norm of b).  Returns
 * the iteration count in *iters and sqrt(c_k)/||b|| in *relres. */
int orc_cg(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, const double* b, double* x,
           double rel_tol, int32_t max_it, const orc_params* prm, int32_t* iters, double* relres,
           int64_t* class_counts) {
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  int status = ORC_OK;
  int64_t dummy[5] = {0, 0, 0, 0, 0};
  int64_t* cc = class_counts ? class_counts : dummy;
  orc_spmv(n, rowptr, col, val, x, q);
  for (int64_t i = 0; i < n; ++i) {
    r[i] = b[i] - q[i];
    p[i] = r[i];
  }
  double bnorm = sqrt(orc_dot_exact(b, b, n));
  double c = orc_qdot_value(r, r, n, prm, &status, cc);
  int32_t k = 0;
  while (status == ORC_OK && k < max_it && sqrt(c) / bnorm > rel_tol) {
    orc_spmv(n, rowptr, col, val, p, q);
    double pq = orc_qdot_value(p, q, n, prm, &status, cc);
    double alpha = c / pq;
    for (int64_t i = 0; i < n; ++i) {
      x[i] = fma(alpha, p[i], x[i]);
      r[i] = fma(-alpha, q[i], r[i]);
    }
    double c_new = orc_qdot_value(r, r, n, prm, &status, cc);
    double beta = c_new / c;
    for (int64_t i = 0; i < n; ++i) p[i] = fma(beta, p[i], r[i]);
    c = c_new;
    k++;
  }
  *iters = k;
  *relres = sqrt(c) / bnorm;
  free(r);
  free(p);
  free(q);
  return status;
}

/* Algorithm 5 (APM) with the Rayleigh-quotient reading of the eigenvalue
 * update: for k = 0..iters-1: w = A x_k; lambda_k = qdot(x_k, w);
 * c = qdot(w, w); x_{k+1} = w * (1/sqrt(c)).  Stops early when tau > 0 and
 * |lambda_k - lambda_{k-1}| <= tau.  x holds x0 (unit norm) on entry. */
int orc_power(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val, double* x, int32_t iters,
              double tau, const orc_params* prm, double* lambda, int32_t* done_iters, int64_t* class_counts) {
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  int status = ORC_OK;
  int64_t dummy[5] = {0, 0, 0, 0, 0};
  int64_t* cc = class_counts ? class_counts : dummy;
  double lam = 0.0, lam_prev = 0.0;
  int32_t k = 0;
  for (; k < iters && status == ORC_OK; ++k) {
    orc_spmv(n, rowptr, col, val, x, w);
    lam = orc_qdot_value(x, w, n, prm, &status, cc);
    double c = orc_qdot_value(w, w, n, prm, &status, cc);
    double s = 1.0 / sqrt(c);
    for (int64_t i = 0; i < n; ++i) x[i] = w[i] * s;
    if (tau > 0.0 && k > 0 && fabs(lam - lam_prev) <= tau) {
      k++;
      break;
    }
    lam_prev = lam;
  }
  *lambda = lam;
  *done_iters = k;
  free(w);
  return status;
}

/* Backward of z = qdot(x, y) with the class map frozen: dz/dx_i = q(y_i),
 * dz/dy_i = q(x_i) for HALF / SINGLE / DOUBLE components, 0 otherwise; both
 * scaled by the upstream gradient g (one rounding each). */
void orc_backward(const double* x, const double* y, const uint8_t* cls, int64_t n, double g, double* gx,
                  double* gy) {
  for (int64_t i = 0; i < n; ++i) {
    gx[i] = g * orc_quantize(y[i], cls[i]);
    gy[i] = g * orc_quantize(x[i], cls[i]);
  }
}

/* ------------------------------------------------------------------------- */
/* CPU baseline: the same computation spread over host threads, and a plain  */
/* FP64 dot.  Used only to time the host cores; the pins check that the      */
/* threaded result equals orc_qdot's exactly.                                */
/* ------------------------------------------------------------------------- */

/* a += b, both exact accumulators (two's complement words with carry). */
static void kacc_merge(kacc* a, const kacc* b) {
  uint64_t carry = 0;
  for (int j = 0; j < KW; ++j) {
    uint64_t s = a->w[j] + b->w[j];
    uint64_t c1 = s < b->w[j];
    uint64_t s2 = s + carry;
    uint64_t c2 = s2 < carry;
    a->w[j] = s2;
    carry = c1 | c2;
  }
}

static int key_of(double a, double b) { return ilogb(a) + ilogb(b); }

/* orc_qdot's value, counts and statistics with the components split over
 * nthreads host threads (OpenMP when built with it): Algorithm 2's
 * statistics per thread, then merged; Algorithm 1's exact sum per thread in
 * its own accumulator, the accumulators added exactly, one rounding.  The
 * bound fields of res are left 0. */
int orc_qdot_threads(const double* x, const double* y, int64_t n, const orc_params* prm, int nthreads,
                     orc_result* res) {
  memset(res, 0, sizeof(*res));
  if (n < 0 || !(prm->eps > 0.0) || !isfinite(prm->eps) || prm->block < 0 || nthreads < 1) {
    res->status = ORC_ERR_ARG;
    return ORC_ERR_ARG;
  }
  const int m_half = prm->mant_reading ? 11 : 10;
  const int m_single = prm->mant_reading ? 24 : 23;
  enum { KMIN = -2148, KCOUNT = 4224 };
  int bad = 0, e_max = INT32_MIN, e_min = INT32_MAX;
  int64_t nonzero = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) reduction(| : bad) reduction(max : e_max) reduction(min : e_min) \
    reduction(+ : nonzero) schedule(static)
#endif
  for (int64_t i = 0; i < n; ++i) {
    if (!isfinite(x[i]) || !isfinite(y[i])) {
      bad |= 1;
      continue;
    }
    if (x[i] == 0.0 || y[i] == 0.0) continue;
    const int e = key_of(x[i], y[i]);
    if (e > e_max) e_max = e;
    if (e < e_min) e_min = e;
    nonzero++;
  }
  if (bad) {
    res->status = ORC_ERR_NONFINITE;
    return ORC_ERR_NONFINITE;
  }
  if (nonzero == 0) e_max = e_min = 0;
  /* bins: per block (u_b, M_b), or per key (count) */
  int64_t n_bins = 0;
  const int64_t B = prm->block;
  const int64_t nblk = B > 0 ? (n + B - 1) / B : 0;
  int32_t* bu = NULL;
  int64_t* bm = NULL;
  int64_t hist[KCOUNT];
  memset(hist, 0, sizeof(hist));
  if (B > 0) {
    bu = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nblk > 0 ? nblk : 1));
    bm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nblk > 0 ? nblk : 1));
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) reduction(+ : n_bins) schedule(static)
#endif
    for (int64_t b = 0; b < nblk; ++b) {
      int32_t u = INT32_MIN;
      int64_t m = 0;
      for (int64_t i = b * B; i < n && i < (b + 1) * B; ++i) {
        if (x[i] == 0.0 || y[i] == 0.0) continue;
        const int e = key_of(x[i], y[i]);
        if (e > u) u = e;
        m++;
      }
      bu[b] = u;
      bm[b] = m;
      n_bins += m > 0;
    }
  } else {
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
      int64_t h[KCOUNT];
      memset(h, 0, sizeof(h));
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
      for (int64_t i = 0; i < n; ++i)
        if (x[i] != 0.0 && y[i] != 0.0) h[key_of(x[i], y[i]) - KMIN] += 1;
#ifdef _OPENMP
#pragma omp critical
#endif
      for (int k = 0; k < KCOUNT; ++k) hist[k] += h[k];
    }
    for (int k = 0; k < KCOUNT; ++k) n_bins += hist[k] > 0;
  }
  const int32_t f = n_bins > 0 ? orc_floor_log2_ratio(prm->eps, prm->split_budget ? n_bins : 1) : 0;
  /* Algorithm 1 per thread */
  kacc* accs = (kacc*)malloc(sizeof(kacc) * (size_t)nthreads);
  int64_t counts[5] = {0, 0, 0, 0, 0};
  int64_t* tcounts = (int64_t*)calloc((size_t)nthreads * 5, sizeof(int64_t));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    kacc_zero(&accs[t]);
    int64_t* c = tcounts + 5 * t;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) {
      if (x[i] == 0.0 || y[i] == 0.0) {
        c[ORC_ZERO] += 1;
        continue;
      }
      int64_t sigma;
      if (B > 0) {
        const int64_t b = i / B;
        sigma = (int64_t)ceil_log2_u64((uint64_t)bm[b]) + bu[b] - e_max - f + 1;
      } else {
        const int e = key_of(x[i], y[i]);
        sigma = (int64_t)ceil_log2_u64((uint64_t)hist[e - KMIN]) + e - e_max - f + 1;
      }
      const int cls = precision_of_score(sigma, m_half, m_single);
      c[cls] += 1;
      if (cls == ORC_PERF) continue;
      uint64_t Mx, My, Mqx, Mqy;
      int Ex, Ey, Eqx, Eqy;
      decompose(x[i], &Mx, &Ex);
      decompose(y[i], &My, &Ey);
      const int p = class_bits(cls);
      round_significand(Mx, Ex, p, &Mqx, &Eqx);
      round_significand(My, Ey, p, &Mqy, &Eqy);
      kacc_add(&accs[t], (unsigned __int128)Mqx * Mqy, Eqx + Eqy, (x[i] < 0) != (y[i] < 0));
    }
  }
  for (int t = 1; t < nthreads; ++t) kacc_merge(&accs[0], &accs[t]);
  for (int t = 0; t < nthreads; ++t)
    for (int k = 0; k < 5; ++k) counts[k] += tcounts[5 * t + k];
  res->value = kacc_to_double(&accs[0]);
  res->e_max = e_max;
  res->e_min = e_min;
  res->n_bins = n_bins;
  res->f = f;
  res->status = ORC_OK;
  for (int k = 0; k < 5; ++k) res->count[k] = counts[k];
  free(accs);
  free(tcounts);
  free(bu);
  free(bm);
  return ORC_OK;
}

/* Plain FP64 dot product x.y on nthreads host threads: each thread one
 * fused multiply-add chain over its contiguous share, the thread sums added
 * in thread order (the CPU counterpart of the GPU comparator). */
double orc_dot_fp64(const double* x, const double* y, int64_t n, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  double* part = (double*)calloc((size_t)nthreads, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
  {
    int t = 0, nt = 1;
#ifdef _OPENMP
    t = omp_get_thread_num();
    nt = omp_get_num_threads();
#endif
    const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) s = fma(x[i], y[i], s);
    part[t] = s;
  }
  double s = 0.0;
  for (int t = 0; t < nthreads; ++t) s += part[t];
  free(part);
  return s;
}

/* Threads the OpenMP runtime would use (1 without OpenMP). */
int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
