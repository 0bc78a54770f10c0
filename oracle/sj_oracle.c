/*
 * sj_oracle.c -- reference oracle for the embedding similarity join.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * What it computes (plain definitions, written out):
 *
 *   The join of Sec. 3.1 ("Two-way natural join") forms C = mat(A) mat(B)^T
 *   and keeps (a_i, b_j) exactly when C_ij > 0.  Here the rows of A and B are
 *   real-valued embeddings and C_ij = s_ij = <a_i, b_j>, the EXACT real value
 *   of the dot product of the stored float32 rows.  With one-hot rows this is
 *   the equi-join of Sec. 3.1 at any threshold tau in (0, 1].
 *
 *   top-k(i)      : the k indices j maximising s_ij, listed by (s desc, j asc);
 *                   when k > |B| the tail is padded with (-1, -inf).
 *   threshold(i)  : { j : s_ij >= tau }, listed by (i asc, j asc).
 *   reported score: RN_fp32(s_ij) (and RN_fp64(s_ij) for error reporting).
 *
 * How (the algorithm, in order):
 *   1. FP64 naive sum in index order.  A float32 x float32 product has at
 *      most 48 significant bits and magnitude >= 2^-298, so every product is
 *      exact in FP64; only the d-1 additions round.  Standard recursive
 *      summation bound: |sum - s| <= gamma_{d} * sum|p_k|, gamma_n = n u/(1-n u),
 *      u = 2^-53.  This gives an interval [lo, hi] that contains s.
 *   2. Wherever an interval does not decide (a rank near k, a tie, tau, or the
 *      float32 rounding of the score), s is recomputed EXACTLY: every product
 *      m_a*m_b*2^(e_a+e_b) is added into a fixed-point big integer (32-bit
 *      digits held in int64 slots, deferred carries), so the sum carries no
 *      rounding at all (Kulisch's long accumulator).
 *   3. Sort with the exact comparator; round exactly to float32 / float64
 *      with round-to-nearest-even.
 *
 * The contrastive (InfoNCE) oracle works in FP64 (the join's bfloat16 inputs
 * convert to FP64 exactly):
 *   S = A B^T / T,  l_i = logsumexp_j S_ij,  L = (1/N) sum_i (l_i - S_ii),
 *   dL/dS_ij = (P_ij - [i==j]) / N with P_ij = exp(S_ij - l_i),
 *   dA = (dL/dS) B / T,  dB = (dL/dS)^T A / T.
 * With the symmetric flag the column term (logsumexp over i) is added and the
 * two halves are averaged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Exact fixed-point accumulator                                            */
/* ------------------------------------------------------------------------ */

/* value = sum_t dig[t] * 2^(32 t + LSB_EXP).  A double t = M 2^(e - 53) with
 * an integer mantissa M < 2^53 has e - 53 >= -1126 (the smallest subnormal,
 * 2^-1074, is 2^52 2^-1126), and a product of two floats is an integer
 * < 2^48 times 2^(>= -298); LSB_EXP = -1152 lies below both, so every
 * product and any finite double tau add exactly.  The top is 2^384, far
 * above |s| < 2^288 and the clamped |tau| <= 2^290. */
#define NDIG 48
#define LSB_EXP (-1152)

typedef struct {
  int64_t dig[NDIG];
} exact_t;

static void ex_zero(exact_t *x) { memset(x, 0, sizeof *x); }

/* x += (neg ? -1 : 1) * mag * 2^e, with mag < 2^64 and e - LSB_EXP >= 0
 * (true for every caller: see LSB_EXP). */
static void ex_add(exact_t *x, int neg, uint64_t mag, int e) {
  int pos = e - LSB_EXP;
  int t = pos / 32, r = pos % 32;
  unsigned __int128 v = ((unsigned __int128)mag) << r;
  int64_t p0 = (int64_t)(uint64_t)(v & 0xffffffffu);
  int64_t p1 = (int64_t)(uint64_t)((v >> 32) & 0xffffffffu);
  int64_t p2 = (int64_t)(uint64_t)(v >> 64);
  if (neg) {
    x->dig[t] -= p0;
    x->dig[t + 1] -= p1;
    x->dig[t + 2] -= p2;
  } else {
    x->dig[t] += p0;
    x->dig[t + 1] += p1;
    x->dig[t + 2] += p2;
  }
}

/* Split a finite float into (sign, integer mantissa < 2^24, exponent). */
static void split_float(float f, int *neg, uint64_t *m, int *e) {
  int ex;
  double fr = frexp((double)f, &ex); /* f = fr * 2^ex, 0.5 <= |fr| < 1 */
  *neg = fr < 0;
  if (fr < 0) fr = -fr;
  /* fr * 2^24 is an integer for every float (including subnormals). */
  *m = (uint64_t)ldexp(fr, 24);
  *e = ex - 24;
}

/* Exact dot product of two float32 rows. */
static void exact_dot(const float *a, const float *b, int64_t d, exact_t *x) {
  ex_zero(x);
  for (int64_t k = 0; k < d; ++k) {
    if (a[k] == 0.0f || b[k] == 0.0f) continue;
    int na, nb, ea, eb;
    uint64_t ma, mb;
    split_float(a[k], &na, &ma, &ea);
    split_float(b[k], &nb, &mb, &eb);
    ex_add(x, na ^ nb, ma * mb, ea + eb);
  }
}

/* x -= t for a finite double t with |t| < 2^300. */
static void ex_sub_double(exact_t *x, double t) {
  if (t == 0.0) return;
  int ex;
  double fr = frexp(t, &ex);
  int neg = fr < 0;
  if (fr < 0) fr = -fr;
  uint64_t m = (uint64_t)ldexp(fr, 53);
  ex_add(x, !neg, m, ex - 53);
}

/* Propagate carries.  On return dig[0..NDIG-2] lie in [0, 2^32) and the top
 * digit carries the sign. */
static void ex_carry(exact_t *x) {
  for (int t = 0; t < NDIG - 1; ++t) {
    int64_t v = x->dig[t];
    int64_t low = v & (int64_t)0xffffffff; /* v mod 2^32, in [0, 2^32) */
    int64_t c = (v - low) / (int64_t)4294967296LL;
    x->dig[t] = low;
    x->dig[t + 1] += c;
  }
}

/* Sign of x and |x| as NDIG base-2^32 digits (little endian). */
static int ex_sign_mag(const exact_t *in, uint32_t mag[NDIG]) {
  exact_t x = *in;
  ex_carry(&x);
  int sign = 0;
  if (x.dig[NDIG - 1] < 0) {
    sign = -1;
    for (int t = 0; t < NDIG; ++t) x.dig[t] = -x.dig[t];
    ex_carry(&x);
  } else {
    for (int t = NDIG - 1; t >= 0; --t)
      if (x.dig[t] != 0) { sign = 1; break; }
  }
  for (int t = 0; t < NDIG; ++t) mag[t] = (uint32_t)x.dig[t];
  return sign;
}

/* sign(a - b) */
static int ex_cmp(const exact_t *a, const exact_t *b) {
  exact_t d;
  for (int t = 0; t < NDIG; ++t) d.dig[t] = a->dig[t] - b->dig[t];
  uint32_t mag[NDIG];
  return ex_sign_mag(&d, mag);
}

static int mag_bit(const uint32_t mag[NDIG], int i) {
  if (i < 0 || i >= 32 * NDIG) return 0;
  return (mag[i / 32] >> (i % 32)) & 1u;
}

/* Round x to the nearest p-bit binary float (ties to even) whose quantum
 * exponent is at least qmin; return it as a double (exact for p <= 53).
 * p = 24, qmin = -149 gives float32; p = 53, qmin = -1074 gives float64. */
static double ex_round(const exact_t *x, int p, int qmin) {
  uint32_t mag[NDIG];
  int sign = ex_sign_mag(x, mag);
  if (sign == 0) return 0.0;
  int top = -1;
  for (int i = 32 * NDIG - 1; i >= 0; --i)
    if (mag_bit(mag, i)) { top = i; break; }
  int q = top + LSB_EXP - (p - 1);   /* exponent of the last kept bit */
  if (q < qmin) q = qmin;
  int qb = q - LSB_EXP;               /* its bit index */
  uint64_t M = 0;
  for (int i = top; i >= qb; --i) M = (M << 1) | (uint64_t)mag_bit(mag, i);
  int round_bit = mag_bit(mag, qb - 1);
  int sticky = 0;
  for (int i = qb - 2; i >= 0; --i)
    if (mag_bit(mag, i)) { sticky = 1; break; }
  if (round_bit && (sticky || (M & 1u))) M += 1;
  double r = ldexp((double)M, q);
  if (p == 24 && r > 3.4028234663852886e38) r = INFINITY;
  return sign < 0 ? -r : r;
}

/* ------------------------------------------------------------------------ */
/* Step 1: FP64 naive sum and its enclosure                                  */
/* ------------------------------------------------------------------------ */

/* Interval [lo, hi] containing the exact <a, b>. */
static void fp64_enclose(const float *a, const float *b, int64_t d, double *lo,
                         double *hi) {
  const double u = ldexp(1.0, -53);
  double s = 0.0, sa = 0.0;
  for (int64_t k = 0; k < d; ++k) {
    double p = (double)a[k] * (double)b[k]; /* exact */
    s = s + p;
    sa = sa + fabs(p);
  }
  double n = (double)(d + 2);
  double gamma = n * u / (1.0 - n * u);
  /* Recursive summation error <= gamma_{d-1} sum|p|; sa itself is computed
   * with relative error <= gamma_{d-1}, the factor (1 + 4 gamma) covers it;
   * 4u(|s| + sa) covers the rounding of lo and hi themselves; the 2^-1000
   * floor keeps the interval closed when everything is zero. */
  double w = gamma * sa * (1.0 + 4.0 * gamma) + 4.0 * u * (fabs(s) + sa) +
             ldexp(1.0, -1000);
  *lo = s - w;
  *hi = s + w;
}

/* The enclosure of every pair of a join (step 1 alone): lo/hi are nA x nB,
 * row-major; the exact s_ij lies in [lo_ij, hi_ij]. */
void sjo_enclose_all(const float *A, const float *B, int64_t nA, int64_t nB, int64_t d,
                     double *lo, double *hi) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nA; ++i)
    for (int64_t j = 0; j < nB; ++j)
      fp64_enclose(A + i * d, B + j * d, d, &lo[i * nB + j], &hi[i * nB + j]);
}

/* ------------------------------------------------------------------------ */
/* Top-k                                                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t j;
  exact_t v;
} cand_t;

static int cmp_desc_double(const void *x, const void *y) {
  double a = *(const double *)x, b = *(const double *)y;
  return (a < b) - (a > b);
}

static int cmp_cand(const void *x, const void *y) {
  const cand_t *a = (const cand_t *)x, *b = (const cand_t *)y;
  int c = ex_cmp(&a->v, &b->v);
  if (c != 0) return -c;                 /* larger exact score first */
  return (a->j > b->j) - (a->j < b->j);  /* then lower right index */
}

/* One left row: writes k indices and scores; returns the number of exact
 * evaluations it needed.  Buffers lo/hi/tmp have room for nB doubles. */
static int64_t topk_row(const float *a, const float *B, int64_t nB, int64_t d,
                        int k, int64_t *idx, float *s32, double *s64,
                        double *lo, double *hi, double *tmp) {
  int64_t kk = (int64_t)k < nB ? (int64_t)k : nB;
  for (int64_t r = 0; r < k; ++r) {
    idx[r] = -1;
    s32[r] = -INFINITY;
    s64[r] = -INFINITY;
  }
  if (kk == 0) return 0;
  for (int64_t j = 0; j < nB; ++j) fp64_enclose(a, B + j * d, d, &lo[j], &hi[j]);
  /* k-th largest lower end: at least kk rows have s >= Lk, so any row with
   * hi < Lk has kk rows strictly above it and cannot be in the top-k. */
  memcpy(tmp, lo, (size_t)nB * sizeof(double));
  qsort(tmp, (size_t)nB, sizeof(double), cmp_desc_double);
  double Lk = tmp[kk - 1];
  int64_t nc = 0;
  for (int64_t j = 0; j < nB; ++j) nc += hi[j] >= Lk;
  cand_t *c = (cand_t *)malloc((size_t)nc * sizeof(cand_t));
  int64_t t = 0;
  for (int64_t j = 0; j < nB; ++j)
    if (hi[j] >= Lk) {
      c[t].j = j;
      exact_dot(a, B + j * d, d, &c[t].v);
      ++t;
    }
  qsort(c, (size_t)nc, sizeof(cand_t), cmp_cand);
  for (int64_t r = 0; r < kk; ++r) {
    idx[r] = c[r].j;
    s32[r] = (float)ex_round(&c[r].v, 24, -149);
    s64[r] = ex_round(&c[r].v, 53, -1074);
  }
  free(c);
  return nc;
}

/* rows == NULL: all rows 0..nrows-1; otherwise the listed left rows.
 * Outputs are nrows x k.  Returns the total number of exact evaluations. */
int64_t sjo_topk(const float *A, const float *B, int64_t nB, int64_t d, int k,
                 const int64_t *rows, int64_t nrows, int64_t *out_idx,
                 float *out_s32, double *out_s64) {
  int64_t total = 0;
#pragma omp parallel reduction(+ : total)
  {
    size_t n = (size_t)(nB > 0 ? nB : 1);
    double *lo = (double *)malloc(n * sizeof(double));
    double *hi = (double *)malloc(n * sizeof(double));
    double *tmp = (double *)malloc(n * sizeof(double));
#pragma omp for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
      int64_t i = rows ? rows[r] : r;
      total += topk_row(A + i * d, B, nB, d, k, out_idx + r * k, out_s32 + r * k,
                        out_s64 + r * k, lo, hi, tmp);
    }
    free(lo);
    free(hi);
    free(tmp);
  }
  return total;
}

/* ------------------------------------------------------------------------ */
/* Threshold                                                                 */
/* ------------------------------------------------------------------------ */

/* Decide s >= tau and the rounded score for one pair.  Returns 1 if in. */
static int thr_pair(const float *a, const float *b, int64_t d, double tau,
                    float *s32, double *s64, int64_t *n_exact) {
  double lo, hi;
  fp64_enclose(a, b, d, &lo, &hi);
  int in;
  int have_exact = 0;
  exact_t x;
  if (lo >= tau) {
    in = 1;
  } else if (hi < tau) {
    return 0;
  } else {
    exact_dot(a, b, d, &x);
    have_exact = 1;
    ++*n_exact;
    exact_t y = x;
    ex_sub_double(&y, tau);
    uint32_t mag[NDIG];
    in = ex_sign_mag(&y, mag) >= 0;
    if (!in) return 0;
  }
  /* RN is monotone: if both ends of the enclosure round to the same float,
   * so does every value between them, s included. */
  if (!have_exact && (float)lo == (float)hi) {
    *s32 = (float)lo;
  } else {
    if (!have_exact) {
      exact_dot(a, b, d, &x);
      have_exact = 1;
      ++*n_exact;
    }
    *s32 = (float)ex_round(&x, 24, -149);
  }
  if (s64) {
    if (!have_exact) {
      exact_dot(a, b, d, &x);
      ++*n_exact;
    }
    *s64 = ex_round(&x, 53, -1074);
  }
  return in;
}

/* Pass 1 (out_j == NULL): count pairs per listed row into row_count.
 * Pass 2: write pairs of listed row r at offset row_offset[r].
 * tau outside [-2^290, 2^290] is clamped by the caller. */
int64_t sjo_threshold(const float *A, const float *B, int64_t nB, int64_t d,
                      double tau, const int64_t *rows, int64_t nrows,
                      int64_t *row_count, const int64_t *row_offset,
                      int64_t *out_j, float *out_s32, double *out_s64) {
  int64_t total_exact = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total_exact)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows ? rows[r] : r;
    int64_t cnt = 0, ne = 0;
    for (int64_t j = 0; j < nB; ++j) {
      float s32;
      double s64;
      if (thr_pair(A + i * d, B + j * d, d, tau, &s32, out_s64 ? &s64 : NULL, &ne)) {
        if (out_j) {
          int64_t o = row_offset[r] + cnt;
          out_j[o] = j;
          out_s32[o] = s32;
          if (out_s64) out_s64[o] = s64;
        }
        ++cnt;
      }
    }
    if (!out_j) row_count[r] = cnt;
    total_exact += ne;
  }
  return total_exact;
}

/* ------------------------------------------------------------------------ */
/* Exact helpers exposed for the pin tests                                    */
/* ------------------------------------------------------------------------ */

/* Exact dot product as sign and NDIG magnitude digits; value =
 * sign * sum mag[t] 2^(32 t + LSB_EXP).  Returns LSB_EXP through *lsb_exp. */
int sjo_exact_dot(const float *a, const float *b, int64_t d, uint32_t *mag,
                  int *lsb_exp, int *ndig) {
  exact_t x;
  exact_dot(a, b, d, &x);
  *lsb_exp = LSB_EXP;
  *ndig = NDIG;
  return ex_sign_mag(&x, mag);
}

/* Exact <a, b> - t for a finite double t (|t| <= 2^290), as sign and NDIG
 * magnitude digits like sjo_exact_dot: the difference every threshold
 * decision takes the sign of. */
int sjo_exact_dot_minus(const float *a, const float *b, int64_t d, double t, uint32_t *mag) {
  exact_t x;
  exact_dot(a, b, d, &x);
  ex_sub_double(&x, t);
  return ex_sign_mag(&x, mag);
}

/* RN_fp32 and RN_fp64 of the exact dot product. */
void sjo_exact_dot_rounded(const float *a, const float *b, int64_t d, float *s32,
                           double *s64) {
  exact_t x;
  exact_dot(a, b, d, &x);
  *s32 = (float)ex_round(&x, 24, -149);
  *s64 = ex_round(&x, 53, -1074);
}

int sjo_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Contrastive (InfoNCE) join, FP64                                          */
/* ------------------------------------------------------------------------ */

static double dot_f64(const double *a, const double *b, int64_t d) {
  double s = 0.0;
  for (int64_t k = 0; k < d; ++k) s += a[k] * b[k];
  return s;
}

/* logsumexp over S_i. for one row i (row_of_A != 0) or over S_.j for one
 * column (row_of_A == 0), S = A B^T / T. */
static double lse_line(const double *A, const double *B, int64_t N, int64_t d,
                       double T, int64_t i, int row_of_A) {
  double m = -INFINITY;
  for (int64_t j = 0; j < N; ++j) {
    double s = row_of_A ? dot_f64(A + i * d, B + j * d, d) / T
                        : dot_f64(A + j * d, B + i * d, d) / T;
    if (s > m) m = s;
  }
  double acc = 0.0;
  for (int64_t j = 0; j < N; ++j) {
    double s = row_of_A ? dot_f64(A + i * d, B + j * d, d) / T
                        : dot_f64(A + j * d, B + i * d, d) / T;
    acc += exp(s - m);
  }
  return m + log(acc);
}

/* Full FP64 InfoNCE forward + backward for N paired rows (positives on the
 * diagonal).  Inputs are FP64 (bfloat16 data converts to FP64 exactly).
 * lse_col may be NULL when sym == 0.  g = dLoss upstream. */
void sjo_infonce(const double *A, const double *B, int64_t N, int64_t d,
                 double T, int sym, double g, double *loss, double *lse_row,
                 double *lse_col, double *dA, double *dB) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; ++i) lse_row[i] = lse_line(A, B, N, d, T, i, 1);
  if (sym) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < N; ++j) lse_col[j] = lse_line(A, B, N, d, T, j, 0);
  }
  double lr = 0.0, lc = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    double sii = dot_f64(A + i * d, B + i * d, d) / T;
    lr += lse_row[i] - sii;
    if (sym) lc += lse_col[i] - sii;
  }
  lr /= (double)N;
  lc /= (double)N;
  *loss = sym ? 0.5 * (lr + lc) : lr;
  if (!dA && !dB) return;
  /* G_ij = dLoss/dS_ij; dS/dA_i = B_j / T. */
  double w = sym ? 0.5 : 1.0;
  if (dA) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < N; ++i) {
      for (int64_t k = 0; k < d; ++k) dA[i * d + k] = 0.0;
      for (int64_t j = 0; j < N; ++j) {
        double s = dot_f64(A + i * d, B + j * d, d) / T;
        double G = (exp(s - lse_row[i]) - (i == j ? 1.0 : 0.0)) / (double)N;
        if (sym) G += (exp(s - lse_col[j]) - (i == j ? 1.0 : 0.0)) / (double)N;
        G *= w * g;
        for (int64_t k = 0; k < d; ++k) dA[i * d + k] += G * B[j * d + k] / T;
      }
    }
  }
  if (dB) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < N; ++j) {
      for (int64_t k = 0; k < d; ++k) dB[j * d + k] = 0.0;
      for (int64_t i = 0; i < N; ++i) {
        double s = dot_f64(A + i * d, B + j * d, d) / T;
        double G = (exp(s - lse_row[i]) - (i == j ? 1.0 : 0.0)) / (double)N;
        if (sym) G += (exp(s - lse_col[j]) - (i == j ? 1.0 : 0.0)) / (double)N;
        G *= w * g;
        for (int64_t k = 0; k < d; ++k) dB[j * d + k] += G * A[i * d + k] / T;
      }
    }
  }
}

/* Row statistics for sampled rows of a large contrastive join: the row
 * logsumexp and the one-directional dA row, which depend on row i alone. */
void sjo_infonce_rows(const double *A, const double *B, int64_t N, int64_t d,
                      double T, double g, const int64_t *rows, int64_t nrows,
                      double *lse_row, double *dA_rows) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    double l = lse_line(A, B, N, d, T, i, 1);
    lse_row[r] = l;
    if (!dA_rows) continue;
    double *out = dA_rows + r * d;
    for (int64_t k = 0; k < d; ++k) out[k] = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double s = dot_f64(A + i * d, B + j * d, d) / T;
      double G = g * (exp(s - l) - (i == j ? 1.0 : 0.0)) / (double)N;
      for (int64_t k = 0; k < d; ++k) out[k] += G * B[j * d + k] / T;
    }
  }
}
