/*
 * CPU oracle for GEMV, DOT and GER — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  The product (the CUDA library and its Python binding)
 * never calls it, and it shares no code, header or constant with the CUDA
 * path.
 *
 * What it computes is the plain definition of each operation in Singh &
 * Bassoy, "High Performance Level-1 and Level-2 BLAS" (arXiv 2108.02025),
 * Sec. 3.1:
 *
 *   DOT  (Def. DOT):   alpha += x . y  = alpha + sum_p x_p y_p
 *   GER  (Def. GEM):   C += x (outer) y,  C_ij += x_i y_j   (here with a scale
 *                      alpha: C_ij += x_i (alpha y_j))
 *   GEMV (Def. GEMV):  c += A x,  c_i += sum_j A_ij x_j     (here with a scale
 *                      alpha: c_i += alpha sum_j A_ij x_j)
 *
 * The paper's algorithms (Alg. 1 column-major GEMV, Alg. 2 row-major GEMV and
 * GER, Algs. 3/4 DOT) only reorder these sums, so the oracle is the
 * definition written out, with no blocking.  Two forms exist for each sum:
 *
 *   *_plain : FP64, summed in index order j = 0, 1, ..., n-1.
 *   *_acc   : FP64 compensated dot product "Dot2" (Ogita, Rump & Oishi,
 *             "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
 *             2005, Sec. 5): TwoProduct via fma() and Knuth's TwoSum, so the
 *             result is as accurate as if computed in twice the working
 *             precision and then rounded.  This is the reference the
 *             tolerances are measured against.
 *
 * FP32 inputs are widened to FP64 by the caller (exact).  GER is the one
 * operation computed in the working type, because it is a single rounding
 * per element: t_j = fl(alpha * y_j), C_ij = fma(x_i, t_j, C_ij).
 *
 * Matrix element (i, j) of an m x n matrix with leading dimension ld is
 * M[i*ld + j] in row-major layout (layout 0) and M[i + j*ld] in column-major
 * layout (layout 1).
 *
 * alpha == 0 in GEMV / GER returns at once without reading A, x, y or C (the
 * quick-return reading of the scale, which the paper does not have).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no fast-math, so
 * every operation is one IEEE round-to-nearest operation).  OpenMP only ever
 * splits independent outputs (rows of GEMV / GER, fixed chunks of the
 * compensated DOT), so results do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <omp.h>

#if defined(__FAST_MATH__)
#error "the oracle must not be built with fast-math"
#endif

static inline int64_t idx(int layout, int64_t i, int64_t j, int64_t ld) {
  return layout == 0 ? i * ld + j : i + j * ld;
}

/* Knuth's TwoSum: s + e == a + b exactly. */
static inline void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}

/* TwoProduct with an FMA: p + e == a * b exactly (no overflow/underflow). */
static inline void two_prod(double a, double b, double *p, double *e) {
  double q = a * b;
  *e = fma(a, b, -q);
  *p = q;
}

int oracle_threads(void) { return omp_get_max_threads(); }
void oracle_set_threads(int t) { if (t > 0) omp_set_num_threads(t); }

/* ---------------------------------------------------------------- GEMV --- */

/* Def. GEMV, summed in index order: c_i <- c_i + alpha * (sum_j A_ij x_j). */
void oracle_gemv_plain(int layout, int64_t m, int64_t n, double alpha, const double *A,
                       int64_t lda, const double *x, double *c) {
  if (m <= 0 || n <= 0 || alpha == 0.0) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s = s + A[idx(layout, i, j, lda)] * x[j];
    c[i] = c[i] + alpha * s;
  }
}

/* Def. GEMV with the row sum taken by Dot2, then c_i + alpha*s with one
   TwoProduct and one TwoSum. */
void oracle_gemv_acc(int layout, int64_t m, int64_t n, double alpha, const double *A,
                     int64_t lda, const double *x, double *c) {
  if (m <= 0 || n <= 0 || alpha == 0.0) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double p = 0.0, s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double h, r, q;
      two_prod(A[idx(layout, i, j, lda)], x[j], &h, &r);
      two_sum(p, h, &p, &q);
      s = s + (q + r);
    }
    /* the row sum is the unevaluated pair p + s; scale both parts so that
       the update is rounded once in effect */
    double ap, ae, u, ue;
    two_prod(alpha, p, &ap, &ae);
    ae = ae + alpha * s;
    two_sum(c[i], ap, &u, &ue);
    c[i] = u + (ue + ae);
  }
}

/* Condition-aware scale of row i: |c0_i| + |alpha| * sum_j |A_ij x_j|.  The
   GEMV tolerances are relative to this (a sum of non-negative terms, so the
   plain FP64 sum is accurate to n*u relative). */
void oracle_gemv_scale(int layout, int64_t m, int64_t n, double alpha, const double *A,
                       int64_t lda, const double *x, const double *c0, double *scale) {
  if (m <= 0) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s = s + fabs(A[idx(layout, i, j, lda)] * x[j]);
    scale[i] = fabs(c0[i]) + fabs(alpha) * s;
  }
}

/* ----------------------------------------------------------------- DOT --- */

/* Def. DOT, summed in index order: returns alpha + sum_p x_p y_p. */
double oracle_dot_plain(int64_t n, const double *x, const double *y, double alpha) {
  double s = 0.0;
  for (int64_t p = 0; p < n; ++p) s = s + x[p] * y[p];
  return alpha + s;
}

#define ORACLE_DOT_CHUNK ((int64_t)1 << 16)

/* Def. DOT by Dot2.  The index range is cut into fixed chunks of 2^16 (not
   tied to the thread count); each chunk yields an unevaluated pair (p, s)
   and the pairs are combined in chunk order with TwoSum, so the result is
   the same for any number of threads. */
double oracle_dot_acc(int64_t n, const double *x, const double *y, double alpha) {
  if (n <= 0) return alpha;
  int64_t nchunks = (n + ORACLE_DOT_CHUNK - 1) / ORACLE_DOT_CHUNK;
  double P = 0.0, S = 0.0;
#pragma omp parallel
  {
#pragma omp for ordered schedule(static, 1)
    for (int64_t k = 0; k < nchunks; ++k) {
      int64_t lo = k * ORACLE_DOT_CHUNK;
      int64_t hi = lo + ORACLE_DOT_CHUNK < n ? lo + ORACLE_DOT_CHUNK : n;
      double p = 0.0, s = 0.0;
      for (int64_t i = lo; i < hi; ++i) {
        double h, r, q;
        two_prod(x[i], y[i], &h, &r);
        two_sum(p, h, &p, &q);
        s = s + (q + r);
      }
#pragma omp ordered
      {
        double q;
        two_sum(P, p, &P, &q);
        S = S + (q + s);
      }
    }
  }
  double u, ue;
  two_sum(alpha, P, &u, &ue);
  return u + (ue + S);
}

/* Condition-aware scale of DOT: |alpha| + sum_p |x_p y_p|. */
double oracle_dot_scale(int64_t n, const double *x, const double *y, double alpha) {
  double s = 0.0;
  for (int64_t p = 0; p < n; ++p) s = s + fabs(x[p] * y[p]);
  return fabs(alpha) + s;
}

/* ----------------------------------------------------------------- GER --- */

/* Def. GEM with a scale: t_j = fl(alpha * y_j); C_ij = fma(x_i, t_j, C_ij),
   one rounding per element, FP64. */
void oracle_dger(int layout, int64_t m, int64_t n, double alpha, const double *x,
                 const double *y, double *C, int64_t ldc) {
  if (m <= 0 || n <= 0 || alpha == 0.0) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      double t = alpha * y[j];
      int64_t k = idx(layout, i, j, ldc);
      C[k] = fma(x[i], t, C[k]);
    }
  }
}

/* The same in FP32: t_j = fl32(alpha * y_j); C_ij = fmaf(x_i, t_j, C_ij). */
void oracle_sger(int layout, int64_t m, int64_t n, float alpha, const float *x,
                 const float *y, float *C, int64_t ldc) {
  if (m <= 0 || n <= 0 || alpha == 0.0f) return;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t j = 0; j < n; ++j) {
      float t = alpha * y[j];
      int64_t k = idx(layout, i, j, ldc);
      C[k] = fmaf(x[i], t, C[k]);
    }
  }
}

/* ------------------------------------------------- reduced precision --- */
/* Storage formats for A in the reduced-precision GEMV (not in the paper,
   which is FP64/FP32 only; written from the formats' definitions).

   BF16: the upper 16 bits of an IEEE binary32; round to nearest, ties to
   even, on the 16 dropped bits.  NaN inputs are not defined here.

   E4M3 (OCP 8-bit floating point, "E4M3"): sign, 4 exponent bits with bias
   7, 3 mantissa bits; normals (-1)^s 2^(e-7) (1 + m/8) for e in 1..15 except
   e = 15, m = 7 (NaN); subnormals (-1)^s 2^-6 (m/8); largest finite 448.
   Encoding: round to nearest, ties to even, and saturate to +-448 ("satfinite"). */

uint16_t oracle_bf16_encode(float v) {
  uint32_t u;
  memcpy(&u, &v, 4);
  const uint32_t bias = 0x7FFFu + ((u >> 16) & 1u);  /* ties to even */
  return (uint16_t)((u + bias) >> 16);
}

float oracle_bf16_decode(uint16_t q) {
  const uint32_t u = (uint32_t)q << 16;
  float v;
  memcpy(&v, &u, 4);
  return v;
}

double oracle_e4m3_decode(uint8_t q) {
  const int s = q >> 7, e = (q >> 3) & 15, m = q & 7;
  if (e == 15 && m == 7) return NAN;
  const double mag = e == 0 ? ldexp((double)m / 8.0, -6) : ldexp(1.0 + (double)m / 8.0, e - 7);
  return s ? -mag : mag;
}

/* round half to even of a non-negative value that is an exact multiple of
   a power of two (no rounding happens in the division below) */
static double rne(double a) {
  const double f = floor(a);
  const double r = a - f;
  if (r > 0.5) return f + 1.0;
  if (r < 0.5) return f;
  return fmod(f, 2.0) == 0.0 ? f : f + 1.0;
}

uint8_t oracle_e4m3_encode(double v) {
  if (isnan(v)) return 0x7F;
  const uint8_t sign = signbit(v) ? 0x80 : 0x00;
  const double a = fabs(v);
  if (a >= 448.0) return sign | 0x7E;              /* satfinite */
  if (a < ldexp(1.0, -6)) {                        /* subnormal grid 2^-9 */
    const double k = rne(a / ldexp(1.0, -9));      /* 0..8; 8 is the first normal */
    return sign | (uint8_t)k;
  }
  int e;
  frexp(a, &e);                                    /* a = f 2^e, f in [0.5, 1) */
  e -= 1;                                          /* a in [2^e, 2^(e+1)) */
  double k = rne(a / ldexp(1.0, e - 3));           /* 8..16 */
  if (k == 16.0) { k = 8.0; e += 1; }
  const int code = ((e + 7) << 3) | ((int)k - 8); /* a < 448 keeps code <= 0x7E */
  return sign | (uint8_t)code;
}

void oracle_bf16_encode_array(int64_t n, const float *v, uint16_t *q) {
  for (int64_t i = 0; i < n; ++i) q[i] = oracle_bf16_encode(v[i]);
}

void oracle_e4m3_encode_array(int64_t n, const double *v, uint8_t *q) {
  for (int64_t i = 0; i < n; ++i) q[i] = oracle_e4m3_encode(v[i]);
}

/* Per-row E4M3 quantisation of a row-major m x n FP32 matrix (leading
   dimension lda): s_i = fl32(amax_i / 448), q_ij = E4M3(fl32(A_ij / s_i)),
   all-zero rows get s_i = 0 and q = 0. */
void oracle_quantize_e4m3_rows(int64_t m, int64_t n, const float *A, int64_t lda, uint8_t *Q,
                               int64_t ldq, float *scales) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < m; ++i) {
    float amax = 0.0f;
    for (int64_t j = 0; j < n; ++j) {
      const float a = fabsf(A[i * lda + j]);
      if (a > amax) amax = a;
    }
    const float s = amax / 448.0f;
    scales[i] = s;
    for (int64_t j = 0; j < n; ++j)
      Q[i * ldq + j] = s == 0.0f ? 0 : oracle_e4m3_encode((double)(A[i * lda + j] / s));
  }
}

void oracle_e4m3_decode_array(int64_t n, const uint8_t *q, double *v) {
  for (int64_t i = 0; i < n; ++i) v[i] = oracle_e4m3_decode(q[i]);
}
