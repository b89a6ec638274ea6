/*
 * CPU oracle for single-precision GEMM -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this code.  The product path (the CUDA library) never links it,
 * and this file includes no header of the product.
 *
 * What it computes (Section III-A, problem statement of the BLIS sgemm):
 *   C_out = alpha * op(A) * op(B) + beta * C_in
 * with A, B, C stored column-major with leading dimensions, op(X) = X or X^T,
 * and M, N, K arbitrary.  Written out element by element:
 *   C_out[i + j*ldc] = alpha * sum_{p=0}^{k-1} opA(i,p) * opB(p,j)
 *                      + beta * C_in[i + j*ldc]
 *   opA(i,p) = A[i + p*lda]  for transa in {N,n}
 *            = A[p + i*lda]  for transa in {T,t,C,c}   (real data: C == T)
 *   opB(p,j) = B[p + j*ldb]  for transb in {N,n}
 *            = B[j + p*ldb]  for transb in {T,t,C,c}
 * BLAS conventions the paper does not state, taken from reference BLAS:
 * beta == 0 does not read C; alpha == 0 or k == 0 does not read A and B.
 *
 * oracle_gemm_f64: each float product is exact in double; the sum runs in p
 *   order in double.  It also returns the componentwise acceptance bound
 *     bound_ij = 2*max(k,1)*2^-24*(|alpha| sum_p |opA(i,p)||opB(p,j)| + |beta||C_ij|).
 * oracle_gemm_f32: the naive float loop (p order, no fused multiply-add),
 *   then alpha*acc + beta*c in float.  A second reference.
 *
 * Split reference (the hi/lo BF16 representation of a float and the
 * per-row power-of-two scaling, not in the paper; it is the method's
 * precision-recovery step): restated from the IEEE-754 definitions.
 *   bf16 RNE:   round the float's 32-bit pattern to its top 16 bits, ties to
 *               even; NaN stays NaN; values >= 2^128(1-2^-9) become Inf.
 *   exponent:   scaling is for badly scaled K-vectors only.  With M the
 *               row's max |x|: e = 0 when M is 0, not finite, or in
 *               [2^-48, 2^48) (well scaled); otherwise e = frexp exponent of
 *               M, so that the scaled max lies in [0.5, 1).
 *   split:      x' = x * 2^-e (exact in double, one rounding to float),
 *               hi = bf16(x'), lo = bf16(x' - hi); non-finite x: lo = 0.
 *   three parts (for short k): hi and mid as hi and lo above, then
 *               lo3 = bf16(x' - hi - mid) (both subtractions exact in
 *               float); x' = hi + mid + lo3 exactly for normal x'; non-finite
 *               x: mid = lo3 = 0.
 *
 * Work is split across threads over output columns only; the arithmetic of
 * every output element is the plain loop above.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int op_is_trans(char t) {
  switch (t) {
    case 'N': case 'n': return 0;
    case 'T': case 't': case 'C': case 'c': return 1;
    default: return -1;
  }
}

int oracle_trans_code(char t) { return op_is_trans(t); }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static inline float opA(int ta, const float* A, int64_t lda, int64_t i, int64_t p) {
  return ta ? A[p + i * lda] : A[i + p * lda];
}
static inline float opB(int tb, const float* B, int64_t ldb, int64_t p, int64_t j) {
  return tb ? B[j + p * ldb] : B[p + j * ldb];
}

/* Block [i0,i1) x [j0,j1) of the FP64 result, written to out[(i-i0) + (j-j0)*ldo],
 * and the acceptance bound to bound[...] (same indexing) when bound != NULL.
 * Returns 0, or -1 on a bad transpose flag. */
int oracle_gemm_f64(char transa, char transb, int64_t m, int64_t n, int64_t k,
                    float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                    float beta, const float* C, int64_t ldc,
                    int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                    double* out, int64_t ldo, double* bound, int nthreads) {
  int ta = op_is_trans(transa), tb = op_is_trans(transb);
  if (ta < 0 || tb < 0) return -1;
  (void)m; (void)n;
  const int use_ab = (alpha != 0.0f) && (k > 0);
  const double unit = 2.0 * (double)(k > 1 ? k : 1) * ldexp(1.0, -24);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
  (void)nthreads;
#endif
  for (int64_t j = j0; j < j1; ++j) {
    for (int64_t i = i0; i < i1; ++i) {
      double s = 0.0, sabs = 0.0;
      if (use_ab) {
        for (int64_t p = 0; p < k; ++p) {
          double a = (double)opA(ta, A, lda, i, p);
          double b = (double)opB(tb, B, ldb, p, j);
          s += a * b;
          sabs += fabs(a) * fabs(b);
        }
      }
      double c = (beta != 0.0f) ? (double)C[i + j * ldc] : 0.0;
      double r = (use_ab ? (double)alpha * s : 0.0) + (beta != 0.0f ? (double)beta * c : 0.0);
      out[(i - i0) + (j - j0) * ldo] = r;
      if (bound) {
        double t = (use_ab ? fabs((double)alpha) * sabs : 0.0) + (beta != 0.0f ? fabs((double)beta) * fabs(c) : 0.0);
        bound[(i - i0) + (j - j0) * ldo] = unit * t;
      }
    }
  }
  return 0;
}

/* Naive FP32 loop; same block interface, float output. */
int oracle_gemm_f32(char transa, char transb, int64_t m, int64_t n, int64_t k,
                    float alpha, const float* A, int64_t lda, const float* B, int64_t ldb,
                    float beta, const float* C, int64_t ldc,
                    int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                    float* out, int64_t ldo, int nthreads) {
  int ta = op_is_trans(transa), tb = op_is_trans(transb);
  if (ta < 0 || tb < 0) return -1;
  (void)m; (void)n;
  const int use_ab = (alpha != 0.0f) && (k > 0);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#else
  (void)nthreads;
#endif
  for (int64_t j = j0; j < j1; ++j) {
    for (int64_t i = i0; i < i1; ++i) {
      float acc = 0.0f;
      if (use_ab) {
        for (int64_t p = 0; p < k; ++p) {
          float prod = opA(ta, A, lda, i, p) * opB(tb, B, ldb, p, j);
          acc = acc + prod;
        }
      }
      float r = use_ab ? alpha * acc : 0.0f;
      if (beta != 0.0f) {
        float bc = beta * C[i + j * ldc];
        r = r + bc;
      }
      out[(i - i0) + (j - j0) * ldo] = r;
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------- */
/* Split reference                                                          */
/* ---------------------------------------------------------------------- */

static inline uint32_t f2u(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static inline float u2f(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* IEEE round-to-nearest-even of a binary32 value to bfloat16 (8-bit exponent,
 * 7 stored mantissa bits): keep the top 16 bits, add half an ulp of the kept
 * part, and break exact ties towards the even kept pattern. */
uint16_t oracle_bf16_rne(float x) {
  uint32_t u = f2u(x);
  if ((u & 0x7F800000u) == 0x7F800000u && (u & 0x007FFFFFu) != 0) {
    return (uint16_t)((u >> 16) | 0x0040u); /* NaN: keep sign and payload top, force quiet */
  }
  uint32_t keep = u >> 16;
  uint32_t rest = u & 0xFFFFu;
  if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
  return (uint16_t)keep;
}

float oracle_bf16_to_f32(uint16_t h) { return u2f((uint32_t)h << 16); }

/* Scaling exponent of a K-vector from its max magnitude: 0 for 0, non-finite
 * or well-scaled maxima (2^-48 <= amax < 2^48), else the frexp exponent. */
int oracle_scale_exponent(float amax) {
  if (!(amax > 0.0f) || !isfinite(amax)) return 0;
  if ((double)amax >= ldexp(1.0, -48) && (double)amax < ldexp(1.0, 48)) return 0;
  int e;
  (void)frexp((double)amax, &e);
  return e;
}

/* x' = x * 2^-e: exact in double, then one rounding to float. */
float oracle_scaled(float x, int e) { return (float)ldexp((double)x, -e); }

void oracle_split(float xs, uint16_t* hi, uint16_t* lo) {
  uint16_t h = oracle_bf16_rne(xs);
  if (!isfinite(xs)) { *hi = h; *lo = 0; return; }
  float r = xs - oracle_bf16_to_f32(h);
  *hi = h;
  *lo = oracle_bf16_rne(r);
}

/* Third BF16 part of a scaled value: bf16((xs - hi) - mid). */
uint16_t oracle_split_third(float xs) {
  if (!isfinite(xs)) return 0;
  uint16_t h, m;
  oracle_split(xs, &h, &m);
  float r1 = xs - oracle_bf16_to_f32(h);
  float r2 = r1 - oracle_bf16_to_f32(m);
  return oracle_bf16_rne(r2);
}

/* Exhaustive check of the three-part split over [u0, u1): counts[0] finite
 * patterns with |x| >= 2^-100, counts[1] those where x != hi + mid + lo3
 * exactly (evaluated in double), counts[2] where xs - hi - mid is not exact
 * in float. */
void oracle_split3_exhaustive(uint64_t u0, uint64_t u1, int64_t* counts, int nthreads) {
  int64_t c0 = 0, c1 = 0, c2 = 0;
  const double tiny = ldexp(1.0, -100);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) reduction(+ : c0, c1, c2) num_threads(nthreads)
#else
  (void)nthreads;
#endif
  for (int64_t ui = (int64_t)u0; ui < (int64_t)u1; ++ui) {
    float x = u2f((uint32_t)ui);
    if (!isfinite(x) || fabs((double)x) < tiny) continue;
    if (fabs((double)x) >= ldexp(1.0, 128) * (1.0 - ldexp(1.0, -9))) continue; /* hi overflows */
    c0++;
    uint16_t h, m;
    oracle_split(x, &h, &m);
    uint16_t l = oracle_split_third(x);
    double hd = oracle_bf16_to_f32(h), md = oracle_bf16_to_f32(m), ld = oracle_bf16_to_f32(l);
    if (hd + md + ld != (double)x) c1++;
    float r1 = x - (float)hd;
    float r2 = r1 - (float)md;
    if ((double)r2 != (double)x - hd - md) c2++;
  }
  counts[0] = c0; counts[1] = c1; counts[2] = c2;
}

/* Split `rows` K-vectors of length k.  Element (r, p) of the operand is
 * X[r*sr + p*sp].  Writes e[r], hi[r*k + p], lo[r*k + p]. */
void oracle_split_rows3(int64_t rows, int64_t k, const float* X, int64_t sr, int64_t sp,
                        int32_t* e, uint16_t* hi, uint16_t* lo, uint16_t* lo3);

void oracle_split_rows(int64_t rows, int64_t k, const float* X, int64_t sr, int64_t sp,
                       int32_t* e, uint16_t* hi, uint16_t* lo) {
  oracle_split_rows3(rows, k, X, sr, sp, e, hi, lo, NULL);
}

/* As oracle_split_rows, plus the third part lo3[r*k + p] when lo3 != NULL. */
void oracle_split_rows3(int64_t rows, int64_t k, const float* X, int64_t sr, int64_t sp,
                        int32_t* e, uint16_t* hi, uint16_t* lo, uint16_t* lo3) {
  for (int64_t r = 0; r < rows; ++r) {
    float amax = 0.0f;
    int nonfinite = 0;
    for (int64_t p = 0; p < k; ++p) {
      float a = fabsf(X[r * sr + p * sp]);
      if (!isfinite(a)) nonfinite = 1;
      else if (a > amax) amax = a;
    }
    int ex = nonfinite ? 0 : oracle_scale_exponent(amax);
    e[r] = ex;
    for (int64_t p = 0; p < k; ++p) {
      float x = X[r * sr + p * sp];
      float xs = isfinite(x) ? oracle_scaled(x, ex) : x;
      oracle_split(xs, &hi[r * k + p], &lo[r * k + p]);
      if (lo3) lo3[r * k + p] = oracle_split_third(xs);
    }
  }
}

/* Exhaustive check of the split invariants over the bit patterns [u0, u1).
 * counts[0]: finite patterns checked
 * counts[1]: patterns where x - hi is not exact in float
 * counts[2]: patterns with |x| >= 2^-100 where |x - hi - lo| > 2^-17 |x|
 * counts[3]: finite patterns where hi has another sign than x (x != 0)
 * counts[4]: finite patterns where hi is Inf but |x| < 2^128 (1 - 2^-9)
 * counts[5]: finite patterns where hi is finite but |x| >= 2^128 (1 - 2^-9)
 * counts[6]: non-finite patterns with lo != 0 or hi not of the same class
 * counts[7]: max over |x| >= 2^-100 of |x - hi - lo| / |x|, times 2^40, as an integer */
void oracle_split_exhaustive(uint64_t u0, uint64_t u1, int64_t* counts, int nthreads) {
  int64_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const double ovf = ldexp(1.0, 128) * (1.0 - ldexp(1.0, -9));
  const double tiny = ldexp(1.0, -100);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#else
  (void)nthreads;
#endif
  {
    int64_t lc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
    for (int64_t ui = (int64_t)u0; ui < (int64_t)u1; ++ui) {
      float x = u2f((uint32_t)ui);
      uint16_t h, l;
      oracle_split(x, &h, &l);
      float hf = oracle_bf16_to_f32(h);
      if (!isfinite(x)) {
        int ok = (l == 0) && ((isnan(x) && isnan(hf)) || (isinf(x) && hf == x));
        if (!ok) lc[6]++;
        continue;
      }
      lc[0]++;
      double ax = fabs((double)x);
      if (ax >= ovf) { if (isfinite(hf)) lc[5]++; continue; }
      if (!isfinite(hf)) { lc[4]++; continue; }
      if (x != 0.0f && (signbit(hf) != signbit(x)) && hf != 0.0f) lc[3]++;
      double rd = (double)x - (double)hf;
      float rf = x - hf;
      if ((double)rf != rd) lc[1]++;
      if (ax >= tiny) {
        double err = fabs(rd - (double)oracle_bf16_to_f32(l));
        if (err > ldexp(ax, -17)) lc[2]++;
        int64_t q = (int64_t)ldexp(err / ax, 40);
        if (q > lc[7]) lc[7] = q;
      }
    }
#ifdef _OPENMP
#pragma omp critical
#endif
    {
      for (int t = 0; t < 7; ++t) c[t] += lc[t];
      if (lc[7] > c[7]) c[7] = lc[7];
    }
  }
  for (int t = 0; t < 8; ++t) counts[t] = c[t];
}
