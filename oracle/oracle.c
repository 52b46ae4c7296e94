/*
 * FP64 CPU oracle for the 1D periodic NUFFT / INUFFT of Gumerov & Duraiswami
 * ("Fast Multipole Method based filtering of non-uniformly sampled data").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load, call or execute this
 * file.  The product library (paper_1611_09379_gb300) never uses it, and it
 * shares no code, header, table or helper with the CUDA path.
 *
 * Every routine evaluates a DEFINITION directly, O(N*M), in binary64, with
 * the only numerical care being what the definition itself needs:
 *   - phases n*y are formed with an exact two-product (fma) so that
 *     e^{i n y} is evaluated for the exact binary64 y (reading c8);
 *   - differences y - x_k, with x_k = 2*pi*k/N irrational, use a
 *     double-double 2*pi so the small differences keep full relative
 *     precision (reading c8, c7);
 *   - sums are Neumaier-compensated (reading c17).
 * The conventions: frequencies n = 0..N-1 (Eq. p1, one-sided); the
 * unscaled inverse DFT maps c -> f, f_k = sum_n c_n e^{i n x_k}; the DFT is
 * c_n = (1/N) sum_k f_k e^{-i n x_k} (Eq. p1).
 *
 * Parity status per routine (what pins it is in tests/test_oracle_pins.py):
 *   orc_nudft_fwd    pinned: c=e_m closed form, f==1, dense Eq. p2 matrix
 *   orc_kernel_fwd   pinned: f==1 (paper's own test, Sec. 3.1), cot-sum
 *                    identity, agreement with orc_nudft_fwd
 *   orc_nudft_adj    pinned: dot-product test against orc_nudft_fwd
 *   orc_kernel_adj   pinned: agreement with orc_nudft_adj
 *   orc_logsin_*     pinned: equispaced product identity
 *   orc_inverse_f    pinned: round trip and dense solve at N <= 256
 *   orc_kernel_fwd_plain  the paper's "straightforward method" of Sec. 3.1
 *                    (Eq. p4 in plain binary64, no compensation), the
 *                    measuring stick of the threshold error eps_th(N);
 *                    pinned: agrees with orc_kernel_fwd within the rounding
 *                    bound of its uncompensated differences
 *   orc_inverse_absf pinned: equals sum_j |L_kj| |g_j| of the dense Lagrange
 *                    matrix at N <= 64 (inverse of the dense A, numpy)
 *   orc_fft          pinned: direct DFT and numpy.fft
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* 2*pi as an unevaluated sum hi + lo (hi = fl(2 pi)). */
static const double TWO_PI_HI = 6.283185307179586232e+00;
static const double TWO_PI_LO = 2.449293598294706e-16;

/* ---------- compensated summation (Neumaier) ---------- */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static inline double nval(const nsum *a) { return a->s + a->c; }

/* e^{i n y} for integer n and binary64 y, with n*y formed exactly as p + e. */
static inline void expi_ny(int64_t n, double y, double *re, double *im) {
  double nd = (double)n;
  double p = nd * y;
  double e = fma(nd, y, -p);
  double cp = cos(p), sp = sin(p);
  /* e^{i e} = 1 + i e - e^2/2 (|e| <= 2^-30, so the rest is far below ulp) */
  double er = 1.0 - 0.5 * e * e, ei = e;
  *re = cp * er - sp * ei;
  *im = cp * ei + sp * er;
}

/* 2 pi / N as an unevaluated sum hi + lo with |lo| <= ulp(hi) / 2 and an
 * error of order 2^-106 relative: hi = fl(2 pi_hi / N); the remainder
 * 2 pi_hi - hi N is exact (fma of a correctly rounded quotient), so
 * lo = (remainder + 2 pi_lo) / N.  For N a power of two, lo = 2 pi_lo / N. */
static inline void two_pi_over(int64_t N, double *hi, double *lo) {
  double nd = (double)N;
  double h = TWO_PI_HI / nd;
  double rem = fma(-h, nd, TWO_PI_HI);
  *hi = h;
  *lo = (rem + TWO_PI_LO) / nd;
}

/* Unwrapped difference y - x~ with x~ = 2 pi kk / N for an integer kk
 * (kk = k or a periodic image k +- N), formed with a double-double 2 pi/N and
 * an exact two-product so that a small result keeps full relative precision. */
static inline double diff_y_grid(double y, int64_t kk, int64_t N) {
  double hhi, hlo;
  two_pi_over(N, &hhi, &hlo);
  double kd = (double)kk;
  double P = kd * hhi;
  double E = fma(kd, hhi, -P);
  return ((y - P) - E) - kd * hlo;
}

/* t = y - x_k wrapped into [-pi, pi) (the kernel is 2 pi periodic, Sec. 2.1):
 * the periodic image of x_k is chosen on the integer index before the
 * compensated difference, so no rounded difference is wrapped afterwards. */
static inline double diff_y_xk(double y, int64_t k, int64_t N) {
  double rough = y - (double)k * (TWO_PI_HI / (double)N);
  int64_t kk = k;
  if (rough >= 0.5 * TWO_PI_HI) kk += N;
  else if (rough < -0.5 * TWO_PI_HI) kk -= N;
  return diff_y_grid(y, kk, N);
}

/* a - b for two points of [0, 2 pi), wrapped into [-pi, pi): the exact
 * difference is held as a two-sum before 2 pi (double-double) is removed. */
static inline double wrap_diff(double a, double b) {
  double s = a - b;
  double bb = s - a;
  double err = (a - (s - bb)) + (-b - bb); /* a - b = s + err exactly */
  if (s >= 0.5 * TWO_PI_HI) return (s - TWO_PI_HI) + (err - TWO_PI_LO);
  if (s < -0.5 * TWO_PI_HI) return (s + TWO_PI_HI) + (err + TWO_PI_LO);
  return s + err;
}

/* cos and sin of N y / 2 with N y formed exactly as p + e (two-product;
 * e = 0 when N is a power of two): sin(p/2 + e/2) by the expansion of e^{i e/2}
 * to second order (|e| <= ulp(N y), so the rest is below the rounding). */
static inline void half_ny(double y, int64_t N, double *c, double *s) {
  double nd = (double)N;
  double p = nd * y;
  double e = fma(nd, y, -p);
  double a = 0.5 * p, h = 0.5 * e;
  double ca = cos(a), sa = sin(a);
  double er = 1.0 - 0.5 * h * h;
  *c = ca * er - sa * h;
  *s = sa * er + ca * h;
}

/* F_j = (e^{i N y} - 1)/N  (Eq. p5), written as (2i/N) e^{i N y/2} sin(N y/2). */
static inline void F_of_y(double y, int64_t N, double *re, double *im) {
  double c, s;
  half_ny(y, N, &c, &s);
  *re = -2.0 * s * s / (double)N;
  *im = 2.0 * c * s / (double)N;
}

/* G(t) = 1/(e^{it}-1) = -(1 + i cot(t/2))/2  (Eq. p5), t in [-pi, pi), t != 0 */
static inline void G_of_t(double t, double *re, double *im) {
  *re = -0.5;
  *im = -0.5 / tan(0.5 * t);
}

#define IDX(i) (idx ? idx[i] : (int64_t)(i))

/* Forward NUDFT, the definition (Eq. p1 at y_j):
 *   g_j = sum_{n=0}^{N-1} c_n e^{i n y_j}.
 * c: interleaved complex [N]; y: [M]; idx: target subset (NULL = all);
 * g: interleaved complex [nidx]. */
void orc_nudft_fwd(const double *c, int64_t N, const double *y, int64_t M,
                   const int64_t *idx, int64_t nidx, double *g) {
  (void)M;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    double yj = y[IDX(i)];
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t n = 0; n < N; ++n) {
      double er, ei;
      expi_ny(n, yj, &er, &ei);
      nadd(&sr, c[2 * n] * er - c[2 * n + 1] * ei);
      nadd(&si, c[2 * n] * ei + c[2 * n + 1] * er);
    }
    g[2 * i] = nval(&sr);
    g[2 * i + 1] = nval(&si);
  }
}

/* Forward interpolation in the paper's factored form (Eq. p2, p4, p5):
 *   g_j = sum_k F_j G(y_j - x_k) f_k,
 * with the exact-hit limit F_j G(t) -> 1 at t = 0 (reading c7).
 * f: samples on the uniform grid [N]. */
void orc_kernel_fwd(const double *f, int64_t N, const double *y, int64_t M,
                    const int64_t *idx, int64_t nidx, double *g) {
  (void)M;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    double yj = y[IDX(i)];
    double Fr, Fi;
    F_of_y(yj, N, &Fr, &Fi);
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
      double t = diff_y_xk(yj, k, N);
      double Kr, Ki;
      /* K_jk = (1/N) sum_n e^{i n t} (Eq. p2) is 1 to binary64 resolution when
       * N|t| < 2^-60; this covers the exact hit t = 0 (reading c7) and
       * subnormal t, where t/2 underflows. */
      if (fabs(t) * (double)N < 0x1p-60) { Kr = 1.0; Ki = 0.0; }
      else {
        double Gr, Gi;
        G_of_t(t, &Gr, &Gi);
        Kr = Fr * Gr - Fi * Gi;
        Ki = Fr * Gi + Fi * Gr;
      }
      nadd(&sr, Kr * f[2 * k] - Ki * f[2 * k + 1]);
      nadd(&si, Kr * f[2 * k + 1] + Ki * f[2 * k]);
    }
    g[2 * i] = nval(&sr);
    g[2 * i + 1] = nval(&si);
  }
}

/* The paper's "straightforward method" (Sec. 3.1): g_j = sum_k K_jk f_k with
 * the matrix entry of Eq. p4 evaluated literally in binary64,
 *   K_jk = ((e^{i N y_j} - 1) / N) / (e^{i (y_j - x_k)} - 1),
 * x_k = k fl(2 pi / N), the difference y_j - x_k, both exponentials (libm
 * cos / sin), the complex quotient and the sum all in plain binary64, no
 * compensation.  Its error for f = 1 is what the paper calls the machine
 * precision threshold eps_th(N).  A point that hits a grid point exactly
 * (t == 0) takes K = 1 (reading c7). */
void orc_kernel_fwd_plain(const double *f, int64_t N, const double *y, int64_t M,
                          const int64_t *idx, int64_t nidx, double *g) {
  (void)M;
  const double h = TWO_PI_HI / (double)N;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    double yj = y[IDX(i)];
    double a = (double)N * yj;
    double nr = (cos(a) - 1.0) / (double)N, ni = sin(a) / (double)N;
    double sr = 0.0, si = 0.0;
    for (int64_t k = 0; k < N; ++k) {
      double t = yj - (double)k * h;
      double Kr, Ki;
      if (t == 0.0) { Kr = 1.0; Ki = 0.0; }
      else {
        double dr = cos(t) - 1.0, di = sin(t);
        double den = dr * dr + di * di;
        Kr = (nr * dr + ni * di) / den;
        Ki = (ni * dr - nr * di) / den;
      }
      sr += Kr * f[2 * k] - Ki * f[2 * k + 1];
      si += Kr * f[2 * k + 1] + Ki * f[2 * k];
    }
    g[2 * i] = sr;
    g[2 * i + 1] = si;
  }
}

/* h(y) = sum_k f_k cot((y - x_k)/2) for real f, skipping exact hits: the
 * quantity the fast method approximates (Eq. p9).  Exposed so the closed
 * form sum_k cot((y - 2 pi k/N)/2) = N cot(N y/2) can pin the kernel part. */
void orc_cot_sum(const double *f, int64_t N, const double *y, int64_t M, double *h) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t j = 0; j < M; ++j) {
    nsum s = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
      double t = diff_y_xk(y[j], k, N);
      if (t != 0.0) nadd(&s, f[k] / tan(0.5 * t));
    }
    h[j] = nval(&s);
  }
}

/* Adjoint NUDFT, the definition: c'_n = sum_j e^{-i n y_j} g_j.
 * idx selects output frequencies (NULL = all N). */
void orc_nudft_adj(const double *g, const double *y, int64_t M, int64_t N,
                   const int64_t *idx, int64_t nidx, double *c) {
  (void)N;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t n = IDX(i);
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t j = 0; j < M; ++j) {
      double er, ei;
      expi_ny(n, y[j], &er, &ei);
      ei = -ei; /* e^{-i n y} */
      nadd(&sr, g[2 * j] * er - g[2 * j + 1] * ei);
      nadd(&si, g[2 * j] * ei + g[2 * j + 1] * er);
    }
    c[2 * i] = nval(&sr);
    c[2 * i + 1] = nval(&si);
  }
}

/* Adjoint interpolation in factored form (conjugate transpose of Eq. p4):
 *   u_k = sum_j conj(F_j) G(x_k - y_j) g_j, exact hits contributing g_j.
 * Output on the uniform grid (all N points or the idx subset). */
void orc_kernel_adj(const double *g, const double *y, int64_t M, int64_t N,
                    const int64_t *idx, int64_t nidx, double *u) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t k = IDX(i);
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t j = 0; j < M; ++j) {
      double t = -diff_y_xk(y[j], k, N); /* x_k - y_j */
      double Kr, Ki;
      if (fabs(t) * (double)N < 0x1p-60) { Kr = 1.0; Ki = 0.0; } /* as in orc_kernel_fwd */
      else {
        double Fr, Fi, Gr, Gi;
        F_of_y(y[j], N, &Fr, &Fi);
        Fi = -Fi;
        G_of_t(t, &Gr, &Gi);
        Kr = Fr * Gr - Fi * Gi;
        Ki = Fr * Gi + Fi * Gr;
      }
      nadd(&sr, Kr * g[2 * j] - Ki * g[2 * j + 1]);
      nadd(&si, Kr * g[2 * j + 1] + Ki * g[2 * j]);
    }
    u[2 * i] = nval(&sr);
    u[2 * i + 1] = nval(&si);
  }
}

/* log-sums for the inverse coefficients (Eq. p8, reading c4):
 *   lamC_k = sum_l log|2 sin((x_k - y_l)/2)|,  nC_k = #{l : y_l > x_k}
 * so that C_k = (-1)^(k + nC_k) * 2^{-M} * exp(lamC_k) (exact hit: C_k = 0,
 * reported as lamC_k = -inf).  k runs over idx (NULL = 0..N-1). */
void orc_logsin_C(const double *y, int64_t M, int64_t N, const int64_t *idx,
                  int64_t nidx, double *lamC, int64_t *nC) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t k = IDX(i);
    nsum s = {0, 0};
    int64_t cnt = 0, hit = 0;
    for (int64_t l = 0; l < M; ++l) {
      double t = -diff_y_xk(y[l], k, N); /* x_k - y_l wrapped */
      /* y_l > x_k  <=>  the unwrapped difference y_l - x_k > 0 */
      if (diff_y_grid(y[l], k, N) > 0.0) ++cnt;
      if (t == 0.0) { hit = 1; continue; }
      nadd(&s, log(fabs(2.0 * sin(0.5 * t))));
    }
    lamC[i] = hit ? -INFINITY : nval(&s);
    nC[i] = cnt;
  }
}

/*   lamD_j = -sum_{l != j} log|2 sin((y_j - y_l)/2)|,  nD_j = #{l : y_l > y_j}
 * so that D_j = (-1)^(nD_j) * 2^{M-1} * 2i e^{-i N y_j/2} * exp(lamD_j)
 * (Eq. p8).  Duplicate points give lamD_j = +inf. */
void orc_logsin_D(const double *y, int64_t M, const int64_t *idx, int64_t nidx,
                  double *lamD, int64_t *nD) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t j = IDX(i);
    nsum s = {0, 0};
    int64_t cnt = 0, dup = 0;
    for (int64_t l = 0; l < M; ++l) {
      if (l == j) continue;
      if (y[l] > y[j]) ++cnt;
      if (y[l] == y[j]) { dup = 1; continue; }
      double t = wrap_diff(y[j], y[l]);
      nadd(&s, log(fabs(2.0 * sin(0.5 * t))));
    }
    lamD[i] = dup ? INFINITY : -nval(&s);
    nD[i] = cnt;
  }
}

/* Square inverse interpolation, Lagrange form (Eq. p6, p8, M = N):
 *   f_k = sum_j C_k G(x_k - y_j) D_j g_j,
 * with C_k D_j = (-1)^(k+nC_k+nD_j) e^{lamC_k + lamD_j} i e^{-i N y_j/2}
 * (the powers of two leave 2^{-M} 2^{M-1} = 1/2, which halves the 2i of D_j).
 * An exact hit y_j = x_k gives f_k = g_j.
 * lamC/nC over all k in idx order, lamD/nD over all j (full arrays). */
void orc_inverse_f(const double *g, const double *y, int64_t M, int64_t N,
                   const double *lamC, const int64_t *nC, const double *lamD,
                   const int64_t *nD, const int64_t *idx, int64_t nidx, double *f) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t k = IDX(i);
    int64_t hitj = -1;
    for (int64_t j = 0; j < M; ++j)
      if (diff_y_xk(y[j], k, N) == 0.0) { hitj = j; break; }
    if (hitj >= 0) { f[2 * i] = g[2 * hitj]; f[2 * i + 1] = g[2 * hitj + 1]; continue; }
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t j = 0; j < M; ++j) {
      double t = -diff_y_xk(y[j], k, N);
      double sgn = ((k + nC[i] + nD[j]) & 1) ? -1.0 : 1.0;
      double mag = sgn * exp(lamC[i] + lamD[j]);
      /* i e^{-i N y_j / 2} */
      double ca, sa;
      half_ny(y[j], N, &ca, &sa);
      double Dr = sa, Di = ca;
      double Gr, Gi;
      G_of_t(t, &Gr, &Gi);
      double Lr = mag * (Gr * Dr - Gi * Di), Li = mag * (Gr * Di + Gi * Dr);
      nadd(&sr, Lr * g[2 * j] - Li * g[2 * j + 1]);
      nadd(&si, Lr * g[2 * j + 1] + Li * g[2 * j]);
    }
    f[2 * i] = nval(&sr);
    f[2 * i + 1] = nval(&si);
  }
}

/* ---------- transforms on the uniform grid (Eq. p1) ---------- */

/* Direct DFT: out_n = sum_k x_k e^{sign * 2 pi i n k / N}, no scaling.
 * The angle index n*k is reduced mod N in integers first. */
void orc_dft(const double *x, int64_t N, int sign, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < N; ++n) {
    nsum sr = {0, 0}, si = {0, 0};
    for (int64_t k = 0; k < N; ++k) {
      int64_t r = (int64_t)(((__int128)n * k) % N);
      double a = (TWO_PI_HI * (double)r) / (double)N;
      double cr = cos(a), ci = sign * sin(a);
      nadd(&sr, x[2 * k] * cr - x[2 * k + 1] * ci);
      nadd(&si, x[2 * k] * ci + x[2 * k + 1] * cr);
    }
    out[2 * n] = nval(&sr);
    out[2 * n + 1] = nval(&si);
  }
}

/* Radix-2 decimation-in-time FFT (Cooley-Tukey), same convention as orc_dft.
 * N must be a power of two.  Twiddles are evaluated directly, not by
 * recurrence. */
void orc_fft(const double *x, int64_t N, int sign, double *out) {
  int L = 0;
  while (((int64_t)1 << L) < N) ++L;
  /* bit-reversal permutation */
  for (int64_t i = 0; i < N; ++i) {
    int64_t r = 0;
    for (int b = 0; b < L; ++b) r |= ((i >> b) & 1) << (L - 1 - b);
    out[2 * r] = x[2 * i];
    out[2 * r + 1] = x[2 * i + 1];
  }
  for (int64_t len = 2; len <= N; len <<= 1) {
    int64_t half = len >> 1;
#pragma omp parallel for schedule(static) if (N >= 4096)
    for (int64_t base = 0; base < N; base += len) {
      for (int64_t j = 0; j < half; ++j) {
        double a = (TWO_PI_HI * (double)j) / (double)len;
        double wr = cos(a), wi = sign * sin(a);
        double *u = out + 2 * (base + j), *v = out + 2 * (base + j + half);
        double tr = v[0] * wr - v[1] * wi, ti = v[0] * wi + v[1] * wr;
        v[0] = u[0] - tr; v[1] = u[1] - ti;
        u[0] = u[0] + tr; u[1] = u[1] + ti;
      }
    }
  }
}

int orc_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Normaliser of the square inverse's matrix-vector product (reading c16):
 *   a_k = sum_j |C_k G(x_k - y_j) D_j| |g_j|,
 * the same terms as orc_inverse_f with every factor replaced by its
 * modulus, |i e^{-i N y_j / 2}| = 1.  An exact hit y_j = x_k gives |g_j|. */
void orc_inverse_absf(const double *g, const double *y, int64_t M, int64_t N,
                      const double *lamC, const double *lamD, const int64_t *idx,
                      int64_t nidx, double *a) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nidx; ++i) {
    int64_t k = IDX(i);
    int64_t hitj = -1;
    for (int64_t j = 0; j < M; ++j)
      if (diff_y_xk(y[j], k, N) == 0.0) { hitj = j; break; }
    if (hitj >= 0) { a[i] = hypot(g[2 * hitj], g[2 * hitj + 1]); continue; }
    nsum s = {0, 0};
    for (int64_t j = 0; j < M; ++j) {
      double t = -diff_y_xk(y[j], k, N);
      double Gr, Gi;
      G_of_t(t, &Gr, &Gi);
      nadd(&s, exp(lamC[i] + lamD[j]) * hypot(Gr, Gi) * hypot(g[2 * j], g[2 * j + 1]));
    }
    a[i] = nval(&s);
  }
}
