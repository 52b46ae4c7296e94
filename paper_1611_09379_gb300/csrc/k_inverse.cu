// Coefficients of the square inverse (Eq. p6, p8, M = N):
//   C_k = (-1)^k prod_l sin((x_k - y_l)/2),
//   D_j = 2i e^{-i N y_j/2} / prod_{l != j} sin((y_j - y_l)/2),
// "precomputed using the FMM" (Sec. 2).  With S(t) = log|2 sin(t/2)|,
//   lamC_k = sum_l S(x_k - y_l),  lamD_j = -sum_{l != j} S(y_j - y_l),
// C_k D_j = (-1)^(k + nC_k + nD_j) e^{lamC_k + lamD_j} i e^{-i N y_j/2}
// (nC_k = #{y_l > x_k}, nD_j = #{y_l > y_j}; the powers of two leave 1/2).
//
// The sums run through the same tree with the log kernel.  Like Eq. 10/11
// for cot, S splits on Omega_1 into log|t| (a 1D log MLFMM) minus the even
// series sum_m a_m/(2m) (t/pi)^{2m}, and on Omega_2 into log 2 minus
// sum_m b_m/(2m) (t/pi)^{2m} (the integrals of Eq. 10 and 11).  To avoid
// the O(N) cancellation of unit charges (box sums ~N/8 whose logs cancel to
// O(1)), every point carries charge +1 and each half-grid point
// X = l + 1/2 (grid units) charge -1; the half-grid sum has the closed form
//   sum_l S(x - 2 pi (l + 1/2)/N) = log|2 cos(N x / 2)|
// (the product identity of equispaced sines), added back at the end.  Box
// charges are then nearly neutral and the FP64 sums stay at the 1e-14 level.
//
// Nc points on a larger grid (Nc < N, N = 2^ceil(log2 Nc): the inverse for
// Nc coefficients of a general size): the interpolant is the same, and the
// Lagrange form holds at any x with C(x) = e^{i Nc x / 2} prod_l sin((x -
// y_l)/2) and D_j = 2i e^{-i Nc y_j / 2} / prod_{l != j} sin((y_j - y_l)/2),
// so it is evaluated at the N grid points (whose N-point DFT gives the first
// Nc coefficients exactly).  C keeps its sign (-1)^{nC_k} here and the phase
// e^{i pi k Nc / N} is applied by the target kernels; the half-grid charges
// weigh Nc / N each (total -Nc, the boxes stay neutral) and their closed
// forms scale by the same weight.
#include <cmath>
#include <vector>

#include "common.cuh"

using namespace nufft;

template <class T>
int fmm_upward_downward(nufft_plan_s* pl, const FmmOps& ops, bool uniform_sources,
                        const cplx<T>* charge, double2* lvl2, float2* lvl2f);

namespace {

__global__ void k_fill_ones(double2* __restrict__ q, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) q[i] = make_double2(1.0, 0.0);
}

__device__ inline void local_of(int32_t k0, double delta, int64_t N, int s, int64_t* leaf,
                                int64_t* o) {
  int64_t fl = (delta < 0.0) ? (int64_t)k0 - 1 : (int64_t)k0;
  fl = (fl + N) % N;
  int64_t b = fl / s;
  int64_t off = (int64_t)k0 - b * s;
  if (off < -(N >> 1)) off += N;
  if (off > (N >> 1)) off -= N;
  *leaf = b;
  *o = off;
}

// running log of a product, folded every 8 factors
struct LogProd {
  double acc = 0.0, prod = 1.0;
  int cnt = 0;
  __device__ inline void mul(double t) {
    prod *= fabs(t);
    if (++cnt == 8) { acc += log(prod); prod = 1.0; cnt = 0; }
  }
  __device__ inline double get() { return acc + log(prod); }
};

__device__ inline double horner_re(const double2* __restrict__ c, int n, double u) {
  double a = c[n - 1].x;
  for (int k = n - 2; k >= 0; --k) a = fma(a, u, c[k].x);
  return a;
}

// unwrapped grid index for ordering (a point just below 2 pi has k0 = 0, delta < 0)
__device__ inline int64_t kk_of(int32_t k0, double d, int64_t N) {
  return (k0 == 0 && d < 0.0) ? N : (int64_t)k0;
}

// lamC_k and nC_k on the grid.
__global__ void k_logsum_grid(TreeDims d, const int32_t* __restrict__ start,
                              const int32_t* __restrict__ k0s, const double* __restrict__ dels,
                              const double2* __restrict__ lexp, const double2* __restrict__ lvl2,
                              const double* __restrict__ hg, int64_t M, double wc,
                              double* __restrict__ lamC, int32_t* __restrict__ nC) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = d.N;
  if (k >= N) return;
  const int s = d.s;
  const int64_t B = int64_t(1) << d.L;
  int64_t b = k / s, o = k - b * s;
  double u = (double)o / (double)s - 0.5;
  double far = (d.L >= 3) ? horner_re(lexp + (level_off(d.L) - 4 + b) * d.p, d.p, u) : 0.0;
  LogProd lp;
  bool hit = false;
  for (int nb = -1; nb <= 1; ++nb) {
    int64_t bb = (b + nb + B) & (B - 1);
    int32_t a = start[bb], e = start[bb + 1];
    for (int32_t i = a; i < e; ++i) {
      int64_t rel = (int64_t)nb * s + (((int64_t)k0s[i] - bb * s + N) & (N - 1));
      double t = (double)(o - rel) - dels[i];
      if (t == 0.0) { hit = true; continue; }
      lp.mul(t);
    }
  }
  int nq = 2 * d.q + 1;
  int64_t arc = b >> (d.L - 2);
  double uh = (double)(k - arc * (N >> 2) - (N >> 3)) * (2.0 / (double)N);
  double reg = horner_re(lvl2 + arc * nq, nq, uh);
  // closed form of the half-grid sum at x_k: log|2 cos(pi k)| = log 2 (times
  // the half-grid charge weight wc; hg is weighted already)
  double lam = far + (lp.get() - hg[o]) + reg + wc * 0.6931471805599453;
  lamC[k] = hit ? -INFINITY : lam;
  // nC_k = #{Y_l > k}: all points of later leaves plus those of leaf b above k
  int32_t cnt = (int32_t)(M - start[b + 1]);
  for (int32_t i = start[b]; i < start[b + 1]; ++i) {
    int64_t kk = kk_of(k0s[i], dels[i], N);
    if (kk > k || (kk == k && dels[i] > 0.0)) ++cnt;
  }
  nC[k] = cnt;
}

// exact a - b as hi + lo
__device__ inline void two_sum(double a, double b, double* hi, double* lo) {
  double s = a + b, bb = s - a;
  *hi = s;
  *lo = (a - (s - bb)) + (b - bb);
}

// lamD_j and nD_j for sorted points.
__global__ void k_logsum_pts(TreeDims d, const int32_t* __restrict__ start,
                             const int32_t* __restrict__ k0s, const double* __restrict__ dels,
                             const double2* __restrict__ lexp, const double2* __restrict__ lvl2,
                             int64_t M, double wc, double* __restrict__ lamD,
                             int32_t* __restrict__ nD, int* __restrict__ status) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t N = d.N;
  const int s = d.s;
  const int64_t B = int64_t(1) << d.L;
  int32_t kj = k0s[j];
  double dj = dels[j];
  int64_t b, o;
  local_of(kj, dj, N, s, &b, &o);
  double u = ((double)o + dj) / (double)s - 0.5;
  double far = (d.L >= 3) ? horner_re(lexp + (level_off(d.L) - 4 + b) * d.p, d.p, u) : 0.0;
  LogProd lp, lh;
  bool dup = false;
  for (int nb = -1; nb <= 1; ++nb) {
    int64_t bb = (b + nb + B) & (B - 1);
    int32_t a = start[bb], e = start[bb + 1];
    for (int32_t i = a; i < e; ++i) {
      if (i == j) continue;
      // both grid indices relative to leaf b's origin, unwrapped via nb
      int64_t rel = (int64_t)nb * s + (((int64_t)k0s[i] - bb * s + N) & (N - 1));
      int64_t D = o - rel;
      double h1, l1, h2, l2;
      two_sum(dj, -dels[i], &h1, &l1);
      two_sum((double)D, h1, &h2, &l2);
      double t = h2 + (l1 + l2);
      if (t == 0.0) { dup = true; continue; }
      lp.mul(t);
    }
  }
  // half-grid charges of the three leaves: X = b s + r + 1/2, r in [-s, 2s)
  for (int64_t r = -s; r < 2 * s; ++r) lh.mul(((double)(o - r) - 0.5) + dj);
  int nq = 2 * d.q + 1;
  int64_t arc = b >> (d.L - 2);
  int64_t I = b * s + o - arc * (N >> 2) - (N >> 3);
  double uh = ((double)I + dj) * (2.0 / (double)N);
  double reg = horner_re(lvl2 + arc * nq, nq, uh);
  // closed form at y_j: log|2 cos(N y_j / 2)| = log|2 cos(pi delta_j)|; the
  // point's own charge added c1 = log(2 pi/N) to the constant term.
  double cf = log(2.0 * cospi(dj));
  double c1 = log(kTwoPiHi / (double)N);
  double S = far + (lp.get() - wc * lh.get()) + reg + wc * cf - c1;
  lamD[j] = -S;
  if (dup) atomicOr(status, kDevIllCond);
  // nD_j = #{Y_l > Y_j}
  int64_t kkj = kk_of(kj, dj, N);
  int32_t cnt = (int32_t)(M - start[b + 1]);
  for (int32_t i = start[b]; i < start[b + 1]; ++i) {
    if (i == j) continue;
    int64_t kk = kk_of(k0s[i], dels[i], N);
    if (kk > kkj || (kk == kkj && dels[i] > dj)) ++cnt;
  }
  nD[j] = cnt;
}

// Lambda = midpoint of the range of lamD (one CTA)
__global__ void k_lambda(const double* __restrict__ lamD, int64_t M, double* __restrict__ out) {
  __shared__ double mn[1024], mx[1024];
  double a = INFINITY, b = -INFINITY;
  for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
    double v = lamD[i];
    a = fmin(a, v);
    b = fmax(b, v);
  }
  mn[threadIdx.x] = a;
  mx[threadIdx.x] = b;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) {
      mn[threadIdx.x] = fmin(mn[threadIdx.x], mn[threadIdx.x + h]);
      mx[threadIdx.x] = fmax(mx[threadIdx.x], mx[threadIdx.x + h]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * (mn[0] + mx[0]);
}

constexpr double kExpLimit = 700.0;

// Ctf (optional): FP32 copy for the mixed path, whose exponent limit elim
// keeps C_k e^Lambda / N below the FP32 overflow threshold.  Below the FP32
// range only the FP64 limit applies: a tiny C~_k (a point next to x_k: C~_k
// carries sin((x_k - y_j)/2)) scales sums that are O(1), so its FP32 copy
// losing digits or vanishing changes f_k by less than rounding, and the one
// term it does not leave small, the self term of that point, comes from the
// FP64-formed factor S_j.
// phase_sep: the phase of C(x_k) is applied by the target kernels (Nc < N),
// so only the sign of the sine product is kept here.
__global__ void k_assemble_C(const double* __restrict__ lamC, const int32_t* __restrict__ nC,
                             int64_t N, const double* __restrict__ Lam, double elim,
                             int phase_sep, double* __restrict__ Ct, float* __restrict__ Ctf,
                             int* __restrict__ status) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= N) return;
  double l = lamC[k];
  double v = 0.0;
  if (l != -INFINITY) {
    double e = l + *Lam;
    if (!(e < elim && e > -kExpLimit)) atomicOr(status, kDevIllCond);
    double sg = (((phase_sep ? 0 : k) + nC[k]) & 1) ? -1.0 : 1.0;
    v = sg * exp(e) / (double)N;  // with the 1/N of Eq. p1
  }
  Ct[k] = v;
  if (Ctf) Ctf[k] = (float)v;
}

// elim: largest |exponent| of D_j e^{-Lambda} (the mixed path forms the
// charges D_j g_j in FP32, so it allows less than FP64 range).
// nc, N: the points' count and the grid (nc = N: a power-of-two inverse)
__global__ void k_assemble_D(const double* __restrict__ lamD, const int32_t* __restrict__ nD,
                             const int32_t* __restrict__ k0s, const double* __restrict__ dels,
                             int64_t M, int64_t nc, int64_t N, const double* __restrict__ Lam,
                             double elim, double2* __restrict__ Dt, float2* __restrict__ Dtf,
                             int* __restrict__ status) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  double e = lamD[j] - *Lam;
  if (!(fabs(e) < elim)) atomicOr(status, kDevIllCond);
  double mag = exp(e);
  double sn, cs;
  if (nc == N) {
    // i e^{-i N y_j / 2} = (-1)^k0 (sin(pi delta) + i cos(pi delta))
    if ((nD[j] + k0s[j]) & 1) mag = -mag;
    sincospi(dels[j], &sn, &cs);
  } else {
    // i e^{-i nc y_j / 2} = sin(pi a) + i cos(pi a), a = (nc / N)(k0 + delta):
    // the integer part (nc k0 mod 2N) / N exactly, the rest (nc / N) delta
    if (nD[j] & 1) mag = -mag;
    const int64_t A = ((int64_t)k0s[j] * nc) % (2 * N);
    double s1, c1, s2, c2;
    sincospi((double)A / (double)N, &s1, &c1);
    sincospi(((double)nc / (double)N) * dels[j], &s2, &c2);
    sn = s1 * c2 + c1 * s2;
    cs = c1 * c2 - s1 * s2;
  }
  Dt[j] = make_double2(mag * sn, mag * cs);
  if (Dtf) Dtf[j] = make_float2((float)(mag * sn), (float)(mag * cs));
}

inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

struct Bin {
  std::vector<long double> c;
  int n;
  explicit Bin(int nmax) : c((size_t)(nmax + 1) * (nmax + 1), 0.0L), n(nmax) {
    for (int i = 0; i <= nmax; ++i) {
      c[(size_t)i * (nmax + 1)] = 1;
      for (int k = 1; k <= i; ++k)
        c[(size_t)i * (nmax + 1) + k] =
            c[(size_t)(i - 1) * (nmax + 1) + k - 1] + (k <= i - 1 ? c[(size_t)(i - 1) * (nmax + 1) + k] : 0);
    }
  }
  long double operator()(int i, int k) const { return (k < 0 || k > i) ? 0 : c[(size_t)i * (n + 1) + k]; }
};

long double zeta_even_l(int s) {
  const int K = 64;
  long double sum = 0;
  for (int k = 1; k < K; ++k) sum += powl((long double)k, -(long double)s);
  long double Kl = K;
  sum += powl(Kl, 1.0L - s) / (s - 1) + 0.5L * powl(Kl, -(long double)s);
  sum += (1.0L / 12.0L) * s * powl(Kl, -(long double)s - 1);
  sum += (-1.0L / 720.0L) * s * (s + 1.0L) * (s + 2.0L) * powl(Kl, -(long double)s - 3);
  sum += (1.0L / 30240.0L) * s * (s + 1.0L) * (s + 2.0L) * (s + 3.0L) * (s + 4.0L) *
         powl(Kl, -(long double)s - 5);
  return sum;
}

struct TmpLayout {
  size_t mexp, lexp, ones, lvl2, m2m, m2l, l2l, reg, shift, hg, lamC, lamD, nC, nD, lam, total;
};

TmpLayout layout(const nufft_plan_s* pl) {
  TmpLayout t{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t r = off; off += (bytes + 255) & ~size_t(255); return r; };
  int64_t nm = (int64_t(2) << pl->L) - 4, nl = (int64_t(2) << pl->L) - 8;
  int nq = 2 * pl->q + 1;
  t.mexp = take((size_t)nm * pl->pm * 16);
  t.lexp = take((size_t)(nl > 0 ? nl : 1) * pl->p * 16);
  t.ones = take((size_t)pl->M * 16);
  t.lvl2 = take((size_t)(4 * nq + 1) * 16);
  t.m2m = take((size_t)2 * pl->pm * pl->pm * 8);
  t.m2l = take((size_t)4 * pl->p * pl->p * 8);
  t.l2l = take((size_t)2 * pl->p * pl->p * 8);
  t.reg = take((size_t)4 * nq * nq * 8);
  t.shift = take((size_t)pl->pm * 8);
  t.hg = take((size_t)pl->s * 8);
  t.lamC = take((size_t)pl->N * 8);
  t.lamD = take((size_t)pl->M * 8);
  t.nC = take((size_t)pl->N * 4);
  t.nD = take((size_t)pl->M * 4);
  t.lam = take(64);
  t.total = off;
  return t;
}

}  // namespace

size_t inverse_tmp_bytes(const nufft_plan_s* pl) { return layout(pl).total; }

// The inverse's self term of sorted point j (the closed form of its pair with
// the nearest grid point x_k0, Eq. p6 with Eq. p8's factors) is its charge
// q_j = D~_j g_j times a factor of the points alone:
//   S_j = i C~_k0 (N / 2pi) / delta_j  (times e^{i pi k0 Nc / N} when the
//         coefficient count Nc is below the grid size N),
//   S_j = 1 / (N D~_j) at an exact hit (the grid value there is g_j / N).
// Formed in FP64 once per plan (with an FP32 copy for the mixed path), so
// the near-field kernels' staging multiplies instead of dividing.
__global__ void k_assemble_S(TreeDims d, int64_t M, const int32_t* __restrict__ k0s,
                             const double* __restrict__ dels, const double* __restrict__ Ct,
                             const double2* __restrict__ Dt, double2* __restrict__ S,
                             float2* __restrict__ Sf) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const double dl = dels[j];
  double2 v;
  if (dl == 0.0) {
    const double2 q = Dt[j];
    const double n2 = (q.x * q.x + q.y * q.y) * (double)d.N;
    v = make_double2(q.x / n2, -q.y / n2);
  } else {
    const int k0 = k0s[j];
    const double w = Ct[k0] * (0.5 * (double)d.N * kInvPi) / dl;
    v = make_double2(0.0, w);
    if (d.nc) v = cmul(v, inv_phase(d, k0));
  }
  S[j] = v;
  if (Sf) Sf[j] = make_float2((float)v.x, (float)v.y);
}

int inverse_precompute(nufft_plan_s* pl, void* tmp, size_t tmp_bytes) {
  TmpLayout t = layout(pl);
  if (tmp_bytes < t.total) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  char* base = (char*)tmp;
  const int p = pl->p, pm = pl->pm, q = pl->q, nq = 2 * q + 1, s = pl->s;
  const int64_t N = pl->N, M = pl->M;
  if (cudaMalloc((void**)&pl->Ct, N * 8) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMalloc((void**)&pl->Dt, M * 16) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMalloc((void**)&pl->Lambda, 8) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMalloc((void**)&pl->Sinv, M * 16) != cudaSuccess) return NUFFT_ENOMEM;
  if (pl->prec != NUFFT_FP64 && (cudaMalloc((void**)&pl->Ctf, N * 4) != cudaSuccess ||
                                 cudaMalloc((void**)&pl->Dtf, M * 8) != cudaSuccess ||
                                 cudaMalloc((void**)&pl->Sinvf, M * 8) != cudaSuccess))
    return NUFFT_ENOMEM;
  // ---- operators of the log kernel (host, long double)
  Bin C(2 * 64 + 2);
  std::vector<double> m2m((size_t)2 * pm * pm, 0.0), m2l((size_t)4 * p * p, 0.0),
      l2l((size_t)2 * p * p, 0.0), reg((size_t)4 * nq * nq, 0.0), shift(pm), hg(s);
  for (int sg = 0; sg < 2; ++sg) {
    long double sig = sg ? 0.25L : -0.25L;
    for (int m = 0; m < pm; ++m)
      for (int k = 0; k <= m; ++k)
        m2m[(size_t)sg * pm * pm + (size_t)k * pm + m] = (double)(C(m, k) * powl(0.5L, k) * powl(sig, m - k));
    for (int n = 0; n < p; ++n)
      for (int k = n; k < p; ++k)
        l2l[(size_t)sg * p * p + (size_t)k * p + n] = (double)(C(k, n) * powl(0.5L, n) * powl(sig, k - n));
  }
  const int dval[4] = {-3, -2, 2, 3};
  for (int tt = 0; tt < 4; ++tt) {
    long double dd = dval[tt];
    for (int m = 0; m < p; ++m)
      for (int n = 0; n < p; ++n) {
        long double v;
        if (m == 0 && n == 0) v = logl(fabsl(dd));
        else if (m == 0) v = -1.0L / (n * powl(dd, n));
        else v = -(1.0L / m) * powl(-dd, -(long double)m) * C(m + n - 1, n) * powl(dd, -(long double)n);
        m2l[(size_t)tt * p * p + (size_t)m * p + n] = (double)v;
      }
  }
  for (int l = 0; l < nq; ++l)
    for (int m = 1; m <= q; ++m) {
      int i = 2 * m - l;
      if (i < 0 || i >= nq) continue;
      long double z = zeta_even_l(2 * m);
      long double am = 2.0L * z * powl(0.25L, m), bm = 2.0L * z * (1.0L - powl(0.25L, m));
      reg[(size_t)l * nq + i] = (double)(-C(2 * m, l) * am / (2 * m));
      reg[(size_t)nq * nq + (size_t)l * nq + i] = (double)(-C(2 * m, l) * bm / (2 * m));
    }
  for (int i = 0; i < nq; ++i)
    for (int r = 0; r <= i; ++r) {
      long double c = C(i, r) * powl(0.5L, i - r);
      reg[(size_t)2 * nq * nq + (size_t)i * nq + r] = (double)(((i - r) & 1) ? -c : c);
      reg[(size_t)3 * nq * nq + (size_t)i * nq + r] = (double)c;
    }
  // half-grid charges of weight wc = Nc / N (1 for a power-of-two inverse)
  const long double wcl = (long double)pl->Nc / (long double)N;
  const double wc = (double)wcl;
  for (int m = 0; m < pm; ++m) {
    long double acc = 0;
    for (int o = 0; o < s; ++o) acc += powl(((long double)o + 0.5L) / s - 0.5L, m);
    shift[m] = (double)(wcl * acc);
  }
  for (int o = 0; o < s; ++o) {
    long double acc = 0;
    for (int r = -s; r < 2 * s; ++r) acc += logl(fabsl((long double)o - r - 0.5L));
    hg[o] = (double)(wcl * acc);
  }
  auto up = [&](size_t off, const std::vector<double>& v) {
    return cudaMemcpyAsync(base + off, v.data(), v.size() * 8, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  if (!up(t.m2m, m2m) || !up(t.m2l, m2l) || !up(t.l2l, l2l) || !up(t.reg, reg) ||
      !up(t.shift, shift) || !up(t.hg, hg))
    return NUFFT_ECUDA;
  // ---- FMM with the log kernel in FP64 on a shadow of the plan
  nufft_plan_s sh = *pl;
  sh.batch = 1;  // the log-sums are one real "signal" (unit charges)
  sh.side_ok = 0;  // plan time: one stream, no side branch of its own
  sh.upcnt = nullptr;  // (the plan's counters are sized for its own expansions)
  sh.mexp = base + t.mexp;
  sh.lexp = base + t.lexp;
  sh.op_m2m = base + t.m2m;
  double2* ones = (double2*)(base + t.ones);
  double2* lvl2 = (double2*)(base + t.lvl2);
  k_fill_ones<<<nblk(M, 256), 256, 0, st>>>(ones, M);
  FmmOps ops;
  ops.m2l = base + t.m2l;
  ops.l2l = base + t.l2l;
  ops.reg = (const double*)(base + t.reg);
  ops.nq = nq;
  ops.c1 = std::log(6.283185307179586 / (double)N);
  ops.c2 = std::log(2.0);
  ops.log_kernel = 1;
  ops.leaf_shift = (const double*)(base + t.shift);
  int rc = fmm_upward_downward<double>(&sh, ops, false, ones, lvl2, nullptr);
  if (rc) return rc;
  TreeDims d{N, pl->L, s, p, q, pm};
  double* lamC = (double*)(base + t.lamC);
  double* lamD = (double*)(base + t.lamD);
  int32_t* nC = (int32_t*)(base + t.nC);
  int32_t* nD = (int32_t*)(base + t.nD);
  double* Lam = pl->Lambda;
  const double2* lexp = (const double2*)sh.lexp;
  k_logsum_grid<<<nblk(N, 128), 128, 0, st>>>(d, pl->leaf_start, pl->k0, pl->delta, lexp, lvl2,
                                              (const double*)(base + t.hg), M, wc, lamC, nC);
  k_logsum_pts<<<nblk(M, 128), 128, 0, st>>>(d, pl->leaf_start, pl->k0, pl->delta, lexp, lvl2, M,
                                             wc, lamD, nD, pl->status);
  k_lambda<<<1, 1024, 0, st>>>(lamD, M, Lam);
  double elim = pl->prec == NUFFT_FP64 ? kExpLimit : 60.0;
  const int sep = pl->Nc != N;
  k_assemble_C<<<nblk(N, 256), 256, 0, st>>>(lamC, nC, N, Lam, elim, sep, pl->Ct, pl->Ctf,
                                             pl->status);
  k_assemble_D<<<nblk(M, 256), 256, 0, st>>>(lamD, nD, pl->k0, pl->delta, M, pl->Nc, N, Lam, elim,
                                             pl->Dt, pl->Dtf, pl->status);
  TreeDims dn = d;
  dn.nc = pl->inv_nc;
  k_assemble_S<<<nblk(M, 256), 256, 0, st>>>(dn, M, pl->k0, pl->delta, pl->Ct, pl->Dt, pl->Sinv,
                                             pl->Sinvf);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
