// The multilevel FMM for h(y) = sum_k q_k cot((y - x_k)/2) on the circle
// (Sec. 2.1-2.3).  The sum over the level-2 neighbourhood Omega_1 of the
// target's arc is split (Eq. 10) into the singular part 2/t, summed by a 1D
// 1/t MLFMM (levels 3..L plus the near field of adjacent leaves), and a
// regular part, which together with the opposite arc Omega_2 (Eq. 11) is a
// degree 2q-1 polynomial per level-2 arc (Eq. p20).  All positions are in
// grid units (see common.cuh); with t in grid units, 2/t_rad = (N/pi)/t.
//
// Scaled expansions (box width W, centre C, rho = (X - C)/W):
//   multipole  M_m = sum q rho^m,            far field (1/W) sum_m M_m z^{-(m+1)}
//   local      field(Y) = (1/W) sum_n L_n u^n,   u = (Y - C)/W
// Operators (level independent):
//   M2M  child (sigma = -1 left, +1 right) -> parent:
//        M'_m = sum_k C(m,k) 2^-k (sigma/4)^(m-k) M_k
//   M2L  source box at offset d (in box widths) from the target box:
//        L_n += sum_m C(m+n,n) (-1)^(m+1) d^-(m+n+1) M_m
//   L2L  parent -> child: L'_k = 1/2 sum_n C(n,k) 2^-k (sigma/4)^(n-k) L_n
#include <cmath>

#include "common.cuh"

namespace nufft {

// ---------------------------------------------------------------- P2M

// Uniform sources (the grid): every leaf holds s points at the same relative
// positions, so the leaf moments are a product with the table rho_o^m.
template <class T>
__global__ void k_p2m_uniform(TreeDims d, const double2* __restrict__ q,
                              const T* __restrict__ rp, cplx<T>* __restrict__ mleaf) {
  int64_t B = int64_t(1) << d.L;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= B * d.pm) return;
  int64_t b = tid / d.pm;
  int m = (int)(tid - b * d.pm);
  const double2* qb = q + b * d.s;
  T ar = 0, ai = 0;
  for (int o = 0; o < d.s; ++o) {
    double2 v = qb[o];
    T w = rp[o * d.pm + m];
    ar += (T)v.x * w;
    ai += (T)v.y * w;
  }
  mleaf[b * d.pm + m] = mk<T>(ar, ai);
}

// Leaf-relative data of a sorted non-uniform point.
__device__ inline void point_local(int32_t k0, double delta, int64_t N, int s, int64_t* leaf,
                                   int64_t* o) {
  int64_t fl = (delta < 0.0) ? (int64_t)k0 - 1 : (int64_t)k0;
  fl = (fl + N) % N;
  int64_t b = fl / s;
  int64_t off = (int64_t)k0 - b * s;  // in [0, s] up to a period
  if (off < -(N >> 1)) off += N;
  if (off > (N >> 1)) off -= N;
  *leaf = b;
  *o = off;
}

// Non-uniform sources: one warp per leaf; a chunk of 32 sources writes
// q rho^m for 32 consecutive m into shared memory, lanes then reduce rows.
template <class T> struct P2mWarps { static constexpr int value = sizeof(T) == 8 ? 2 : 4; };

template <class T>
__global__ void __launch_bounds__(128) k_p2m_nonuniform(TreeDims d,
                                                        const int32_t* __restrict__ start,
                                                        const int32_t* __restrict__ k0,
                                                        const double* __restrict__ delta,
                                                        const cplx<T>* __restrict__ charge,
                                                        cplx<T>* __restrict__ mleaf) {
  constexpr int WPB = P2mWarps<T>::value;  // keeps the tile under 48 KB
  __shared__ cplx<T> tile[WPB][32][33];
  int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t B = int64_t(1) << d.L;
  int64_t b = blockIdx.x * WPB + warp;
  if (b >= B) return;
  int32_t a = start[b], e = start[b + 1];
  for (int mc = 0; mc < d.pm; mc += 32) {
    T accr = 0, acci = 0;
    for (int c0 = a; c0 < e; c0 += 32) {
      int i = c0 + lane;
      cplx<T> q = mk<T>(0, 0);
      T rho = 0;
      if (i < e) {
        int64_t lb, o;
        point_local(k0[i], delta[i], d.N, d.s, &lb, &o);
        rho = (T)(((double)o + delta[i]) / (double)d.s - 0.5);
        q = charge[i];
      }
      T pw = 1;
      for (int m = 0; m < mc; ++m) pw *= rho;
      for (int m = 0; m < 32; ++m) {
        tile[warp][m][lane] = mk<T>(q.x * pw, q.y * pw);
        pw *= rho;
      }
      __syncwarp();
      for (int k = 0; k < 32; ++k) {
        cplx<T> v = tile[warp][lane][k];
        accr += v.x;
        acci += v.y;
      }
      __syncwarp();
    }
    if (mc + lane < d.pm) mleaf[b * d.pm + mc + lane] = mk<T>(accr, acci);
  }
}

// mleaf[b][m] -= shift[m]: charges of a fixed pattern repeated in every leaf
template <class T>
__global__ void k_leaf_shift(int64_t B, int pm, const double* __restrict__ shift,
                             cplx<T>* __restrict__ mleaf) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= B * pm) return;
  int m = (int)(tid % pm);
  mleaf[tid].x -= (T)shift[m];
}

// ---------------------------------------------------------------- M2M

// level lc (children) -> lc - 1.  op: [2][pm][pm], op[sg][k][m] (transposed).
template <class T>
__global__ void k_m2m(TreeDims d, int lc, const T* __restrict__ op, cplx<T>* __restrict__ mexp) {
  extern __shared__ unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);
  int pm = d.pm;
  for (int i = threadIdx.x; i < 2 * pm * pm; i += blockDim.x) A[i] = op[i];
  __syncthreads();
  int64_t np = int64_t(1) << (lc - 1);
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= np * pm) return;
  int64_t ip = tid / pm;
  int m = (int)(tid - ip * pm);
  const cplx<T>* c0 = mexp + (level_off(lc) + 2 * ip) * pm;
  const cplx<T>* c1 = c0 + pm;
  T ar = 0, ai = 0;
  for (int k = 0; k <= m; ++k) {
    T w0 = A[k * pm + m], w1 = A[pm * pm + k * pm + m];
    cplx<T> x0 = c0[k], x1 = c1[k];
    ar += w0 * x0.x + w1 * x1.x;
    ai += w0 * x0.y + w1 * x1.y;
  }
  mexp[(level_off(lc - 1) + ip) * pm + m] = mk<T>(ar, ai);
}

// ---------------------------------------------------------------- M2L + L2L

// Level l (3..L): L[l][i] = L2L(L[l-1][i/2]) + sum_{d in IL(i)} T_d M[l][i+d].
// Interaction list (children of the parent's neighbours that are not
// neighbours): even i: d in {-2, +2, +3}; odd i: {-3, -2, +2}; box indices
// periodic mod 2^l, displacement unwrapped.  op_m2l [4][p][p] = T_d^T for
// d = -3, -2, +2, +3; op_l2l [2][p][p] transposed.
// For the log kernel (lw != 0) the constant term also receives
// M_0 log W_l of each interacting box, W_l the box width in grid units.
template <class T>
__global__ void k_m2l_l2l(TreeDims d, int l, const T* __restrict__ op_m2l,
                          const T* __restrict__ op_l2l, const cplx<T>* __restrict__ mexp,
                          cplx<T>* __restrict__ lexp, double lw) {
  extern __shared__ unsigned char smraw[];
  T* Tm = reinterpret_cast<T*>(smraw);  // 4 p^2
  T* Tl = Tm + 4 * d.p * d.p;           // 2 p^2
  int p = d.p, pm = d.pm;
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  if (l > 3)
    for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  __syncthreads();
  int64_t nb = int64_t(1) << l;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= nb * p) return;
  int64_t i = tid / p;
  int n = (int)(tid - i * p);
  const cplx<T>* ml = mexp + level_off(l) * pm;
  T ar = 0, ai = 0;
  int odd = (int)(i & 1);
  // offsets and operator slots: slot 0:-3, 1:-2, 2:+2, 3:+3
  int offs[3] = {odd ? -3 : -2, odd ? -2 : 2, odd ? 2 : 3};
  int slot[3] = {odd ? 0 : 1, odd ? 1 : 2, odd ? 2 : 3};
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    int64_t src = (i + offs[t] + nb) & (nb - 1);
    const cplx<T>* mv = ml + src * pm;
    const T* Tt = Tm + slot[t] * p * p;
    for (int m = 0; m < p; ++m) {
      T w = Tt[m * p + n];
      cplx<T> x = mv[m];
      ar += w * x.x;
      ai += w * x.y;
    }
    if (lw != 0.0 && n == 0) {
      ar += (T)lw * mv[0].x;
      ai += (T)lw * mv[0].y;
    }
  }
  if (l > 3) {
    const cplx<T>* lp = lexp + (level_off(l - 1) - 4 + (i >> 1)) * p;
    const T* Tt = Tl + odd * p * p;
    for (int k = n; k < p; ++k) {
      T w = Tt[k * p + n];
      cplx<T> x = lp[k];
      ar += w * x.x;
      ai += w * x.y;
    }
  }
  lexp[(level_off(l) - 4 + i) * p + n] = mk<T>(ar, ai);
}

// ---------------------------------------------------------------- level 2

// Regular part (Eq. p20) from the level-2 multipoles.  With
// mu_{a,i} = sum_{x in P_a} q ((x_c^a - x)/pi)^i = (-1/2)^i M^(2)_{a,i}:
//   A2^(n) = mu_{n+2},  A1^(n)_i = mu_{n,i} + sum_r S-[i][r] mu_{n+1,r}
//                                  + sum_r S+[i][r] mu_{n-1,r}
//   R^(n)_l = sum_i W1[l][i] A1^(n)_i + W2[l][i] A2^(n)_i  (+ c1 A1_0 + c2 A2_0 at l = 0)
// where S+-[i][r] = C(i,r) (+-1/2)^(i-r) shift to the centre of arc n.  For
// the cot kernel W1[l][i] = C(2m-1,l) a_m, W2[l][i] = C(2m-1,l) b_m with
// i = 2m-1-l, a_m = 2 zeta(2m)/4^m, b_m = (4^m - 1) a_m (and the caller
// scales by -2/pi); the log kernel uses its own W and the constants.
// op: [4][nq][nq] = W1, W2, S-, S+.  out: [4][nq] then Q = sum of charges.
// One CTA.
template <class T>
__global__ void k_level2(TreeDims d, int nq, const double* __restrict__ op, double c1, double c2,
                         const cplx<T>* __restrict__ mexp, double2* __restrict__ out) {
  __shared__ double2 mu[4][66];
  __shared__ double2 A1[4][66];
  const cplx<T>* m2 = mexp;  // level 2 sits at offset 0
  for (int e = threadIdx.x; e < 4 * nq; e += blockDim.x) {
    int a = e / nq, i = e - a * nq;
    double2 v = to_d2(m2[a * d.pm + i]);
    double sc = ldexp((i & 1) ? -1.0 : 1.0, -i);
    mu[a][i] = make_double2(v.x * sc, v.y * sc);
  }
  __syncthreads();
  const double* W1 = op;
  const double* W2 = op + nq * nq;
  const double* Sm = op + 2 * nq * nq;
  const double* Sp = op + 3 * nq * nq;
  for (int e = threadIdx.x; e < 4 * nq; e += blockDim.x) {
    int n = e / nq, i = e - n * nq;
    double2 acc = mu[n][i];
    int np1 = (n + 1) & 3, nm1 = (n + 3) & 3;
    for (int r = 0; r <= i; ++r) {
      acc = cadd(acc, cscale(mu[np1][r], Sm[i * nq + r]));
      acc = cadd(acc, cscale(mu[nm1][r], Sp[i * nq + r]));
    }
    A1[n][i] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 4 * nq; e += blockDim.x) {
    int n = e / nq, l = e - n * nq;
    int n2 = (n + 2) & 3;
    double2 acc = make_double2(0, 0);
    for (int i = 0; i < nq; ++i) {
      acc = cadd(acc, cscale(A1[n][i], W1[l * nq + i]));
      acc = cadd(acc, cscale(mu[n2][i], W2[l * nq + i]));
    }
    if (l == 0) {
      acc = cadd(acc, cscale(A1[n][0], c1));
      acc = cadd(acc, cscale(mu[n2][0], c2));
    }
    out[n * nq + l] = acc;
  }
  if (threadIdx.x == 0) {
    double2 qs = make_double2(0, 0);
    for (int a = 0; a < 4; ++a) qs = cadd(qs, to_d2(m2[a * d.pm]));
    out[4 * nq] = qs;
  }
}

// ---------------------------------------------------------------- evaluation helpers

template <class T>
__device__ inline cplx<T> horner(const cplx<T>* __restrict__ c, int n, T u) {
  cplx<T> acc = c[n - 1];
  for (int k = n - 2; k >= 0; --k) {
    cplx<T> v = c[k];
    acc.x = fma(acc.x, u, v.x);
    acc.y = fma(acc.y, u, v.y);
  }
  return acc;
}

__device__ inline double2 horner_d(const double2* __restrict__ c, int n, double u) {
  double2 acc = c[n - 1];
  for (int k = n - 2; k >= 0; --k) {
    acc.x = fma(acc.x, u, c[k].x);
    acc.y = fma(acc.y, u, c[k].y);
  }
  return acc;
}

template <class V> __device__ inline void store_out(V* p, double2 v);
template <> __device__ inline void store_out<double2>(double2* p, double2 v) { *p = v; }
template <> __device__ inline void store_out<float2>(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}

// near-field accumulation: FP64, or FP32 partial sums folded into FP64 every
// 16 terms so the rounding of a long FP32 sum stays at the 1e-7 level.
template <class T> struct NearAcc;
template <> struct NearAcc<double> {
  double2 s = make_double2(0, 0);
  __device__ inline void add(double2 q, double t) {
    double r = 1.0 / t;
    s.x = fma(q.x, r, s.x);
    s.y = fma(q.y, r, s.y);
  }
  __device__ inline void fold() {}
  __device__ inline double2 get() const { return s; }
};
template <> struct NearAcc<float> {
  double2 s = make_double2(0, 0);
  float2 f = make_float2(0, 0);
  int cnt = 0;
  __device__ inline void add(double2 q, double t) {
    float r = __fdividef(1.0f, (float)t);
    f.x = fmaf((float)q.x, r, f.x);
    f.y = fmaf((float)q.y, r, f.y);
    if (++cnt == 16) fold();
  }
  __device__ inline void fold() {
    s.x += f.x; s.y += f.y;
    f = make_float2(0, 0);
    cnt = 0;
  }
  __device__ inline double2 get() { fold(); return s; }
};

// ---------------------------------------------------------------- forward targets

// One thread per sorted target j (Eq. p4, p5, p20):
//   g_j = E_j f_{k0} - (F_j/2) (Q + i h'_j),
//   h'_j = (N/pi) [ (1/s) sum_n L_n u^n + sum_{near, k != k0} f_k / t ]
//          - (2/pi) sum_l D^(arc)_l uhat^l
// where the pair (y_j, x_k0) enters through E_j (its singular 2/t part in
// closed form) and through Q and the regular polynomial like every source.
template <class T, class VO>
__global__ void __launch_bounds__(256) k_targets_fwd(
    TreeDims d, int64_t M, const int32_t* __restrict__ k0s, const double* __restrict__ dels,
    const int32_t* __restrict__ perm, const double2* __restrict__ F,
    const double2* __restrict__ E, const double2* __restrict__ fgrid,
    const cplx<T>* __restrict__ lexp, const double2* __restrict__ lvl2, VO* __restrict__ g) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  const int64_t N = d.N;
  const int s = d.s;
  int32_t k0 = k0s[j];
  double dl = dels[j];
  int64_t b, o;
  point_local(k0, dl, N, s, &b, &o);
  // far field (local expansion of the leaf)
  T u = (T)(((double)o + dl) / (double)s - 0.5);
  const cplx<T>* Lb = lexp + (level_off(d.L) - 4 + b) * d.p;
  double2 far = (d.L >= 3) ? to_d2(horner<T>(Lb, d.p, u)) : make_double2(0, 0);
  // near field: leaves b-1, b, b+1 (periodic, unwrapped displacement)
  NearAcc<T> acc;
  int64_t base = b * s - s;
  for (int64_t r = -s; r < 2 * s; ++r) {
    if (r == o) continue;
    int64_t k = (base + (r + s) + N) & (N - 1);
    double t = (double)(o - r) + dl;
    acc.add(fgrid[k], t);
  }
  double2 nr = acc.get();
  // regular part, arc n = b >> (L-2), uhat = (y - x_c)/pi
  int Q2 = 2 * d.q;  // cot kernel: degree 2q-1
  int64_t arc = b >> (d.L - 2);
  int64_t I = b * s + o - arc * (N >> 2) - (N >> 3);
  double uh = ((double)I + dl) * (2.0 / (double)N);
  double2 reg = horner_d(lvl2 + arc * Q2, Q2, uh);
  double2 Qs = lvl2[4 * Q2];
  double cN = (double)N * kInvPi;
  double hr = cN * (far.x / (double)s + nr.x) - 2.0 * kInvPi * reg.x;
  double hi = cN * (far.y / (double)s + nr.y) - 2.0 * kInvPi * reg.y;
  // Q + i h'
  double2 w = make_double2(Qs.x - hi, Qs.y + hr);
  double2 Fj = F[j];
  double2 res = cscale(cmul(Fj, w), -0.5);
  res = cadd(res, cmul(E[j], fgrid[k0]));
  store_out<VO>(g + perm[j], res);
}

// ---------------------------------------------------------------- adjoint / inverse targets

// Charges in sorted order: adjoint q_i = conj(F_i) g_perm(i);
// inverse q_i = Dt_i g_perm(i) (Eq. p6: D_j g_j, scaled by e^{-Lambda}).
template <class T, class VI>
__global__ void k_charges(int64_t M, const int32_t* __restrict__ perm,
                          const double2* __restrict__ coef, int conj_coef,
                          const VI* __restrict__ gin, cplx<T>* __restrict__ charge) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double2 c = coef[i];
  if (conj_coef) c.y = -c.y;
  double2 gv = to_d2(gin[perm[i]]);
  charge[i] = from_d2<T>(cmul(c, gv));
}

// One thread per grid point k (Eq. p4 transposed, Eq. p6):
//   h_k = sum_j q_j cot((x_k - y_j)/2)   by the same FMM, then
//   adjoint: u_k = sum_{j: k0_j = k} conj(E_j) g_j - (Q + i h'_k)/2  (h' without
//            those pairs' 2/t part)
//   inverse: f_k/N = Ct_k (-(Q + i h_k)/2), or g_j/N when y_j = x_k exactly
//            (Ct_k = C_k e^Lambda / N carries the 1/N of Eq. p1).
template <class T, class VI>
__global__ void __launch_bounds__(256) k_targets_grid(
    TreeDims d, int inverse, const int32_t* __restrict__ start,
    const int32_t* __restrict__ k0s, const double* __restrict__ dels,
    const int32_t* __restrict__ perm, const double2* __restrict__ E,
    const cplx<T>* __restrict__ charge, const VI* __restrict__ gin,
    const cplx<T>* __restrict__ lexp, const double2* __restrict__ lvl2,
    const double* __restrict__ Ct, double2* __restrict__ out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = d.N;
  if (k >= N) return;
  const int s = d.s;
  const int64_t B = int64_t(1) << d.L;
  int64_t b = k / s, o = k - b * s;
  T u = (T)((double)o / (double)s - 0.5);
  const cplx<T>* Lb = lexp + (level_off(d.L) - 4 + b) * d.p;
  double2 far = (d.L >= 3) ? to_d2(horner<T>(Lb, d.p, u)) : make_double2(0, 0);
  NearAcc<T> acc;
  double2 self = make_double2(0, 0);
  int hit = -1;
  NearAcc<double> accd;  // inverse: pairs with k0_j = k in FP64
  for (int nb = -1; nb <= 1; ++nb) {
    int64_t bb = (b + nb + B) & (B - 1);
    int32_t a = start[bb], e = start[bb + 1];
    for (int32_t i = a; i < e; ++i) {
      // k0_i relative to leaf b's origin, unwrapped through the known leaf
      // offset nb (k0_i lies in [bb s, bb s + s] modulo N)
      int64_t rel = (int64_t)nb * s + (((int64_t)k0s[i] - bb * s + N) & (N - 1));
      int64_t D = o - rel;
      double di = dels[i];
      if (D == 0) {
        if (inverse) {
          if (di == 0.0) hit = i;
          else accd.add(to_d2(charge[i]), -di);
        } else {
          self = cadd(self, cmul(cconj(E[i]), to_d2(gin[perm[i]])));
        }
        continue;
      }
      acc.add(to_d2(charge[i]), (double)D - di);
    }
  }
  double2 nr = acc.get();
  if (inverse) nr = cadd(nr, accd.get());
  int Q2 = 2 * d.q;
  int64_t arc = b >> (d.L - 2);
  int64_t I = k - arc * (N >> 2) - (N >> 3);
  double uh = (double)I * (2.0 / (double)N);
  double2 reg = horner_d(lvl2 + arc * Q2, Q2, uh);
  double2 Qs = lvl2[4 * Q2];
  double cN = (double)N * kInvPi;
  double hr = cN * (far.x / (double)s + nr.x) - 2.0 * kInvPi * reg.x;
  double hi = cN * (far.y / (double)s + nr.y) - 2.0 * kInvPi * reg.y;
  double2 res = make_double2(-0.5 * (Qs.x - hi), -0.5 * (Qs.y + hr));
  if (inverse) {
    res = cscale(res, Ct[k]);
    // exact hit: f_k = g_j; Ct carries the 1/N of the final DFT, so apply it here too
    if (hit >= 0) res = cscale(to_d2(gin[perm[hit]]), 1.0 / (double)N);
  } else {
    res = cadd(res, self);
  }
  out[k] = res;
}

}  // namespace nufft

using namespace nufft;

// ---------------------------------------------------------------- host drivers

static inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

template <class T>
int fmm_configure() {
  int big = 200 * 1024;
  if (cudaFuncSetAttribute(k_m2l_l2l<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
      cudaSuccess)
    return NUFFT_ECUDA;
  if (cudaFuncSetAttribute(k_m2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
      cudaSuccess)
    return NUFFT_ECUDA;
  return NUFFT_OK;
}

// Upward pass + far field + level-2 coefficients for charges already laid out
// (uniform: on the grid in `grid`; non-uniform: sorted in plan->charge).
template <class T>
int fmm_upward_downward(nufft_plan_s* pl, const FmmOps& ops, bool uniform_sources,
                        const cplx<T>* charge, double2* lvl2) {
  cudaStream_t st = pl->stream;
  TreeDims d{pl->N, pl->L, pl->s, pl->p, pl->q, pl->pm};
  int64_t B = pl->B;
  cplx<T>* mexp = (cplx<T>*)pl->mexp;
  cplx<T>* lexp = (cplx<T>*)pl->lexp;
  cplx<T>* mleaf = mexp + level_off(pl->L) * pl->pm;
  prof_begin(pl, NUFFT_STAGE_P2M);
  if (uniform_sources) {
    k_p2m_uniform<T><<<nblk(B * pl->pm, 256), 256, 0, st>>>(d, pl->grid, (const T*)pl->op_p2m,
                                                           mleaf);
  } else {
    constexpr int WPB = P2mWarps<T>::value;
    k_p2m_nonuniform<T><<<nblk(B, WPB), 32 * WPB, 0, st>>>(d, pl->leaf_start, pl->k0, pl->delta,
                                                           charge, mleaf);
  }
  if (ops.leaf_shift)
    k_leaf_shift<T><<<nblk(B * pl->pm, 256), 256, 0, st>>>(B, pl->pm, ops.leaf_shift, mleaf);
  prof_end(pl, ops.leaf_shift ? 2 : 1);
  prof_begin(pl, NUFFT_STAGE_M2M);
  size_t sm_m2m = (size_t)2 * pl->pm * pl->pm * sizeof(T);
  for (int lc = pl->L; lc >= 3; --lc) {
    int64_t np = int64_t(1) << (lc - 1);
    k_m2m<T><<<nblk(np * pl->pm, 256), 256, sm_m2m, st>>>(d, lc, (const T*)pl->op_m2m, mexp);
  }
  prof_end(pl, pl->L - 2);
  prof_begin(pl, NUFFT_STAGE_LEVEL2);
  k_level2<T><<<1, 256, 0, st>>>(d, ops.nq, ops.reg, ops.c1, ops.c2, mexp, lvl2);
  prof_end(pl, 1);
  prof_begin(pl, NUFFT_STAGE_M2L);
  size_t sm_m2l = (size_t)6 * pl->p * pl->p * sizeof(T);
  for (int l = 3; l <= pl->L; ++l) {
    int64_t nb = int64_t(1) << l;
    double lw = ops.log_kernel ? std::log((double)(pl->N >> l)) : 0.0;
    k_m2l_l2l<T><<<nblk(nb * pl->p, 256), 256, sm_m2l, st>>>(d, l, (const T*)ops.m2l,
                                                            (const T*)ops.l2l, mexp, lexp, lw);
  }
  prof_end(pl, pl->L >= 3 ? pl->L - 2 : 0);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

static FmmOps cot_ops(nufft_plan_s* pl) {
  FmmOps o;
  o.m2l = pl->op_m2l;
  o.l2l = pl->op_l2l;
  o.reg = pl->op_reg;
  o.nq = 2 * pl->q;
  return o;
}

// forward: grid samples f in pl->grid (complex128) -> g (original order)
template <class T>
int fmm_forward(nufft_plan_s* pl, void* g) {
  int rc = fmm_upward_downward<T>(pl, cot_ops(pl), true, nullptr, pl->lvl2);
  if (rc) return rc;
  TreeDims d{pl->N, pl->L, pl->s, pl->p, pl->q, pl->pm};
  cplx<T>* lexp = (cplx<T>*)pl->lexp;
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  if (pl->flags & NUFFT_IO_C64)
    k_targets_fwd<T, float2><<<nblk(pl->M, 256), 256, 0, pl->stream>>>(
        d, pl->M, pl->k0, pl->delta, pl->perm, pl->F, pl->E, pl->grid, lexp, pl->lvl2,
        (float2*)g);
  else
    k_targets_fwd<T, double2><<<nblk(pl->M, 256), 256, 0, pl->stream>>>(
        d, pl->M, pl->k0, pl->delta, pl->perm, pl->F, pl->E, pl->grid, lexp, pl->lvl2,
        (double2*)g);
  prof_end(pl, 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// adjoint / inverse: samples g (original order) -> values on the grid in pl->grid
template <class T>
int fmm_to_grid(nufft_plan_s* pl, const void* g, int inverse) {
  cudaStream_t st = pl->stream;
  bool c64 = (pl->flags & NUFFT_IO_C64) != 0;
  const double2* coef = inverse ? pl->Dt : pl->F;
  prof_begin(pl, NUFFT_STAGE_P2M);
  if (c64)
    k_charges<T, float2><<<nblk(pl->M, 256), 256, 0, st>>>(pl->M, pl->perm, coef, !inverse,
                                                          (const float2*)g, (cplx<T>*)pl->charge);
  else
    k_charges<T, double2><<<nblk(pl->M, 256), 256, 0, st>>>(pl->M, pl->perm, coef, !inverse,
                                                           (const double2*)g, (cplx<T>*)pl->charge);
  prof_end(pl, 1);
  int rc = fmm_upward_downward<T>(pl, cot_ops(pl), false, (const cplx<T>*)pl->charge, pl->lvl2);
  if (rc) return rc;
  TreeDims d{pl->N, pl->L, pl->s, pl->p, pl->q, pl->pm};
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  if (c64)
    k_targets_grid<T, float2><<<nblk(pl->N, 256), 256, 0, st>>>(
        d, inverse, pl->leaf_start, pl->k0, pl->delta, pl->perm, pl->E,
        (const cplx<T>*)pl->charge, (const float2*)g, (const cplx<T>*)pl->lexp, pl->lvl2, pl->Ct,
        pl->grid);
  else
    k_targets_grid<T, double2><<<nblk(pl->N, 256), 256, 0, st>>>(
        d, inverse, pl->leaf_start, pl->k0, pl->delta, pl->perm, pl->E,
        (const cplx<T>*)pl->charge, (const double2*)g, (const cplx<T>*)pl->lexp, pl->lvl2,
        pl->Ct, pl->grid);
  prof_end(pl, 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template int fmm_configure<double>();
template int fmm_configure<float>();
template int fmm_forward<double>(nufft_plan_s*, void*);
template int fmm_forward<float>(nufft_plan_s*, void*);
template int fmm_to_grid<double>(nufft_plan_s*, const void*, int);
template int fmm_to_grid<float>(nufft_plan_s*, const void*, int);
template int fmm_upward_downward<double>(nufft_plan_s*, const FmmOps&, bool, const double2*,
                                         double2*);
