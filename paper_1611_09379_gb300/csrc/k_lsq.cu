// Least-squares INUFFT for M > N (problem (ii) of Sec. 2 with more samples
// than coefficients): c = argmin sum_j w_j |sum_n c_n e^{i n y_j} - g_j|^2,
// by conjugate gradients on the normal equations
//     A^H W A c = A^H W g,   A_jn = e^{i n y_j},  W = diag(w) (or I),
// whose matrix-vector product is one forward NUFFT (A), a scaling by w and
// one adjoint NUFFT (A^H), both through the plan's FMM.  Vectors of length N
// are complex128; inner products are reduced in a fixed order (per-CTA
// partials, then one CTA), so repeated solves are bit-identical; the CG
// scalars stay on the device.  The stopping test is the residual of the
// unweighted normal equations, ||A^H (g - A c)|| / ||A^H g||, recomputed
// from the iterate (one forward and one adjoint FMM) every `check_every`
// iterations, whatever the weights: weighted and plain solves stop on the
// same quantity (for consistent data g = A c_true both tend to c_true).
#include <climits>
#include <cmath>

#include "common.cuh"

using namespace nufft;

namespace {

constexpr int kDotBlocks = 304;  // 2 per SM
constexpr int kCheckEvery = 16;
constexpr int kScalars = 16;

// partial[b] = sum over the CTA's stride of conj(a_i) b_i (real and imaginary)
__global__ void __launch_bounds__(256) k_dot_partial(const double2* __restrict__ a,
                                                     const double2* __restrict__ b, int64_t n,
                                                     double2* __restrict__ partial) {
  __shared__ double2 sh[256];
  double2 acc = make_double2(0, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2 x = a[i], y = b[i];
    acc.x += x.x * y.x + x.y * y.y;
    acc.y += x.x * y.y - x.y * y.x;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out = sum of the partials in a fixed order (one CTA)
__global__ void k_dot_final(const double2* __restrict__ partial, int nb, double2* __restrict__ out) {
  __shared__ double2 sh[512];
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc = cadd(acc, partial[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

// scalars (see nufft_plan_solve_lsq): [0] rr, [1] pAp, [2] rr_new, [3] alpha, [4] beta
__global__ void k_cg_alpha(double2* __restrict__ sc) {
  double pAp = sc[1].x;
  sc[3].x = (pAp > 0.0) ? sc[0].x / pAp : 0.0;
}
__global__ void k_cg_beta(double2* __restrict__ sc) {
  double rr = sc[0].x;
  sc[4].x = (rr > 0.0) ? sc[2].x / rr : 0.0;
  sc[0].x = sc[2].x;
}

// x += alpha p ; r -= alpha Ap
__global__ void k_cg_xr(double2* __restrict__ x, double2* __restrict__ r,
                        const double2* __restrict__ p, const double2* __restrict__ Ap, int64_t n,
                        const double2* __restrict__ sc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double a = sc[3].x;
  double2 pi = p[i], api = Ap[i];
  x[i] = make_double2(fma(a, pi.x, x[i].x), fma(a, pi.y, x[i].y));
  r[i] = make_double2(fma(-a, api.x, r[i].x), fma(-a, api.y, r[i].y));
}

// p = r + beta p
__global__ void k_cg_p(double2* __restrict__ p, const double2* __restrict__ r, int64_t n,
                       const double2* __restrict__ sc) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double b = sc[4].x;
  p[i] = make_double2(fma(b, p[i].x, r[i].x), fma(b, p[i].y, r[i].y));
}

// g_j *= w_j (original point order)
__global__ void k_weight(double2* __restrict__ g, const float* __restrict__ w, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double wi = (double)w[i];
  g[i] = make_double2(g[i].x * wi, g[i].y * wi);
}

// copy (and weight) the samples into the work vector
__global__ void k_copy_weight(const double2* __restrict__ src, double2* __restrict__ dst,
                              const float* __restrict__ w, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double wi = w ? (double)w[i] : 1.0;
  dst[i] = make_double2(src[i].x * wi, src[i].y * wi);
}

// e = g - e  (e holds A c on entry): the data residual, original order
__global__ void k_resid_data(const double2* __restrict__ g, double2* __restrict__ e, int64_t M) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  double2 a = g[i], b = e[i];
  e[i] = make_double2(a.x - b.x, a.y - b.y);
}

// ---- learned circulant preconditioner -------------------------------------
// A^H A acts on coefficients like the band-limited projection of a product
// with the sample density rho(x) (its Toeplitz symbol), so its inverse is
// close to a product with 1/rho, which the density-compensation weights
// w_j ~ 1/rho(y_j) sample: P = F^-1 diag(wt) F (F: DFT of Eq. p1), wt_k the
// weights carried to the grid points.  wt_k = mean of w_j over the points
// whose nearest grid point is k (a run of the sorted leaf), or, for a grid
// point no point rounds to, the value of the nearest grid point that has
// one; wt is divided by N (the DFT's normalisation).  All in a fixed order.

// ws[i] = w[perm[i]] (weights in sorted point order)
__global__ void k_weights_sorted(const float* __restrict__ w, const int32_t* __restrict__ perm,
                                 int64_t M, float* __restrict__ ws) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < M) ws[i] = w[perm[i]];
}

// the run of sorted points of leaf b whose nearest grid point is k (want =
// k - b s), and for want = 0 the tail of leaf b - 1 rounding up to k
__device__ inline void cell_sum(int k, int N, int s, int B, const int32_t* __restrict__ start,
                                const int32_t* __restrict__ k0s, const float* __restrict__ ws,
                                double* sum, int* cnt) {
  const int b = k / s, want = k - b * s;
  int lo = start[b], hi = start[b + 1];
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (((k0s[mid] - b * s) & (N - 1)) < want) lo = mid + 1; else hi = mid;
  }
  double a = 0.0;
  int c = 0;
  for (int i = lo; i < start[b + 1] && ((k0s[i] - b * s) & (N - 1)) == want; ++i) {
    a += (double)ws[i];
    ++c;
  }
  if (want == 0) {
    const int bp = (b - 1) & (B - 1);
    for (int i = start[bp + 1] - 1; i >= start[bp] && ((k0s[i] - bp * s) & (N - 1)) == s; --i) {
      a += (double)ws[i];
      ++c;
    }
  }
  *sum = a;
  *cnt = c;
}

// one CTA of 1024 threads, thread t owning grid points [t C, t C + C):
// cell means, then the nearest occupied grid point for the empty ones
// (periodic), through block-wide max / min scans of the chunks' last / first
// occupied points.  wt[N] (double), tmpi[N] (int scratch).
constexpr int kWtThreads = 1024;
__global__ void __launch_bounds__(kWtThreads) k_grid_weights(
    int N, int s, int B, const int32_t* __restrict__ start, const int32_t* __restrict__ k0s,
    const float* __restrict__ ws, double* __restrict__ wt, int* __restrict__ tmpi) {
  __shared__ int s_last[kWtThreads], s_first[kWtThreads];
  const int t = threadIdx.x;
  const int C = (N + kWtThreads - 1) / kWtThreads;
  const int k0 = t * C, k1 = (k0 + C < N) ? k0 + C : N;
  int last = -1, first = INT_MAX;
  for (int k = k0; k < k1; ++k) {
    double a;
    int c;
    cell_sum(k, N, s, B, start, k0s, ws, &a, &c);
    if (c > 0) {
      wt[k] = a / (double)c;
      last = k;
      if (first == INT_MAX) first = k;
    } else {
      wt[k] = -1.0;
    }
  }
  s_last[t] = last;
  s_first[t] = first;
  __syncthreads();
  // inclusive max scan of s_last (left to right), min scan of s_first (right to left)
  for (int off = 1; off < kWtThreads; off <<= 1) {
    const int a = t >= off ? s_last[t - off] : -1;
    const int f = t + off < kWtThreads ? s_first[t + off] : INT_MAX;
    __syncthreads();
    if (a > s_last[t]) s_last[t] = a;
    if (f < s_first[t]) s_first[t] = f;
    __syncthreads();
  }
  const int glast = s_last[kWtThreads - 1], gfirst = s_first[0];
  // forward: the occupied point at or before k (periodic: the last one, one turn back)
  int prev = t > 0 ? s_last[t - 1] : -1;
  for (int k = k0; k < k1; ++k) {
    if (wt[k] >= 0.0) prev = k;
    tmpi[k] = prev >= 0 ? prev : glast - N;
  }
  // backward: the occupied point at or after k; empty points take the nearer
  // (ties: the one before); occupied points point at themselves
  int next = t + 1 < kWtThreads ? s_first[t + 1] : INT_MAX;
  for (int k = k1 - 1; k >= k0; --k) {
    if (wt[k] >= 0.0) {
      next = k;
      tmpi[k] = k;
      continue;
    }
    const int nx = next != INT_MAX ? next : gfirst + N;
    const int pv = tmpi[k];
    const int src = (k - pv <= nx - k) ? pv : nx;
    tmpi[k] = ((src % N) + N) % N;
  }
  __syncthreads();
  // empty points copy an occupied one (occupied values are not written here)
  for (int k = k0; k < k1; ++k)
    if (tmpi[k] != k) wt[k] = wt[tmpi[k]];
  __syncthreads();
  const double inv_n = 1.0 / (double)N;
  for (int k = k0; k < k1; ++k) wt[k] *= inv_n;
}

// z = r * wt on the grid (complex by real)
__global__ void k_scale_grid(double2* __restrict__ f, const double* __restrict__ wt, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = wt[i];
  f[i] = make_double2(f[i].x * a, f[i].y * a);
}

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

int dot(nufft_plan_s* pl, const double2* a, const double2* b, int64_t n, double2* partial,
        double2* out) {
  k_dot_partial<<<kDotBlocks, 256, 0, pl->stream>>>(a, b, n, partial);
  k_dot_final<<<1, 512, 0, pl->stream>>>(partial, kDotBlocks, out);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

}  // namespace

// kernels and tables of the plan's FFT (k_fft.cu)
template <class T>
int fft_run(const void* in, int in_f64, void* out, int out_f64, cplx<T>* buf, cplx<T>* buf2,
            int64_t N, int batch, int sign, const cplx<T>* tw, cudaStream_t st, int64_t n_in,
            int64_t n_out);

namespace {
// z = P r = F diag(wt) F^H r: the grid values of r (Eq. p1, unscaled; the Nc
// coefficients zero padded to the grid), times wt (which holds the 1/N),
// back to the first Nc coefficients
int apply_precond(nufft_plan_s* pl, const double2* r, double2* z, double2* ftmp, const double* wt) {
  const int64_t N = pl->N;
  int rc = fft_run<double>(r, 1, ftmp, 1, pl->grid2, pl->grid3, N, 1, +1, pl->fft_tw, pl->stream,
                           pl->Nc, 0);
  if (rc) return rc;
  k_scale_grid<<<nblk(N), 256, 0, pl->stream>>>(ftmp, wt, N);
  return fft_run<double>(ftmp, 1, z, 1, pl->grid2, pl->grid3, N, 1, -1, pl->fft_tw, pl->stream,
                         0, pl->Nc);
}
}  // namespace

extern "C" int nufft_plan_solve_lsq(nufft_plan pl, const void* g, const float* w, unsigned mode,
                                    double tol, int maxit, int check_every, void* c,
                                    nufft_lsq_info* info) {
  if (!pl || !g || !c || maxit < 1 || !(tol > 0.0) || check_every < 0) return NUFFT_EINVAL;
  if (mode & ~NUFFT_LSQ_WEIGHTED) return NUFFT_EINVAL;
  if ((pl->flags & NUFFT_IO_C64) || pl->batch != 1) return NUFFT_ENOTSUP;
  const bool weighted = w && (mode & NUFFT_LSQ_WEIGHTED);
  const bool precond = w && !weighted;
  const int check = check_every > 0 ? check_every : kCheckEvery;
  // coefficient vectors have the caller's Nc entries; the preconditioner's
  // grid arrays the FMM grid's Ng
  const int64_t N = pl->Nc, Ng = pl->N, M = pl->M;
  cudaStream_t st = pl->stream;
  // work vectors, created on first use and kept by the plan
  if (!pl->lsq_work) {
    size_t bytes = (size_t)(4 * N + 2 * Ng + M + kDotBlocks + kScalars) * sizeof(double2) +
                   (size_t)Ng * (sizeof(double) + sizeof(int)) + (size_t)M * sizeof(float);
    if (cudaMalloc(&pl->lsq_work, bytes) != cudaSuccess) {
      pl->lsq_work = nullptr;
      return NUFFT_ENOMEM;
    }
  }
  double2* r = (double2*)pl->lsq_work;
  double2* p = r + N;
  double2* Ap = p + N;
  double2* zb = Ap + N;     // preconditioned residual
  double2* ftmp = zb + N;   // [Ng] grid values inside the preconditioner
  double2* gw = ftmp + Ng;  // M samples
  double2* partial = gw + M;
  double2* sc = partial + kDotBlocks;
  double* wt = (double*)(sc + kScalars);  // [Ng] grid weights / Ng
  int* tmpi = (int*)(wt + Ng);            // [Ng]
  float* ws = (float*)(tmpi + Ng);        // [M] weights, sorted order
  double2* z = precond ? zb : r;
  double2* x = (double2*)c;
  const double2* gd = (const double2*)g;
  // scalars: [0] (r, z), [1] pAp, [2] (r, z) new, [3] alpha, [4] beta, [5] |A^H W g|^2,
  // [6] |g - A c|^2, [7] |A^H (g - A c)|^2, [8] |A^H g|^2, [9] |g|^2, [10] |r|^2
  int rc;
  double* hist = info ? info->hist : nullptr;
  const int hist_cap = (info && info->hist) ? info->hist_cap : 0;
  if (info) *info = nufft_lsq_info{0, 0, 0.0, 0.0, 0.0, hist, hist_cap};
  if (precond) {
    k_weights_sorted<<<nblk(M), 256, 0, st>>>(w, pl->perm, M, ws);
    k_grid_weights<<<1, kWtThreads, 0, st>>>((int)Ng, pl->s, pl->B, pl->leaf_start, pl->k0, ws,
                                             wt, tmpi);
    if (cudaGetLastError() != cudaSuccess) return NUFFT_ECUDA;
  }
  // |A^H g|^2 and |g|^2 (the denominators of the unweighted residuals)
  if ((rc = dot(pl, gd, gd, M, partial, sc + 9))) return rc;
  if ((rc = nufft_plan_exec_adj(pl, gd, r))) return rc;
  if ((rc = dot(pl, r, r, N, partial, sc + 8))) return rc;
  // x = 0; r = b (A^H g, or A^H W g for the weighted equations); z = P r; p = z
  if (cudaMemsetAsync(x, 0, N * sizeof(double2), st) != cudaSuccess) return NUFFT_ECUDA;
  if (weighted) {
    k_copy_weight<<<nblk(M), 256, 0, st>>>(gd, gw, w, M);
    if ((rc = nufft_plan_exec_adj(pl, gw, r))) return rc;
  }
  if ((rc = dot(pl, r, r, N, partial, sc + 5))) return rc;
  if (precond && (rc = apply_precond(pl, r, z, ftmp, wt))) return rc;
  if (cudaMemcpyAsync(p, z, N * sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if ((rc = dot(pl, r, z, N, partial, sc + 0))) return rc;
  double2 host[kScalars];
  if (cudaMemcpyAsync(host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  const double bb = host[5].x, bu = host[8].x, gg = host[9].x;
  if (!(bb > 0.0) || !(bu > 0.0)) {  // A^H g = 0: c = 0 solves the normal equations
    if (info) info->data_resid = gg > 0.0 ? 1.0 : 0.0;
    return NUFFT_OK;
  }
  double rel = 1.0, rel_w = 1.0, rel_d = 1.0;
  int it = 0, checks = 0;
  while (it < maxit) {
    // Ap = A^H A p (A^H W A p for the weighted equations)
    if ((rc = nufft_plan_exec_fwd(pl, p, gw))) return rc;
    if (weighted) k_weight<<<nblk(M), 256, 0, st>>>(gw, w, M);
    if ((rc = nufft_plan_exec_adj(pl, gw, Ap))) return rc;
    if ((rc = dot(pl, p, Ap, N, partial, sc + 1))) return rc;
    k_cg_alpha<<<1, 1, 0, st>>>(sc);
    k_cg_xr<<<nblk(N), 256, 0, st>>>(x, r, p, Ap, N, sc);
    if (precond) {
      if ((rc = apply_precond(pl, r, z, ftmp, wt))) return rc;
      if ((rc = dot(pl, r, r, N, partial, sc + 10))) return rc;
    }
    if ((rc = dot(pl, r, z, N, partial, sc + 2))) return rc;
    ++it;
    if (it % check == 0 || it == maxit) {
      // true residuals from the iterate: e = g - A x, u = A^H e (Ap and gw
      // are free until the next iteration)
      if ((rc = nufft_plan_exec_fwd(pl, x, gw))) return rc;
      k_resid_data<<<nblk(M), 256, 0, st>>>(gd, gw, M);
      if ((rc = dot(pl, gw, gw, M, partial, sc + 6))) return rc;
      if ((rc = nufft_plan_exec_adj(pl, gw, Ap))) return rc;
      if ((rc = dot(pl, Ap, Ap, N, partial, sc + 7))) return rc;
      if (cudaMemcpyAsync(host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return NUFFT_ECUDA;
      rel = std::sqrt(host[7].x / bu);
      rel_w = std::sqrt((precond ? host[10].x : host[2].x) / bb);
      rel_d = gg > 0.0 ? std::sqrt(host[6].x / gg) : 0.0;
      if (checks < hist_cap) hist[checks] = rel;
      ++checks;
      if (rel <= tol) break;
    }
    k_cg_beta<<<1, 1, 0, st>>>(sc);
    k_cg_p<<<nblk(N), 256, 0, st>>>(p, z, N, sc);
  }
  if (cudaGetLastError() != cudaSuccess) return NUFFT_ECUDA;
  if (info) *info = nufft_lsq_info{it, checks, rel, rel_w, rel_d, hist, hist_cap};
  return rel <= tol ? NUFFT_OK : NUFFT_ENOTCONV;
}
