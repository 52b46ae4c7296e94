// Least-squares INUFFT for M > N (problem (ii) of Sec. 2 with more samples
// than coefficients): c = argmin sum_j w_j |sum_n c_n e^{i n y_j} - g_j|^2,
// by conjugate gradients on the normal equations
//     A^H W A c = A^H W g,   A_jn = e^{i n y_j},  W = diag(w) (or I),
// whose matrix-vector product is one forward NUFFT (A), a scaling by w and
// one adjoint NUFFT (A^H), both through the plan's FMM.  Vectors of length N
// are complex128; inner products are reduced in a fixed order (per-CTA
// partials, then one CTA), so repeated solves are bit-identical; the CG
// scalars stay on the device and the host reads the residual only every
// `kCheckEvery` iterations.
#include <cmath>

#include "common.cuh"

using namespace nufft;

namespace {

constexpr int kDotBlocks = 304;  // 2 per SM
constexpr int kCheckEvery = 4;

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

// scalars: [0] rr, [1] pAp, [2] rr_new, [3] alpha, [4] beta, [5] bb (|b|^2)
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

inline unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

int dot(nufft_plan_s* pl, const double2* a, const double2* b, int64_t n, double2* partial,
        double2* out) {
  k_dot_partial<<<kDotBlocks, 256, 0, pl->stream>>>(a, b, n, partial);
  k_dot_final<<<1, 512, 0, pl->stream>>>(partial, kDotBlocks, out);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

}  // namespace

extern "C" int nufft_plan_solve_lsq(nufft_plan pl, const void* g, const float* w, double tol,
                                    int maxit, void* c, int* iters, double* resid) {
  if (!pl || !g || !c || maxit < 1 || !(tol > 0.0)) return NUFFT_EINVAL;
  if ((pl->flags & NUFFT_IO_C64) || pl->batch != 1) return NUFFT_ENOTSUP;
  const int64_t N = pl->N, M = pl->M;
  cudaStream_t st = pl->stream;
  // work vectors, created on first use and kept by the plan
  if (!pl->lsq_work) {
    size_t bytes = (size_t)(4 * N + M + kDotBlocks + 8) * sizeof(double2);
    if (cudaMalloc(&pl->lsq_work, bytes) != cudaSuccess) {
      pl->lsq_work = nullptr;
      return NUFFT_ENOMEM;
    }
  }
  double2* r = (double2*)pl->lsq_work;
  double2* p = r + N;
  double2* Ap = p + N;
  double2* gw = Ap + N;   // M samples
  double2* partial = gw + M;
  double2* sc = partial + kDotBlocks;
  double2* x = (double2*)c;
  int rc;
  // x = 0; r = b = A^H W g; p = r
  if (cudaMemsetAsync(x, 0, N * sizeof(double2), st) != cudaSuccess) return NUFFT_ECUDA;
  k_copy_weight<<<nblk(M), 256, 0, st>>>((const double2*)g, gw, w, M);
  if ((rc = nufft_plan_exec_adj(pl, gw, r))) return rc;
  if (cudaMemcpyAsync(p, r, N * sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if ((rc = dot(pl, r, r, N, partial, sc + 0))) return rc;
  if (cudaMemcpyAsync(sc + 5, sc + 0, sizeof(double2), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  double2 host[6];
  if (cudaMemcpyAsync(host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  const double bb = host[5].x;
  if (!(bb > 0.0)) {  // g = 0: the solution is 0
    if (iters) *iters = 0;
    if (resid) *resid = 0.0;
    return NUFFT_OK;
  }
  double rel = 1.0;
  int it = 0;
  while (it < maxit) {
    // Ap = A^H W A p
    if ((rc = nufft_plan_exec_fwd(pl, p, gw))) return rc;
    if (w) k_weight<<<nblk(M), 256, 0, st>>>(gw, w, M);
    if ((rc = nufft_plan_exec_adj(pl, gw, Ap))) return rc;
    if ((rc = dot(pl, p, Ap, N, partial, sc + 1))) return rc;
    k_cg_alpha<<<1, 1, 0, st>>>(sc);
    k_cg_xr<<<nblk(N), 256, 0, st>>>(x, r, p, Ap, N, sc);
    if ((rc = dot(pl, r, r, N, partial, sc + 2))) return rc;
    ++it;
    if (it % kCheckEvery == 0 || it == maxit) {
      if (cudaMemcpyAsync(host, sc, sizeof(host), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return NUFFT_ECUDA;
      rel = std::sqrt(host[2].x / bb);
      if (rel <= tol) break;
    }
    k_cg_beta<<<1, 1, 0, st>>>(sc);
    k_cg_p<<<nblk(N), 256, 0, st>>>(p, r, N, sc);
  }
  if (cudaGetLastError() != cudaSuccess) return NUFFT_ECUDA;
  if (iters) *iters = it;
  if (resid) *resid = rel;
  return rel <= tol ? NUFFT_OK : NUFFT_ENOTCONV;
}
