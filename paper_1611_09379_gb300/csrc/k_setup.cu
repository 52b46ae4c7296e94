// Setting the data structure (Sec. 3.3): bin the non-uniform points y_j
// into the 2^L leaves of the binary tree on the circle (Sec. 2.1) with a
// stable counting sort, and precompute F_j (Eq. p5) and the factor of the
// singular pair.
#include "common.cuh"

namespace nufft {

// Grid coordinates of one point: Y = y N/(2 pi) = k0 + delta, from an exact
// two-product with a double-double 1/(2 pi).  The absolute error of delta is
// below N 2^-105 plus one rounding of delta itself, far smaller than the
// distance of any binary64 y from a grid point, so k0, the sign of delta
// and the leaf index are exact.
__device__ inline void grid_coords(double y, int64_t N, int64_t s, int64_t* k0,
                                   double* delta, int64_t* leaf) {
  double ph = y * kInvTwoPiHi;
  double pl = fma(y, kInvTwoPiHi, -ph);
  pl = fma(y, kInvTwoPiLo, pl);
  double Nd = (double)N;
  double yh = ph * Nd, yl = pl * Nd;  // exact scalings
  double k = rint(yh);
  double d = (yh - k) + yl;            // yh - k is exact
  int64_t kk = (int64_t)k;
  int64_t lf = (d < 0.0) ? (kk - 1) : kk;  // floor(Y) (d never hits 0 for y != 0)
  if (kk == N) kk = 0;
  lf = ((lf % N) + N) % N;
  *k0 = kk;
  *delta = d;
  *leaf = lf / s;
}

__global__ void k_points_grid(const double* __restrict__ y, int64_t M, int64_t N,
                              int s, int32_t* __restrict__ k0o, double* __restrict__ delo,
                              int32_t* __restrict__ leafo, int32_t* __restrict__ count,
                              int* __restrict__ status) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  double v = y[j];
  // [0, 2 pi): every binary64 up to fl(2 pi) lies below the real 2 pi
  if (!(v >= 0.0 && v <= kTwoPiHi)) {
    atomicOr(status, kDevBadPoint);
    v = 0.0;
  }
  int64_t k0, lf;
  double d;
  grid_coords(v, N, s, &k0, &d, &lf);
  k0o[j] = (int32_t)k0;
  delo[j] = d;
  leafo[j] = (int32_t)lf;
  atomicAdd(&count[lf], 1);
}

// ---- exclusive scan of int32 counts (three phases; n <= 2^26) -------------
constexpr int kScanBlock = 1024;

__global__ void k_scan_blocks(const int32_t* __restrict__ in, int64_t n,
                              int32_t* __restrict__ out, int32_t* __restrict__ bsum) {
  __shared__ int32_t sh[kScanBlock];
  int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  int32_t v = (i < n) ? in[i] : 0;
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    int32_t t = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = sh[threadIdx.x] - v;  // exclusive
  if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = sh[threadIdx.x];
}

// one CTA scans the block sums (nb <= 64 * 1024)
__global__ void k_scan_sums(int32_t* __restrict__ bsum, int nb) {
  __shared__ int32_t sh[kScanBlock];
  int per = (nb + kScanBlock - 1) / kScanBlock;
  int base = threadIdx.x * per;
  int32_t loc = 0;
  for (int k = 0; k < per && base + k < nb; ++k) loc += bsum[base + k];
  sh[threadIdx.x] = loc;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    int32_t t = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int32_t run = sh[threadIdx.x] - loc;
  for (int k = 0; k < per && base + k < nb; ++k) {
    int32_t v = bsum[base + k];
    bsum[base + k] = run;
    run += v;
  }
}

__global__ void k_scan_add(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ bsum) {
  int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

// ---- stable scatter ---------------------------------------------------------
// Positions within a leaf are claimed with atomics (order not fixed), then
// each leaf segment is sorted by original index, which restores the stable
// order of a counting sort exactly.
__global__ void k_scatter(const int32_t* __restrict__ leafo, int64_t M,
                          int32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= M) return;
  int32_t pos = atomicAdd(&cursor[leafo[j]], 1);
  perm[pos] = (int32_t)j;
}

constexpr int kSegMax = 8192;  // largest leaf population the segment sort handles

// One CTA per leaf b: bitonic sort of perm[start, end) in shared memory by
// the key (k0 - b s mod N, original index): inside a leaf the points follow
// their nearest grid points (0..s from the leaf's first one), ties in the
// original order.  Sources that share a nearest grid point are then
// contiguous, which the adjoint / inverse target kernel uses.
__global__ void k_segment_sort(int32_t* __restrict__ perm, const int32_t* __restrict__ start,
                               const int32_t* __restrict__ k0o, int N, int s,
                               int* __restrict__ status) {
  extern __shared__ unsigned long long shk[];  // [kSegMax]
  int b = blockIdx.x;
  int32_t a = start[b], e = start[b + 1];
  int n = e - a;
  if (n <= 1) return;
  if (n > kSegMax) {
    if (threadIdx.x == 0) atomicOr(status, kDevSegTooLarge);
    return;
  }
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    unsigned long long key = ~0ull;
    if (i < n) {
      const int32_t j = perm[a + i];
      const unsigned krel = (unsigned)((k0o[j] - b * s) & (N - 1));
      key = ((unsigned long long)krel << 32) | (unsigned)j;
    }
    shk[i] = key;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool up = ((i & k) == 0);
          unsigned long long u = shk[i], v = shk[ixj];
          if ((u > v) == up) { shk[i] = v; shk[ixj] = u; }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[a + i] = (int32_t)(shk[i] & 0xFFFFFFFFull);
}

// Gather the sorted point data and form F_j (Eq. p5) and
// E_j = e^{i pi delta} sin(pi delta)/(pi delta), the exact value of
// -(F_j/2) i (2/t) for the pair (y_j, x_k0), t = 2 pi delta / N: the singular
// part of the nearest grid point, kept finite at the exact hit (E = 1).
__global__ void k_points_finalize(const int32_t* __restrict__ perm, int64_t M, int64_t N,
                                  const int32_t* __restrict__ k0o, const double* __restrict__ delo,
                                  int32_t* __restrict__ k0s, double* __restrict__ dels,
                                  double2* __restrict__ F, double2* __restrict__ E,
                                  float* __restrict__ dels_f, float2* __restrict__ Ff,
                                  float2* __restrict__ Ef) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  int32_t j = perm[i];
  double d = delo[j];
  k0s[i] = k0o[j];
  dels[i] = d;
  double sn, cs;
  sincospi(d, &sn, &cs);  // e^{i pi d}; N y = 2 pi (k0 + d) so e^{i N y} = e^{2 pi i d}
  double invN = 1.0 / (double)N;
  F[i] = make_double2(-2.0 * sn * sn * invN, 2.0 * cs * sn * invN);
  double sinc = (d == 0.0) ? 1.0 : sn / (kPi * d);
  E[i] = make_double2(cs * sinc, sn * sinc);
  if (dels_f) {  // FP32 copies for the mixed path
    dels_f[i] = (float)d;
    Ff[i] = make_float2((float)F[i].x, (float)F[i].y);
    Ef[i] = make_float2((float)(cs * sinc), (float)(sn * sinc));
  }
}

}  // namespace nufft

using namespace nufft;

int setup_configure() {
  return cudaFuncSetAttribute(k_segment_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              kSegMax * (int)sizeof(unsigned long long)) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}


// Host driver: returns a nufft_status.  Temporary buffers come from tmp
// (caller-owned device memory of at least setup_tmp_bytes(M, B) bytes).
static inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t setup_tmp_bytes(int64_t M, int64_t B) {
  size_t nb = (size_t)((B + 1 + kScanBlock - 1) / kScanBlock);
  return align256((size_t)M * 4) + align256((size_t)M * 8) + align256((size_t)M * 4) +
         2 * align256((size_t)(B + 1) * 4) + align256(nb * 4);
}

int setup_points(nufft_plan_s* pl, const double* y, void* tmp) {
  cudaStream_t st = pl->stream;
  int64_t M = pl->M, N = pl->N, B = pl->B;
  // every sub-buffer starts on a 256-byte boundary
  char* t = (char*)tmp;
  int32_t* k0o = (int32_t*)t;            t += align256((size_t)M * 4);
  double* delo = (double*)t;             t += align256((size_t)M * 8);
  int32_t* leafo = (int32_t*)t;          t += align256((size_t)M * 4);
  int32_t* count = (int32_t*)t;          t += align256((size_t)(B + 1) * 4);
  int32_t* cursor = (int32_t*)t;         t += align256((size_t)(B + 1) * 4);
  int32_t* bsum = (int32_t*)t;
  int nb = (int)((B + 1 + kScanBlock - 1) / kScanBlock);
  if (cudaMemsetAsync(count, 0, (B + 1) * 4, st) != cudaSuccess) return NUFFT_ECUDA;
  int th = 256;
  int64_t gb = (M + th - 1) / th;
  k_points_grid<<<(unsigned)gb, th, 0, st>>>(y, M, N, pl->s, k0o, delo, leafo, count, pl->status);
  k_scan_blocks<<<nb, kScanBlock, 0, st>>>(count, B + 1, pl->leaf_start, bsum);
  k_scan_sums<<<1, kScanBlock, 0, st>>>(bsum, nb);
  k_scan_add<<<nb, kScanBlock, 0, st>>>(pl->leaf_start, B + 1, bsum);
  if (cudaMemcpyAsync(cursor, pl->leaf_start, (B + 1) * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  k_scatter<<<(unsigned)gb, th, 0, st>>>(leafo, M, cursor, pl->perm);
  k_segment_sort<<<(unsigned)B, 256, kSegMax * sizeof(unsigned long long), st>>>(
      pl->perm, pl->leaf_start, k0o, (int)N, pl->s, pl->status);
  k_points_finalize<<<(unsigned)gb, th, 0, st>>>(pl->perm, M, N, k0o, delo, pl->k0, pl->delta,
                                                 pl->F, pl->E, pl->delta_f, pl->Ff, pl->Ef);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
