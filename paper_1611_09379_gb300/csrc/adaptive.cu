// Adaptive tree depth for the forward transform (plan flag NUFFT_ADAPTIVE).
//
// The tree of Sec. 2.1 is uniform: a target in leaf b meets the 3 s grid
// points of leaves b-1, b, b+1 (the near-field count 3NM/2^L of Sec. 2.4),
// whatever the density of the targets around it.  Where the targets cluster,
// a leaf holds many more targets than grid points; refining such a leaf by
// d levels gives each of its targets a near field of 3 s / 2^d grid points,
// and a local expansion at level L + d.  Because the forward's sources are
// the uniform grid, the source multipoles exist at every level: the deeper
// locals are the downward pass continued below the refined leaves only (L2L
// of the parent plus the M2L of the three boxes of the interaction list,
// whose multipoles come from the grid samples), and the targets of each
// depth class are evaluated by the uniform tree's target kernels with the
// tree depth L + d.  This file chooses the depths (host) and lays out the
// class-major copies of the target data the class launches read.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace nufft {

namespace {

// Class-major copies of the sorted target data: slot i takes sorted point
// idx[i] (packed position of esz bytes, permutation, F and E in FP64 and,
// when Ff is set, FP32).
__global__ void k_ad_gather(int64_t M, const int32_t* __restrict__ idx, int esz,
                            const int32_t* __restrict__ perm, const void* __restrict__ pos,
                            const double2* __restrict__ F, const double2* __restrict__ E,
                            const float2* __restrict__ Ff, const float2* __restrict__ Ef,
                            int32_t* __restrict__ operm, void* __restrict__ opos,
                            double2* __restrict__ oF, double2* __restrict__ oE,
                            float2* __restrict__ oFf, float2* __restrict__ oEf) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t j = idx[i];
  operm[i] = perm[j];
  if (esz == 8)
    reinterpret_cast<uint2*>(opos)[i] = reinterpret_cast<const uint2*>(pos)[j];
  else
    reinterpret_cast<uint4*>(opos)[i] = reinterpret_cast<const uint4*>(pos)[j];
  oF[i] = F[j];
  oE[i] = E[j];
  if (oFf) {
    oFf[i] = Ff[j];
    oEf[i] = Ef[j];
  }
}

int ilog2i(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

template <class X>
int ad_alloc(X** p, size_t bytes) {
  return cudaMalloc((void**)p, bytes ? bytes : 16) == cudaSuccess ? NUFFT_OK : NUFFT_ENOMEM;
}

}  // namespace

}  // namespace nufft

using namespace nufft;

int adaptive_setup(nufft_plan_s* pl) {
  const int64_t B = pl->B, M = pl->M;
  pl->ad_D = 0;
  std::vector<int32_t> start((size_t)B + 1);
  if (cudaMemcpyAsync(start.data(), pl->leaf_start, (B + 1) * 4, cudaMemcpyDeviceToHost,
                      pl->stream) != cudaSuccess ||
      cudaStreamSynchronize(pl->stream) != cudaSuccess)
    return NUFFT_ECUDA;
  // (an invalid point set leaves the tree uniform; plan creation reports it)
  if (start[0] != 0 || start[B] != M) return NUFFT_OK;
  for (int64_t b = 0; b < B; ++b)
    if (start[b + 1] < start[b]) return NUFFT_OK;
  std::vector<int> dep((size_t)B);
  const int D = nufft_adaptive_depths(start.data(), B, M, pl->s, dep.data());
  if (D <= 0) return NUFFT_OK;
  // class-major order (within a class: the sorted order, leaf by leaf)
  std::vector<int32_t> idx((size_t)M);
  int64_t n = 0;
  for (int c = 0; c <= D; ++c) {
    pl->ad_off[c] = n;
    for (int64_t b = 0; b < B; ++b)
      if (dep[b] == c)
        for (int32_t j = start[b]; j < start[b + 1]; ++j) idx[n++] = j;
  }
  pl->ad_off[D + 1] = n;
  // boxes of the deeper levels: the descendants of the leaves refined that far
  std::vector<int32_t> box;
  for (int c = 1; c <= D; ++c) {
    for (int64_t b = 0; b < B; ++b)
      if (dep[b] >= c)
        for (int64_t k = 0; k < (int64_t(1) << c); ++k) box.push_back((int32_t)((b << c) + k));
    pl->ad_boff[c] = (int64_t)box.size();
  }
  // rho_o^m of the s >> c grid points of a box of level L + c: rho_o = o / s_c - 1/2
  const int p = pl->p;
  const bool f32 = pl->prec != NUFFT_FP64;
  std::vector<double> tab;
  for (int c = 1; c <= D; ++c) {
    pl->ad_toff[c - 1] = (int64_t)tab.size();
    const int sc = pl->s >> c;
    for (int o = 0; o < sc; ++o) {
      long double rho = (long double)o / sc - 0.5L, pw = 1;
      for (int m = 0; m < p; ++m) {
        tab.push_back((double)pw);
        pw *= rho;
      }
    }
  }
  pl->ad_toff[D] = (int64_t)tab.size();
  const size_t csz = f32 ? sizeof(float2) : sizeof(double2);
  const int64_t nl = (int64_t(2) << (pl->L + D)) - 8;
  int rc;
  if ((rc = ad_alloc(&pl->ad_box, box.size() * 4)) || (rc = ad_alloc(&pl->ad_perm, M * 4)) ||
      (rc = ad_alloc(&pl->ad_pos, M * csz)) || (rc = ad_alloc(&pl->ad_F, M * 16)) ||
      (rc = ad_alloc(&pl->ad_E, M * 16)) ||
      (rc = ad_alloc(&pl->ad_p2m, tab.size() * (f32 ? 4 : 8))) ||
      (rc = ad_alloc(&pl->ad_lexp, nl * p * csz)))
    return rc;
  if (f32 && ((rc = ad_alloc(&pl->ad_Ff, M * 8)) || (rc = ad_alloc(&pl->ad_Ef, M * 8)))) return rc;
  std::vector<float> tabf;
  if (f32) tabf.assign(tab.begin(), tab.end());
  int32_t* didx = nullptr;
  if ((rc = ad_alloc(&didx, M * 4))) return rc;
  cudaStream_t st = pl->stream;
  bool ok = cudaMemcpyAsync(didx, idx.data(), M * 4, cudaMemcpyHostToDevice, st) == cudaSuccess &&
            cudaMemcpyAsync(pl->ad_box, box.data(), box.size() * 4, cudaMemcpyHostToDevice, st) ==
                cudaSuccess &&
            (f32 ? cudaMemcpyAsync(pl->ad_p2m, tabf.data(), tabf.size() * 4,
                                   cudaMemcpyHostToDevice, st)
                 : cudaMemcpyAsync(pl->ad_p2m, tab.data(), tab.size() * 8,
                                   cudaMemcpyHostToDevice, st)) == cudaSuccess;
  if (ok) {
    k_ad_gather<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(
        M, didx, (int)csz, pl->perm, pl->srcpos, pl->F, pl->E, pl->Ff, pl->Ef, pl->ad_perm,
        pl->ad_pos, pl->ad_F, pl->ad_E, pl->ad_Ff, pl->ad_Ef);
    // (the host vectors are read by the copies: wait before they go)
    ok = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  cudaFree(didx);
  if (!ok) return NUFFT_ECUDA;
  pl->ad_D = D;
  return NUFFT_OK;
}

extern "C" {

int nufft_adaptive_depths(const int32_t* leaf_start, int64_t B, int64_t M, int s, int* depth) {
  if (!leaf_start || !depth || B < 1 || (B & (B - 1)) || s < 1 || (s & (s - 1)) || M < 0 ||
      leaf_start[B] != M)
    return -1;
  int dmax = ilog2i(s) - 3;
  if (dmax > nufft_plan_s::kAdMax) dmax = nufft_plan_s::kAdMax;
  if (dmax < 0) dmax = 0;
  if (M == 0) dmax = 0;  // (no targets: nothing to refine)
  const double nbar = (double)M / (double)B;
  int D = 0;
  for (int64_t b = 0; b < B; ++b) {
    const double nb = (double)leaf_start[b + 1] - (double)leaf_start[b];
    if (nb < 0) return -1;
    int d = 0;
    while (d < dmax && nb >= nbar * (double)(2 << d)) ++d;
    depth[b] = d;
    if (d > D) D = d;
  }
  return D;
}

int nufft_plan_adaptive(nufft_plan pl, int* levels, int64_t count[4]) {
  if (!pl || !levels || !count) return NUFFT_EINVAL;
  *levels = pl->ad_D;
  for (int d = 0; d < 4; ++d)
    count[d] = d <= pl->ad_D ? pl->ad_off[d + 1] - pl->ad_off[d] : 0;
  if (pl->ad_D == 0) count[0] = pl->M;
  return NUFFT_OK;
}

}  // extern "C"
