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
// tree depth L + d.  The adjoint and the inverse (the same sums with the
// roles of points and grid exchanged) use the same classes as sources:
// class d, its points sorted by leaf of level L + d, is the uniform tree of
// that depth for the near field; the pairs a refined leaf's sources no
// longer meet directly (grid boxes of its interaction lists at levels L + 1
// .. L + d) go through the multipoles of the deep boxes, M2L into those
// grid boxes and their evaluation at the grid points.  This file chooses
// the depths (host) and lays out the class-major copies of the point data
// and the index lists the class launches read.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace nufft {

namespace {

// Class-major copies of the sorted target data: slot i takes sorted point
// idx[i] (packed position of esz bytes, permutation, F and E in FP64 and,
// when Ff is set, FP32).
struct GatherPtrs {
  const double2 *F, *E, *Dt, *S;
  const float2 *Ff, *Ef, *Dtf, *Sf;
  double2 *oF, *oE, *oDt, *oS;
  float2 *oFf, *oEf, *oDtf, *oSf;
};
__global__ void k_ad_gather(int64_t M, const int32_t* __restrict__ idx, int esz,
                            const int32_t* __restrict__ perm, const void* __restrict__ pos,
                            int32_t* __restrict__ operm, void* __restrict__ opos, GatherPtrs g) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t j = idx[i];
  operm[i] = perm[j];
  if (esz == 8)
    reinterpret_cast<uint2*>(opos)[i] = reinterpret_cast<const uint2*>(pos)[j];
  else
    reinterpret_cast<uint4*>(opos)[i] = reinterpret_cast<const uint4*>(pos)[j];
  g.oF[i] = g.F[j];
  g.oE[i] = g.E[j];
  if (g.oFf) {
    g.oFf[i] = g.Ff[j];
    g.oEf[i] = g.Ef[j];
  }
  if (g.oDt) {
    g.oDt[i] = g.Dt[j];
    g.oS[i] = g.S[j];
  }
  if (g.oDtf) {
    g.oDtf[i] = g.Dtf[j];
    g.oSf[i] = g.Sf[j];
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
  const int64_t B = pl->B, M = pl->M, N = pl->N;
  const int L = pl->L, s = pl->s, p = pl->p;
  cudaStream_t st = pl->stream;
  pl->ad_D = 0;
  std::vector<int32_t> start((size_t)B + 1), k0((size_t)M);
  std::vector<double> dl((size_t)M);
  if (cudaMemcpyAsync(start.data(), pl->leaf_start, (B + 1) * 4, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      (M > 0 && (cudaMemcpyAsync(k0.data(), pl->k0, M * 4, cudaMemcpyDeviceToHost, st) !=
                     cudaSuccess ||
                 cudaMemcpyAsync(dl.data(), pl->delta, M * 8, cudaMemcpyDeviceToHost, st) !=
                     cudaSuccess)) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  // (an invalid point set leaves the tree uniform; plan creation reports it)
  if (start[0] != 0 || start[B] != M) return NUFFT_OK;
  for (int64_t b = 0; b < B; ++b)
    if (start[b + 1] < start[b]) return NUFFT_OK;
  std::vector<int> dep((size_t)B);
  const int D = nufft_adaptive_depths(start.data(), B, M, s, dep.data());
  if (D <= 0) return NUFFT_OK;
  const int ls = ilog2i(s);
  // the leaf of level L + c of sorted point j: its position's grid cell
  // (k0 - 1 below the grid point, k0 from it on) >> log2(s_c)
  auto deep_leaf = [&](int64_t j, int c) {
    const int64_t fl = ((dl[j] < 0.0 ? k0[j] - 1 : k0[j]) + N) & (N - 1);
    return fl >> (ls - c);
  };
  // class-major order; within class c: by leaf of level L + c (stable: by
  // offset from the leaf's first grid point, then as sorted)
  std::vector<int32_t> idx((size_t)M);
  std::vector<int32_t> sstart;
  int64_t n = 0;
  for (int c = 0; c <= D; ++c) {
    pl->ad_off[c] = n;
    for (int64_t b = 0; b < B; ++b)
      if (dep[b] == c) {
        const int64_t a0 = n;
        for (int32_t j = start[b]; j < start[b + 1]; ++j) idx[n++] = j;
        std::stable_sort(idx.begin() + a0, idx.begin() + n, [&](int32_t x, int32_t y) {
          return deep_leaf(x, c) < deep_leaf(y, c);
        });
      }
    // leaf starts of level L + c within the class
    pl->ad_soff[c] = (int64_t)sstart.size();
    const int64_t nb = B << c;
    std::vector<int32_t> cnt((size_t)nb + 1, 0);
    for (int64_t i = pl->ad_off[c]; i < n; ++i) ++cnt[(size_t)deep_leaf(idx[i], c) + 1];
    for (int64_t b = 0; b < nb; ++b) cnt[(size_t)b + 1] += cnt[(size_t)b];
    sstart.insert(sstart.end(), cnt.begin(), cnt.end());
  }
  pl->ad_off[D + 1] = n;
  // grid tiles (2 kTgtThreads points) within one leaf of level L + c of a class-c leaf
  const int64_t tpts = 512, ntile = (N + tpts - 1) / tpts;
  std::vector<int32_t> tiles;
  for (int c = 1; c <= D; ++c) {
    pl->ad_tioff[c - 1] = (int64_t)tiles.size();
    std::vector<char> mark((size_t)ntile, 0);
    const int64_t sc = s >> c;
    for (int64_t b = 0; b < B; ++b)
      if (dep[b] == c)
        for (int64_t t = (b * s - sc) >> 9; t <= ((b + 1) * s + sc - 1) >> 9; ++t)
          mark[(size_t)((t + ntile) % ntile)] = 1;
    for (int64_t t = 0; t < ntile; ++t)
      if (mark[(size_t)t]) tiles.push_back((int32_t)t);
  }
  pl->ad_tioff[D] = (int64_t)tiles.size();
  // boxes of the deeper levels (the descendants of the leaves refined that
  // far), their sources (class-major ranges), and the grid boxes whose
  // interaction lists hold them, with the slots (even box {-2, +2, +3}, odd
  // {-3, -2, +2}) as indices into the level's box list
  std::vector<int32_t> box, srange, gbox, gil, rleaf;
  for (int64_t b = 0; b < B; ++b)
    if (dep[b] > 0) {
      rleaf.push_back((int32_t)b);
      rleaf.push_back(dep[b]);
    }
  pl->ad_nrleaf = (int64_t)rleaf.size() / 2;
  for (int c = 1; c <= D; ++c) {
    const int64_t b0 = (int64_t)box.size(), nbl = B << c;
    std::vector<int32_t> at((size_t)nbl, -1);
    for (int64_t b = 0; b < B; ++b) {
      const int db = dep[b];
      if (db < c) continue;
      const int32_t* cs = sstart.data() + pl->ad_soff[db];
      for (int64_t k = 0; k < (int64_t(1) << c); ++k) {
        const int64_t S = (b << c) + k;
        at[(size_t)S] = (int32_t)((int64_t)box.size() - b0);
        box.push_back((int32_t)S);
        const int64_t f0 = S << (db - c), f1 = (S + 1) << (db - c);
        srange.push_back((int32_t)(pl->ad_off[db] + cs[f0]));
        srange.push_back((int32_t)(pl->ad_off[db] + cs[f1]));
      }
    }
    pl->ad_boff[c] = (int64_t)box.size();
    pl->ad_goff[c - 1] = (int64_t)gbox.size();
    std::vector<char> seen((size_t)nbl, 0);
    for (int64_t i = b0; i < (int64_t)box.size(); ++i) {
      const int64_t S = box[(size_t)i];
      const int odd = (int)(S & 1);
      for (int t = 0; t < 3; ++t) {
        const int off = odd ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
        seen[(size_t)((S + off + nbl) & (nbl - 1))] = 1;
      }
    }
    for (int64_t I = 0; I < nbl; ++I) {
      if (!seen[(size_t)I]) continue;
      gbox.push_back((int32_t)I);
      const int odd = (int)(I & 1);
      for (int t = 0; t < 3; ++t) {
        const int off = odd ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
        gil.push_back(at[(size_t)((I + off + nbl) & (nbl - 1))]);
      }
    }
  }
  pl->ad_goff[D] = (int64_t)gbox.size();
  // rho_o^m of the s >> c grid points of a box of level L + c: rho_o = o / s_c - 1/2
  const bool f32 = pl->prec != NUFFT_FP64;
  std::vector<double> tab;
  for (int c = 1; c <= D; ++c) {
    pl->ad_toff[c - 1] = (int64_t)tab.size();
    const int sc = s >> c;
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
  const int64_t nl = (int64_t(2) << (L + D)) - 8;
  const bool inv = pl->Dt != nullptr && pl->Sinv != nullptr;
  int rc;
  if ((rc = ad_alloc(&pl->ad_box, box.size() * 4)) || (rc = ad_alloc(&pl->ad_perm, M * 4)) ||
      (rc = ad_alloc(&pl->ad_pos, M * csz)) || (rc = ad_alloc(&pl->ad_F, M * 16)) ||
      (rc = ad_alloc(&pl->ad_E, M * 16)) ||
      (rc = ad_alloc(&pl->ad_p2m, tab.size() * (f32 ? 4 : 8))) ||
      (rc = ad_alloc(&pl->ad_lexp, nl * p * csz)) ||
      (rc = ad_alloc(&pl->ad_start, sstart.size() * 4)) ||
      (rc = ad_alloc(&pl->ad_tiles, tiles.size() * 4)) ||
      (rc = ad_alloc(&pl->ad_srange, srange.size() * 4)) ||
      (rc = ad_alloc(&pl->ad_gbox, gbox.size() * 4)) ||
      (rc = ad_alloc(&pl->ad_gil, gil.size() * 4)) ||
      (rc = ad_alloc(&pl->ad_mexp, box.size() * p * csz)) ||
      (rc = ad_alloc(&pl->ad_charge, M * csz)) || (rc = ad_alloc(&pl->ad_st, M * csz)) ||
      (rc = ad_alloc(&pl->ad_rleaf, rleaf.size() * 4)))
    return rc;
  if (f32 && ((rc = ad_alloc(&pl->ad_Ff, M * 8)) || (rc = ad_alloc(&pl->ad_Ef, M * 8)))) return rc;
  if (inv && ((rc = ad_alloc(&pl->ad_Dt, M * 16)) || (rc = ad_alloc(&pl->ad_S, M * 16))))
    return rc;
  if (inv && f32 && ((rc = ad_alloc(&pl->ad_Dtf, M * 8)) || (rc = ad_alloc(&pl->ad_Sf, M * 8))))
    return rc;
  std::vector<float> tabf;
  if (f32) tabf.assign(tab.begin(), tab.end());
  int32_t* didx = nullptr;
  if ((rc = ad_alloc(&didx, M * 4))) return rc;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    return bytes == 0 || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  bool ok = up(didx, idx.data(), M * 4) && up(pl->ad_box, box.data(), box.size() * 4) &&
            up(pl->ad_start, sstart.data(), sstart.size() * 4) &&
            up(pl->ad_tiles, tiles.data(), tiles.size() * 4) &&
            up(pl->ad_srange, srange.data(), srange.size() * 4) &&
            up(pl->ad_gbox, gbox.data(), gbox.size() * 4) &&
            up(pl->ad_gil, gil.data(), gil.size() * 4) &&
            up(pl->ad_rleaf, rleaf.data(), rleaf.size() * 4) &&
            (f32 ? up(pl->ad_p2m, tabf.data(), tabf.size() * 4)
                 : up(pl->ad_p2m, tab.data(), tab.size() * 8));
  if (ok) {
    GatherPtrs g{pl->F,     pl->E,     inv ? pl->Dt : nullptr,  inv ? pl->Sinv : nullptr,
                 pl->Ff,    pl->Ef,    inv ? pl->Dtf : nullptr, inv ? pl->Sinvf : nullptr,
                 pl->ad_F,  pl->ad_E,  pl->ad_Dt,               pl->ad_S,
                 pl->ad_Ff, pl->ad_Ef, pl->ad_Dtf,              pl->ad_Sf};
    k_ad_gather<<<(unsigned)((M + 255) / 256), 256, 0, st>>>(M, didx, (int)csz, pl->perm,
                                                             pl->srcpos, pl->ad_perm, pl->ad_pos, g);
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
