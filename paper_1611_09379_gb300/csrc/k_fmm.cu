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
#include <climits>
#include <cmath>

#include <type_traits>

#include <cstdlib>

#include "common.cuh"

namespace nufft {

// caller samples (complex64 or complex128) in the arithmetic type
template <class T> __device__ inline cplx<T> load_in(const double2* p) { return c128_to<T>(*p); }
template <class T> __device__ inline cplx<T> load_in(const float2* p) {
  const float2 v = *p;
  return mk<T>((T)v.x, (T)v.y);
}

// ---------------------------------------------------------------- P2M

// Uniform sources (the grid): every leaf holds s points at the same relative
// positions, so the leaf moments are a product with the table rho_o^m.
template <class T>
__global__ void k_p2m_uniform(TreeDims d, const cplx<T>* __restrict__ q,
                              const T* __restrict__ rp, cplx<T>* __restrict__ mleaf) {
  pdl_wait();
  pdl_trigger();
  int64_t B = int64_t(1) << d.L;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= B * d.pm) return;
  q += blockIdx.y * d.N;
  mleaf += blockIdx.y * d.mstride;
  int64_t b = tid / d.pm;
  int m = (int)(tid - b * d.pm);
  const cplx<T>* qb = q + b * d.s;
  T ar = 0, ai = 0;
  for (int o = 0; o < d.s; ++o) {
    cplx<T> v = qb[o];
    T w = rp[o * d.pm + m];
    ar = fma(v.x, w, ar);
    ai = fma(v.y, w, ai);
  }
  mleaf[b * d.pm + m] = mk<T>(ar, ai);
}


// The same product with the grid samples of kP2mChunk consecutive grid
// points (chunk / s leaves) staged in shared memory by coalesced loads, one
// row of s + 1 per leaf (odd pitch: rows of different leaves fall in
// different banks), and the table rho_o^m beside them; each thread then
// forms outputs (leaf, m) from shared memory.  For s <= kP2mChunk.
constexpr int kP2mChunk = 2048;
template <class T>
size_t p2m_grid_smem(int s, int pm) {
  return ((size_t)(kP2mChunk / s) * (s + 1)) * sizeof(cplx<T>) + (size_t)s * pm * sizeof(T);
}

template <class T>
__global__ void __launch_bounds__(256) k_p2m_grid(TreeDims d, const cplx<T>* __restrict__ q,
                                                  const T* __restrict__ rp,
                                                  cplx<T>* __restrict__ mleaf) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int s = d.s, pm = d.pm;
  const int nlf = kP2mChunk / s;  // leaves per CTA
  cplx<T>* qs = reinterpret_cast<cplx<T>*>(smraw);              // [nlf][s + 1]
  T* rps = reinterpret_cast<T*>(qs + (size_t)nlf * (s + 1));      // [s][pm]
  for (int i = threadIdx.x; i < s * pm; i += blockDim.x) rps[i] = rp[i];
  // (the table is a plan constant: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  q += blockIdx.y * d.N + (int64_t)blockIdx.x * kP2mChunk;
  mleaf += blockIdx.y * d.mstride + (int64_t)blockIdx.x * nlf * pm;
  for (int i = threadIdx.x; i < kP2mChunk; i += blockDim.x) {
    const int lf = i / s;  // s is a power of two
    qs[lf * (s + 1) + (i - lf * s)] = q[i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nlf * pm; e += blockDim.x) {
    const int lf = e / pm, m = e - lf * pm;
    const cplx<T>* row = qs + lf * (s + 1);
    T ar = 0, ai = 0;
    for (int o = 0; o < s; ++o) {
      const cplx<T> v = row[o];
      const T w = rps[o * pm + m];
      ar = fma(v.x, w, ar);
      ai = fma(v.y, w, ai);
    }
    mleaf[e] = mk<T>(ar, ai);
  }
}

// Non-uniform sources: one warp per leaf; a chunk of 32 sources writes
// q rho^m for up to 32 consecutive m (the moments of this pass, nm rows)
// into shared memory, lanes then reduce rows.  The source's offset in the
// leaf comes from its grid index alone: o = (k0 - b s) mod N lies in
// [0, s] for every source binned into leaf b.
template <class T> struct P2mWarps { static constexpr int value = 4; };
constexpr int kP2mPitch = 33;  // row pitch of the tile (odd: no bank conflicts)

template <class T>
size_t p2m_smem(int pm) {
  const int rows = pm < 32 ? pm : 32;
  return (size_t)P2mWarps<T>::value * rows * kP2mPitch * sizeof(cplx<T>);
}

// P2M of leaf b by one warp (tile: rows x kP2mPitch of shared memory): a
// chunk of 32 sources writes q rho^m for up to 32 consecutive m into the
// tile, lanes then reduce rows.  rho = (o + delta) / s - 1/2 in T: 1/s is a
// power of two, so the only roundings are of o + delta and of the final
// subtraction (no division).  qget(i, first) returns the charge of sorted
// source i (first: in the first pass over the moments); out(m, v) stores
// moment m.
// The same over the sources [a, e) of leaf b (a part of the leaf: the
// moments of those sources alone).
template <class T, int PM = 0, class QGet, class Out>
__device__ inline void p2m_range_warp(const TreeDims& d, int64_t b, int32_t a, int32_t e,
                                      int lane, cplx<T>* tile, const int32_t* __restrict__ k0,
                                      const T* __restrict__ delta_t, QGet qget, Out out) {
  const int N = (int)d.N;
  const int bs = (int)b * d.s;
  const T inv_s = (T)1 / (T)d.s;
  const int pmv = PM > 0 ? PM : d.pm;  // (PM <= 32: one pass over the moments)
  for (int mc = 0; mc < pmv; mc += 32) {
    const int nm = pmv - mc < 32 ? pmv - mc : 32;
    T accr = 0, acci = 0;
    // two chunks of 32 sources per step: both chunks' loads (and charge
    // gathers) are issued before either is reduced
    for (int c0 = a; c0 < e; c0 += 64) {
      cplx<T> q[2];
      T rho[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = c0 + 32 * h + lane;
        q[h] = mk<T>(0, 0);
        rho[h] = 0;
        if (i < e) {
          const int o = (k0[i] - bs) & (N - 1);
          rho[h] = fma((T)o + delta_t[i], inv_s, (T)-0.5);
          q[h] = qget(i, mc == 0);
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = c0 + 32 * h;
        if (cb >= e) break;
        T pw = 1;
        for (int m = 0; m < mc; ++m) pw *= rho[h];
#pragma unroll(PM > 0 ? PM : 1)
        for (int m = 0; m < nm; ++m) {
          tile[m * kP2mPitch + lane] = mk<T>(q[h].x * pw, q[h].y * pw);
          pw *= rho[h];
        }
        __syncwarp();
        const int nk = e - cb < 32 ? e - cb : 32;
        if (lane < nm) {
          for (int k = 0; k < nk; ++k) {
            const cplx<T> v = tile[lane * kP2mPitch + k];
            accr += v.x;
            acci += v.y;
          }
        }
        __syncwarp();
      }
    }
    if (lane < nm) out(mc + lane, mk<T>(accr, acci));
  }
}

template <class T, int PM = 0, class QGet, class Out>
__device__ inline void p2m_leaf_warp(const TreeDims& d, int64_t b, int lane, cplx<T>* tile,
                                     const int32_t* __restrict__ start,
                                     const int32_t* __restrict__ k0,
                                     const T* __restrict__ delta_t, QGet qget, Out out) {
  p2m_range_warp<T, PM>(d, b, start[b], start[b + 1], lane, tile, k0, delta_t, qget, out);
}

// P2M for clustered sources, where one warp per leaf would leave the warps of
// the dense leaves with nearly all the work: one warp per chunk of at most
// kP2mChunkSrc sources of one leaf (chunk i: leaf, first, end), its moments
// to part[i]; k_p2m_chunk_sum then adds each leaf's chunks in chunk order,
// so the result does not depend on the schedule.
constexpr int kP2mChunkSrc = 256;
template <class T>
__global__ void __launch_bounds__(128) k_p2m_chunks(TreeDims d, int nchunk,
                                                    const int32_t* __restrict__ chunk,
                                                    const int32_t* __restrict__ k0,
                                                    const T* __restrict__ delta_t,
                                                    const cplx<T>* __restrict__ charge,
                                                    cplx<T>* __restrict__ part) {
  pdl_wait();
  pdl_trigger();
  constexpr int WPB = P2mWarps<T>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rows = d.pm < 32 ? d.pm : 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smraw) + warp * rows * kP2mPitch;
  const int i = blockIdx.x * WPB + warp;
  if (i >= nchunk) return;
  charge += blockIdx.y * d.M_;
  part += ((int64_t)blockIdx.y * nchunk + i) * d.pm;
  p2m_range_warp<T>(
      d, chunk[3 * i], chunk[3 * i + 1], chunk[3 * i + 2], lane, tile, k0, delta_t,
      [&](int j, bool) { return charge[j]; }, [&](int m, cplx<T> v) { part[m] = v; });
}

// mleaf[b][m] = sum of the moments of leaf b's chunks cfirst[b] .. cfirst[b + 1] - 1
template <class T>
__global__ void k_p2m_chunk_sum(TreeDims d, int nchunk, const int32_t* __restrict__ cfirst,
                                const cplx<T>* __restrict__ part, cplx<T>* __restrict__ mleaf) {
  pdl_wait();
  pdl_trigger();
  const int64_t B = int64_t(1) << d.L;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= B * d.pm) return;
  const int64_t b = t / d.pm;
  const int m = (int)(t - b * d.pm);
  part += (int64_t)blockIdx.y * nchunk * d.pm;
  mleaf += blockIdx.y * d.mstride;
  T ar = 0, ai = 0;
  for (int c = cfirst[b]; c < cfirst[b + 1]; ++c) {
    const cplx<T> v = part[(int64_t)c * d.pm + m];
    ar += v.x;
    ai += v.y;
  }
  mleaf[b * d.pm + m] = mk<T>(ar, ai);
}

template <class T>
__global__ void __launch_bounds__(128) k_p2m_nonuniform(TreeDims d,
                                                        const int32_t* __restrict__ start,
                                                        const int32_t* __restrict__ k0,
                                                        const T* __restrict__ delta_t,
                                                        const cplx<T>* __restrict__ charge,
                                                        cplx<T>* __restrict__ mleaf) {
  pdl_wait();
  pdl_trigger();
  constexpr int WPB = P2mWarps<T>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rows = d.pm < 32 ? d.pm : 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smraw) + warp * rows * kP2mPitch;
  const int64_t B = int64_t(1) << d.L;
  const int64_t b = blockIdx.x * WPB + warp;
  if (b >= B) return;
  charge += blockIdx.y * d.M_;
  mleaf += blockIdx.y * d.mstride;
  p2m_leaf_warp<T>(
      d, b, lane, tile, start, k0, delta_t, [&](int i, bool) { return charge[i]; },
      [&](int m, cplx<T> v) { mleaf[b * d.pm + m] = v; });
}

// mleaf[b][m] -= shift[m]: charges of a fixed pattern repeated in every leaf
template <class T>
__global__ void k_leaf_shift(int64_t B, int pm, const double* __restrict__ shift,
                             cplx<T>* __restrict__ mleaf) {
  pdl_wait();
  pdl_trigger();
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= B * pm) return;
  int m = (int)(tid % pm);
  mleaf[tid].x -= (T)shift[m];
}

// ---------------------------------------------------------------- upward pass (M2M)

// M2M of one parent box: M'_m = sum_{k<=m} A_-[m][k] M(left)_k + A_+[m][k] M(right)_k,
// A in shared memory as [sigma][k][m].
template <class T>
__device__ inline cplx<T> m2m_one(const T* __restrict__ A, int pm, int m,
                                  const cplx<T>* __restrict__ c0, const cplx<T>* __restrict__ c1) {
  T ar = 0, ai = 0;
  for (int k = 0; k <= m; ++k) {
    T w0 = A[k * pm + m], w1 = A[pm * pm + k * pm + m];
    cplx<T> x0 = c0[k], x1 = c1[k];
    ar = fma(w0, x0.x, fma(w1, x1.x, ar));
    ai = fma(w0, x0.y, fma(w1, x1.y, ai));
  }
  return mk<T>(ar, ai);
}

// m2m_one over all k < pm (the table is zero for k > m, and fma(0, x, a) = a
// for finite x): the same value, with a loop length that is the same for
// every lane (unrolled where pm is a compile-time constant)
template <class T>
__device__ inline cplx<T> m2m_full(const T* __restrict__ A, int pm, int m,
                                   const cplx<T>* __restrict__ c0, const cplx<T>* __restrict__ c1) {
  T ar = 0, ai = 0;
#pragma unroll
  for (int k = 0; k < pm; ++k) {
    T w0 = A[k * pm + m], w1 = A[pm * pm + k * pm + m];
    cplx<T> x0 = c0[k], x1 = c1[k];
    ar = fma(w0, x0.x, fma(w1, x1.x, ar));
    ai = fma(w0, x0.y, fma(w1, x1.y, ai));
  }
  return mk<T>(ar, ai);
}

// Subtree upward pass: one CTA per box at level lt; its 2^(lb - lt) descendants
// at level lb are reduced level by level in shared memory, every level's
// multipoles written to global memory (M2L needs them all).
template <class T>
__global__ void __launch_bounds__(512) k_up_sub(TreeDims d, int lb, int lt, const T* __restrict__ op,
                                                cplx<T>* __restrict__ mexp) {
  extern __shared__ unsigned char smraw[];
  const int pm = d.pm;
  T* A = reinterpret_cast<T*>(smraw);
  cplx<T>* cur = reinterpret_cast<cplx<T>*>(A + 2 * pm * pm);
  const int depth = lb - lt;
  cplx<T>* nxt = cur + (pm << depth);
  for (int i = threadIdx.x; i < 2 * pm * pm; i += blockDim.x) A[i] = op[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  const int64_t b0 = (int64_t)blockIdx.x << depth;  // first box at level lb
  const cplx<T>* src = mexp + (level_off(lb) + b0) * pm;
  for (int i = threadIdx.x; i < (pm << depth); i += blockDim.x) cur[i] = src[i];
  __syncthreads();
  for (int lev = lb; lev > lt; --lev) {
    const int np = 1 << (lev - 1 - lt);  // parents in this subtree
    cplx<T>* dst = mexp + (level_off(lev - 1) + ((int64_t)blockIdx.x << (lev - 1 - lt))) * pm;
    for (int e = threadIdx.x; e < np * pm; e += blockDim.x) {
      int ip = e / pm, m = e - ip * pm;
      cplx<T> v = m2m_one<T>(A, pm, m, cur + 2 * ip * pm, cur + (2 * ip + 1) * pm);
      nxt[e] = v;
      dst[e] = v;
    }
    __syncthreads();
    cplx<T>* t = cur; cur = nxt; nxt = t;
  }
}

// Top of the upward pass in one CTA: levels lb -> 2 (2^lb <= 32 boxes) in
// shared memory, every level written to global memory.
template <class T>
__global__ void __launch_bounds__(512) k_up_top(TreeDims d, int lb, const T* __restrict__ op,
                                                cplx<T>* __restrict__ mexp) {
  extern __shared__ unsigned char smraw[];
  const int pm = d.pm;
  T* A = reinterpret_cast<T*>(smraw);
  cplx<T>* cur = reinterpret_cast<cplx<T>*>(A + 2 * pm * pm);  // [2^lb * pm]
  cplx<T>* nxt = cur + (pm << lb);                             // [2^(lb-1) * pm]
  for (int i = threadIdx.x; i < 2 * pm * pm; i += blockDim.x) A[i] = op[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  const cplx<T>* src = mexp + level_off(lb) * pm;
  for (int i = threadIdx.x; i < (pm << lb); i += blockDim.x) cur[i] = src[i];
  __syncthreads();
  for (int lev = lb; lev > 2; --lev) {
    const int np = 1 << (lev - 1);
    cplx<T>* par = mexp + level_off(lev - 1) * pm;
    for (int e = threadIdx.x; e < np * pm; e += blockDim.x) {
      int ip = e / pm, m = e - ip * pm;
      cplx<T> v = m2m_one<T>(A, pm, m, cur + 2 * ip * pm, cur + (2 * ip + 1) * pm);
      nxt[e] = v;
      par[e] = v;
    }
    __syncthreads();
    cplx<T>* t = cur; cur = nxt; nxt = t;
  }
}

// Upward pass in one launch.  Stage k reduces level lev[k] to lev[k + 1]
// (lev[0] = L, lev[n] = 2, at most `dmax` levels per stage).  In stage 0 each
// CTA owns one box of level lev[1]: it forms or loads the multipoles of its
// leaves (see UpSrc) and reduces them level by level in shared memory
// (every level written to global memory: M2L needs them all).  A CTA that
// has finished stage k counts itself in the counter of its ancestor at
// level lev[k + 2]; the last CTA of that group (its atomicAdd returns the
// group size - 1) resets the counter to zero and goes on to reduce the
// group's boxes in stage k + 1; the others exit.  No CTA ever waits for
// another.  The writers' results are made visible by __threadfence() before
// the count, and the last CTA reads them from L2.
struct UpStages {
  int n;      // stages
  int dmax;   // largest depth of a stage
  int lev[16];
};

// Leaf multipoles of k_up_fused.  SRC 0: already in mexp (a P2M kernel ran
// before); SRC 1: P2M of the grid samples q (uniform sources), the CTA's
// samples staged in shared memory (one row of s + 1 per leaf), with the
// table rp = rho_o^m; SRC 2: P2M of the sorted non-uniform sources, one warp
// per leaf (p2m_leaf_warp), their charges read from q or, with gin set,
// formed here as coef_i g_perm(i) (conj(coef_i) when conj) and stored to
// `charge` for the near field.  Per signal: q, gin and charge at stride N
// (SRC 1) or M (SRC 2).
template <class T, class VI> struct UpSrc {
  const cplx<T>* q = nullptr;
  const T* rp = nullptr;
  const int32_t* start = nullptr;
  const int32_t* k0 = nullptr;
  const T* delta_t = nullptr;
  const int32_t* perm = nullptr;
  const cplx<T>* coef = nullptr;
  const VI* gin = nullptr;
  cplx<T>* charge = nullptr;
  int conj = 0;
};
constexpr int kUpThreads = 512;  // (1024 for the P2M source modes measured slower)

// dst[e] = src(e) for e < n by the whole CTA, U loads per thread issued
// before any of them is stored, so a thread waits for one memory latency
// per U elements rather than per element (the staging loops of the tree
// passes are latency bound)
template <int U, class V, class Src>
__device__ inline void stage_batched(int n, V* __restrict__ dst, Src src) {
  for (int e0 = threadIdx.x; e0 < n; e0 += U * (int)blockDim.x) {
    V r[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) r[u] = src(e);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) dst[e] = r[u];
    }
  }
}

// PM > 0: the multipole length pm as a compile-time constant (d.pm == PM),
// so the M2M and P2M loops over moments are unrolled and their divisions by
// pm are by a constant; PM = 0: pm from d.
template <class T, int SRC, class VI, int PM = 0>
__global__ void __launch_bounds__(kUpThreads) k_up_fused(TreeDims d, UpStages sg,
                                                         const T* __restrict__ op,
                                                         cplx<T>* __restrict__ mexp,
                                                         int* __restrict__ cnt, int cstride,
                                                         UpSrc<T, VI> src) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_last;
  const int pm = PM > 0 ? PM : d.pm;
  T* A = reinterpret_cast<T*>(smraw);
  cplx<T>* cur0 = reinterpret_cast<cplx<T>*>(A + 2 * pm * pm);  // [pm << dmax]
  cplx<T>* nxt0 = cur0 + (pm << sg.dmax);                       // [pm << (dmax - 1)]
  cplx<T>* xtra = nxt0 + (pm << (sg.dmax - 1));                 // SRC 1 / 2 work area
  for (int i = threadIdx.x; i < 2 * pm * pm; i += blockDim.x) A[i] = op[i];
  const int nl0 = 1 << (sg.lev[0] - sg.lev[1]);  // leaves per CTA in stage 0
  T* rps = reinterpret_cast<T*>(xtra + (size_t)nl0 * (d.s + 1));  // SRC 1: [s][pm]
  if constexpr (SRC == 1)
    for (int i = threadIdx.x; i < d.s * pm; i += blockDim.x) rps[i] = src.rp[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  cnt += blockIdx.y * (int64_t)cstride;
  int64_t box = blockIdx.x;  // box of level lev[k + 1] reduced in stage k
  for (int k = 0; k < sg.n; ++k) {
    const int lb = sg.lev[k], lt = sg.lev[k + 1];
    cplx<T>* lvl = mexp + (level_off(lb) + (box << (lb - lt))) * pm;
    const int nsrc = pm << (lb - lt);
    if (k > 0) {  // written by other CTAs of this grid: read through L2
      stage_batched<4>(nsrc, cur0, [&](int i) { return __ldcg(lvl + i); });
    } else if constexpr (SRC == 0) {
      stage_batched<4>(nsrc, cur0, [&](int i) { return lvl[i]; });
    } else if constexpr (SRC == 1) {
      const int sN = d.s;
      cplx<T>* qs = xtra;  // [nl0][s + 1]
      const cplx<T>* q = src.q + blockIdx.y * d.N + (box << (lb - lt)) * sN;
      {
        const int tot = nl0 * sN;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * kUpThreads) {
          cplx<T> r[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * kUpThreads;
            if (i < tot) r[u] = q[i];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * kUpThreads;
            if (i < tot) {
              const int lf = i / sN;
              qs[lf * (sN + 1) + (i - lf * sN)] = r[u];
            }
          }
        }
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nsrc; e += blockDim.x) {
        const int lf = e / pm, m = e - lf * pm;
        const cplx<T>* row = qs + lf * (sN + 1);
        T ar = 0, ai = 0;
#pragma unroll 8
        for (int o = 0; o < sN; ++o) {
          const cplx<T> v = row[o];
          const T w = rps[o * pm + m];
          ar = fma(v.x, w, ar);
          ai = fma(v.y, w, ai);
        }
        const cplx<T> v = mk<T>(ar, ai);
        cur0[e] = v;
        lvl[e] = v;
      }
    } else {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int rows = pm < 32 ? pm : 32;
      cplx<T>* tile = xtra + warp * rows * kP2mPitch;
      const int64_t b0 = box << (lb - lt);
      const int64_t so = (int64_t)blockIdx.y * d.M_;
      const cplx<T>* chg = src.q ? src.q + so : nullptr;
      const VI* gin = src.gin ? src.gin + so : nullptr;
      cplx<T>* cout = src.charge ? src.charge + so : nullptr;
      for (int lf = warp; lf < nl0; lf += kUpThreads / 32) {
        p2m_leaf_warp<T, PM>(
            d, b0 + lf, lane, tile, src.start, src.k0, src.delta_t,
            [&](int i, bool first) {
              if (!gin) return chg[i];
              cplx<T> c = src.coef[i];
              if (src.conj) c.y = -c.y;
              c = cmul(c, load_in<T>(gin + src.perm[i]));
              if (first) cout[i] = c;
              return c;
            },
            [&](int m, cplx<T> v) {
              cur0[lf * pm + m] = v;
              lvl[lf * pm + m] = v;
            });
      }
    }
    __syncthreads();
    cplx<T>* cur = cur0;
    cplx<T>* nxt = nxt0;
    for (int lev = lb; lev > lt; --lev) {
      const int np = 1 << (lev - 1 - lt);  // parents of this level under `box`
      cplx<T>* dst = mexp + (level_off(lev - 1) + (box << (lev - 1 - lt))) * pm;
      for (int e = threadIdx.x; e < np * pm; e += blockDim.x) {
        int ip = e / pm, m = e - ip * pm;
        cplx<T> v = m2m_full<T>(A, pm, m, cur + 2 * ip * pm, cur + (2 * ip + 1) * pm);
        nxt[e] = v;
        dst[e] = v;
      }
      __syncthreads();
      cplx<T>* t = cur; cur = nxt; nxt = t;
    }
    if (k + 1 == sg.n) break;
    const int lp = sg.lev[k + 2];
    if (threadIdx.x == 0) {
      int* c = cnt + level_off(lp) + (box >> (lt - lp));
      __threadfence();
      const int last = atomicAdd(c, 1) == (1 << (lt - lp)) - 1;
      if (last) {
        atomicExch(c, 0);
        __threadfence();
      }
      s_last = last;
    }
    __syncthreads();
    if (!s_last) return;
    box >>= lt - lp;
  }
}

// shared memory of k_up_fused: the M2M tables and the two level buffers,
// plus the grid samples and table (SRC 1) or the warps' P2M tiles (SRC 2)
template <class T>
size_t up_fused_smem(int pm, const UpStages& sg, int src, int s) {
  size_t b = (size_t)2 * pm * pm * sizeof(T) + (size_t)3 * ((size_t)pm << sg.dmax) / 2 * sizeof(cplx<T>);
  const size_t nl0 = (size_t)1 << (sg.lev[0] - sg.lev[1]);
  if (src == 1) b += nl0 * (s + 1) * sizeof(cplx<T>) + (size_t)s * pm * sizeof(T);
  if (src == 2) b += (size_t)(kUpThreads / 32) * (pm < 32 ? pm : 32) * kP2mPitch * sizeof(cplx<T>);
  return b;
}

// ---------------------------------------------------------------- downward pass (M2L + L2L)

// One output L[l][i][n]: sum over the interaction list (even i: d in
// {-2, +2, +3}; odd i: {-3, -2, +2}; slots 0:-3 1:-2 2:+2 3:+3) plus the L2L
// of the parent.  Tm: [4][p][p] as [slot][m][n]; Tl: [2][p][p] as
// [sigma][n'][n]; msrc(off) returns the multipole vector of box i + off;
// lw (log kernel only) adds M_0 log W_l per interacting box.
template <class T, class MSrc>
__device__ inline cplx<T> m2l_one(const T* __restrict__ Tm, const T* __restrict__ Tl, int p, int n,
                                  int odd, MSrc msrc, const cplx<T>* __restrict__ lpar, T lw) {
  T ar = 0, ai = 0;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int off = odd ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
    const int slot = odd ? t : t + 1;
    const cplx<T>* mv = msrc(off);
    const T* Tt = Tm + slot * p * p + n;
#pragma unroll
    for (int m = 0; m < p; ++m) {
      T w = Tt[m * p];
      cplx<T> x = mv[m];
      ar = fma(w, x.x, ar);
      ai = fma(w, x.y, ai);
    }
    if (n == 0 && lw != (T)0) {
      ar = fma(lw, mv[0].x, ar);
      ai = fma(lw, mv[0].y, ai);
    }
  }
  if (lpar) {
    const T* Tt = Tl + odd * p * p + n;
    for (int k = n; k < p; ++k) {
      T w = Tt[k * p];
      cplx<T> x = lpar[k];
      ar = fma(w, x.x, ar);
      ai = fma(w, x.y, ai);
    }
  }
  return mk<T>(ar, ai);
}

// log W_l of the log kernel (0 for the cot kernel's 1/t expansions)
__device__ inline double level_logw(int log_kernel, int log2N, int l) {
  return log_kernel ? (double)(log2N - l) * 0.6931471805599453 : 0.0;
}

// Top of the downward pass in one CTA: levels 3..lt (2^lt <= 32 boxes), each
// level's multipoles and the locals staged in shared memory.
// L2L of the parent's local expansion into output n of a child (odd: which
// child): sum_{k >= n} Tl[odd][k][n] lpar[k]
template <class T>
__device__ inline cplx<T> l2l_one(const T* __restrict__ Tl, int p, int n, int odd,
                                  const cplx<T>* __restrict__ lpar) {
  T ar = 0, ai = 0;
  const T* Tt = Tl + odd * p * p + n;
  for (int k = n; k < p; ++k) {
    T w = Tt[k * p];
    cplx<T> x = lpar[k];
    ar = fma(w, x.x, ar);
    ai = fma(w, x.y, ai);
  }
  return mk<T>(ar, ai);
}

// l2l_one over all k (the table is zero for k < n, and fma(0, x, a) = a
// for finite x): the same value, with a loop length that is the same for
// every lane
template <class T>
__device__ inline cplx<T> l2l_full(const T* __restrict__ Tl, int p, int n, int odd,
                                   const cplx<T>* __restrict__ lpar) {
  T ar = 0, ai = 0;
  const T* Tt = Tl + odd * p * p + n;
#pragma unroll
  for (int k = 0; k < p; ++k) {
    T w = Tt[k * p];
    cplx<T> x = lpar[k];
    ar = fma(w, x.x, ar);
    ai = fma(w, x.y, ai);
  }
  return mk<T>(ar, ai);
}

template <class T>
__global__ void __launch_bounds__(512) k_down_top(TreeDims d, int lt, const T* __restrict__ op_m2l,
                                                  const T* __restrict__ op_l2l,
                                                  const cplx<T>* __restrict__ mexp,
                                                  cplx<T>* __restrict__ lexp, int log_kernel,
                                                  int log2N) {
  extern __shared__ unsigned char smraw[];
  const int p = d.p, pm = d.pm;
  const int nmax = 1 << lt;
  T* Tm = reinterpret_cast<T*>(smraw);
  T* Tl = Tm + 4 * p * p;
  cplx<T>* Ms = reinterpret_cast<cplx<T>*>(Tl + 2 * p * p);  // [nmax * p]
  cplx<T>* La = Ms + nmax * p;                               // [nmax * p]
  cplx<T>* Lb = La + nmax * p;                               // [nmax * p]
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  lexp += blockIdx.y * d.lstride;
  cplx<T>* par = La;
  cplx<T>* cur = Lb;
  for (int l = 3; l <= lt; ++l) {
    const int nb = 1 << l;
    cplx<T>* lout = lexp + (level_off(l) - 4) * p;
    const cplx<T>* ml = mexp + level_off(l) * pm;
    __syncthreads();
    for (int e = threadIdx.x; e < nb * p; e += blockDim.x) {
      int i = e / p, m = e - i * p;
      Ms[e] = ml[(int64_t)i * pm + m];
    }
    __syncthreads();
    const T lw = log_kernel ? (T)level_logw(log_kernel, log2N, l) : (T)0;
    for (int e = threadIdx.x; e < nb * p; e += blockDim.x) {
      int i = e / p, n = e - i * p;
      auto msrc = [&](int off) { return Ms + ((i + off + nb) & (nb - 1)) * p; };
      cplx<T> v = m2l_one<T>(Tm, Tl, p, n, i & 1, msrc, l > 3 ? par + (i >> 1) * p : nullptr, lw);
      cur[e] = v;
      lout[e] = v;
    }
    cplx<T>* t = par; par = cur; cur = t;
  }
}

// Subtree downward pass: one CTA per box at level lt (whose local expansion
// is in global memory); levels lt+1..lb of its 2^(lb-lt) descendants are
// formed in shared memory: the multipoles of the boxes and their +-3
// neighbours are staged per level, the parents' locals stay on chip.  Only
// level lb is written back.
template <class T>
__global__ void __launch_bounds__(512) k_down_sub(TreeDims d, int lt, int lb,
                                                  const T* __restrict__ op_m2l,
                                                  const T* __restrict__ op_l2l,
                                                  const cplx<T>* __restrict__ mexp,
                                                  cplx<T>* __restrict__ lexp, int log_kernel,
                                                  int log2N) {
  extern __shared__ unsigned char smraw[];
  const int p = d.p, pm = d.pm;
  const int depth = lb - lt;
  T* Tm = reinterpret_cast<T*>(smraw);
  T* Tl = Tm + 4 * p * p;
  cplx<T>* Ms = reinterpret_cast<cplx<T>*>(Tl + 2 * p * p);  // [(2^depth + 6) * p]
  cplx<T>* La = Ms + ((1 << depth) + 6) * p;                 // [2^depth * p]
  cplx<T>* Lb = La + (p << depth);                           // [2^depth * p]
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  lexp += blockIdx.y * d.lstride;
  // root local expansion
  const cplx<T>* lroot = lexp + (level_off(lt) - 4 + blockIdx.x) * (int64_t)p;
  for (int i = threadIdx.x; i < p; i += blockDim.x) La[i] = lroot[i];
  cplx<T>* par = La;
  cplx<T>* cur = Lb;
  for (int l = lt + 1; l <= lb; ++l) {
    const int nbx = 1 << (l - lt);          // boxes of this subtree at level l
    const int nb = 1 << l;
    const int c0 = blockIdx.x << (l - lt);  // first box
    const cplx<T>* ml = mexp + level_off(l) * pm;
    __syncthreads();  // previous level finished with Ms
    for (int e = threadIdx.x; e < (nbx + 6) * p; e += blockDim.x) {
      int bi = e / p, m = e - bi * p;
      int box = (c0 - 3 + bi + nb) & (nb - 1);
      Ms[e] = ml[(int64_t)box * pm + m];
    }
    __syncthreads();
    const T lw = log_kernel ? (T)level_logw(log_kernel, log2N, l) : (T)0;
    for (int e = threadIdx.x; e < nbx * p; e += blockDim.x) {
      int bi = e / p, n = e - bi * p;
      auto msrc = [&](int off) { return Ms + (bi + 3 + off) * p; };
      cur[e] = m2l_one<T>(Tm, Tl, p, n, (c0 + bi) & 1, msrc, par + (bi >> 1) * p, lw);
    }
    cplx<T>* t = par; par = cur; cur = t;
  }
  __syncthreads();
  // par holds level lb
  cplx<T>* dst = lexp + (level_off(lb) - 4 + ((int64_t)blockIdx.x << depth)) * p;
  for (int i = threadIdx.x; i < (p << depth); i += blockDim.x) dst[i] = par[i];
}

// Downward pass in one launch: CTA c owns box c of level lt and its subtree
// down to level lb.  The M2L parts of every box it needs -- the subtree's
// boxes of levels lt + 1 .. lb and the ancestors a_l = c >> (lt - l),
// l = 3 .. lt -- depend on multipoles only, so they are formed at once by
// all threads from multipoles staged in shared memory.  Then the L2L chain:
// the ancestors' in one warp,
//   Loc_3 = Lambda_3(a_3),  Loc_l = Lambda_l(a_l) + L2L_{a_l & 1}(Loc_{l-1}),
// (every CTA repeats its own ancestors' chain, (lt - 2)(3 p^2 + p^2 / 2)
// multiply-adds, so no CTA waits for another), then the subtree's levels in
// place.  Only level lb is written back.  P > 0: the expansion length p as
// a compile-time constant (d.p == P), so every loop over coefficients is
// unrolled and every index into the tables is a constant offset; P = 0:
// p from d.  512 threads.
constexpr int kDownThreads = 512;
template <class T, int P = 0>
__global__ void __launch_bounds__(kDownThreads) k_down_fused(TreeDims d, int lt, int lb,
                                                    const T* __restrict__ op_m2l,
                                                    const T* __restrict__ op_l2l,
                                                    const cplx<T>* __restrict__ mexp,
                                                    cplx<T>* __restrict__ lexp, int log_kernel,
                                                    int log2N) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = P > 0 ? P : d.p, pm = d.pm;
  const int depth = lb - lt;
  const int na = lt - 2;  // ancestors' levels 3..lt
  // level l = lt + j (j = 1..depth): its 2^j boxes' parts at Lam + (2^j - 2) p,
  // its staged multipoles (boxes -3 .. 2^j + 2) at Ms + (2^j - 2 + 6 (j - 1)) p
  const int nlam = ((2 << depth) - 2) * p;
  T* Tm = reinterpret_cast<T*>(smraw);
  T* Tl = Tm + 4 * p * p;
  cplx<T>* Ms = reinterpret_cast<cplx<T>*>(Tl + 2 * p * p);  // [nlam + 6 depth p]
  cplx<T>* Lam = Ms + nlam + 6 * depth * p;                  // [nlam]
  cplx<T>* An = Lam + nlam;                                  // [na][3][p]
  cplx<T>* AL = An + na * 3 * p;                             // [na][p]
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  // (operator tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  mexp += blockIdx.y * d.mstride;
  lexp += blockIdx.y * d.lstride;
  const int64_t c = blockIdx.x;
  // slot t of the interaction list: even box {-2, +2, +3}, odd {-3, -2, +2}
  auto list_off = [](int odd, int t) {
    return odd ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
  };
  stage_batched<4>(na * 3 * p, An, [&](int e) {
    const int li = e / (3 * p), r = e - li * 3 * p, t = r / p, m = r - t * p;
    const int l = 3 + li;
    const int64_t a = c >> (lt - l), nb = int64_t(1) << l;
    const int64_t box = (a + list_off((int)(a & 1), t) + nb) & (nb - 1);
    return mexp[(level_off(l) + box) * pm + m];
  });
  // the subtree levels' multipoles (boxes -3 .. 2^j + 2 of level lt + j) in
  // one flat pass: element e of Ms lies in level j with (2^j - 2 + 6 (j - 1)) p
  // <= e < (2^(j+1) - 2 + 6 j) p
  stage_batched<4>((((2 << depth) - 2) + 6 * depth) * p, Ms, [&](int e) {
    int j = 1;
    while (j < depth && e >= ((2 << j) - 2 + 6 * j) * p) ++j;
    const int r = e - ((1 << j) - 2 + 6 * (j - 1)) * p;
    const int bi = r / p, m = r - bi * p;
    const int l = lt + j;
    const int64_t nb = int64_t(1) << l, c0 = c << j;
    const int64_t box = (c0 - 3 + bi + nb) & (nb - 1);
    return mexp[(level_off(l) + box) * pm + m];
  });
  __syncthreads();
  // M2L parts: the ancestors' and, level by level, the subtree's; a thread's
  // outputs (box bi, coefficient n) advance by kDownThreads = sb p + sn
  const int sb = kDownThreads / p, sn = kDownThreads - sb * p;
  for (int e = threadIdx.x; e < na * p; e += kDownThreads) {
    const int li = e / p, n = e - li * p;
    const int l = 3 + li;
    const int odd = (int)((c >> (lt - l)) & 1);
    const cplx<T>* mv = An + li * 3 * p;
    auto msrc = [&](int off) {
      const int t = odd ? (off == -3 ? 0 : (off == -2 ? 1 : 2)) : (off == -2 ? 0 : (off == 2 ? 1 : 2));
      return mv + t * p;
    };
    const T lw = log_kernel ? (T)level_logw(log_kernel, log2N, l) : (T)0;
    AL[e] = m2l_one<T>(Tm, Tl, p, n, odd, msrc, nullptr, lw);
  }
  const int bi0 = (int)threadIdx.x / p, n0 = (int)threadIdx.x - bi0 * p;
  for (int j = 1; j <= depth; ++j) {
    const int nbx = 1 << j;
    const cplx<T>* ms = Ms + (nbx - 2 + 6 * (j - 1)) * p;
    cplx<T>* lam = Lam + (nbx - 2) * p;
    const T lw = log_kernel ? (T)level_logw(log_kernel, log2N, lt + j) : (T)0;
    for (int bi = bi0, n = n0; bi < nbx;) {
      auto msrc = [&](int off) { return ms + (bi + 3 + off) * p; };
      lam[bi * p + n] = m2l_one<T>(Tm, Tl, p, n, bi & 1, msrc, nullptr, lw);
      bi += sb;
      n += sn;
      if (n >= p) { n -= p; ++bi; }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int li = 1; li < na; ++li) {
      const int odd = (int)((c >> (lt - 3 - li)) & 1);
      for (int n = threadIdx.x; n < p; n += 32)
        AL[li * p + n] = cadd(AL[li * p + n], l2l_full<T>(Tl, p, n, odd, AL + (li - 1) * p));
      __syncwarp();
    }
  }
  // the subtree's levels in place, from the root's local AL[na - 1]
  for (int j = 1; j <= depth; ++j) {
    __syncthreads();  // the parent level is complete
    const int nbx = 1 << j;
    cplx<T>* cur = Lam + (nbx - 2) * p;
    const cplx<T>* par = j == 1 ? AL + (na - 1) * p : Lam + (nbx / 2 - 2) * p;
    for (int bi = bi0, n = n0; bi < nbx;) {
      cur[bi * p + n] = cadd(cur[bi * p + n], l2l_full<T>(Tl, p, n, bi & 1, par + (bi >> 1) * p));
      bi += sb;
      n += sn;
      if (n >= p) { n -= p; ++bi; }
    }
  }
  __syncthreads();
  const cplx<T>* fin = Lam + ((1 << depth) - 2) * p;
  cplx<T>* dst = lexp + (level_off(lb) - 4 + (c << depth)) * p;
  for (int i = threadIdx.x; i < (p << depth); i += kDownThreads) dst[i] = fin[i];
}

// The downward pass continued below the leaf level L where the tree is
// refined (adaptive depth, forward only): one CTA per refined leaf b (the
// list `rleaf`: leaf, depth d_b), which runs the levels L + 1 .. L + d_b of its
// subtree one after the other, a warp per box.  The local expansion of box B
// of level l is the L2L of its parent's (level l - 1: the plan's locals
// `lmain` for l - 1 = L, else this pass's `lad`) plus the M2L of the three
// boxes of its interaction list.  The sources are the grid at every level,
// so the warp forms those boxes' multipoles itself from the grid samples:
// M_m = sum_o f_{I s_l + o} rho_o^m over the s_l = N >> l points of box I
// (rho_o = o / s_l - 1/2, the table rp[l - L - 1], [s_l][p]), the P2M of
// Sec. 2.1 at level l.  A subtree needs nothing from another leaf's, so one
// launch covers every level.  lad: the locals in the plan's layout of levels
// 3..L + 3.
constexpr int kDeepWarps = 8;
template <class T> struct DeepTabs {
  const T* rp[3];
};
template <class T>
__global__ void __launch_bounds__(kDeepWarps * 32) k_down_deep(
    TreeDims d, const int32_t* __restrict__ rleaf, DeepTabs<T> tabs,
    const T* __restrict__ op_m2l, const T* __restrict__ op_l2l, const cplx<T>* __restrict__ f,
    const cplx<T>* __restrict__ lmain, cplx<T>* __restrict__ lad) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = d.p;
  T* Tm = reinterpret_cast<T*>(smraw);
  T* Tl = Tm + 4 * p * p;
  cplx<T>* Mv = reinterpret_cast<cplx<T>*>(Tl + 2 * p * p);  // [kDeepWarps][3 p]
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int64_t b = rleaf[2 * blockIdx.x];
  const int db = rleaf[2 * blockIdx.x + 1];
  cplx<T>* mv = Mv + w * 3 * p;
  for (int c = 1; c <= db; ++c) {
    const int l = d.L + c;
    const int64_t nb = int64_t(1) << l;
    const int sl = (int)(d.N >> l);
    const T* __restrict__ rp = tabs.rp[c - 1];
    const cplx<T>* lpb = c == 1 ? lmain : lad;
    for (int j = w; j < (1 << c); j += kDeepWarps) {
      const int64_t B = (b << c) + j;
      const int odd = (int)(B & 1);
      // multipoles of the interaction list (slot t: even box {-2, +2, +3}, odd {-3, -2, +2})
      for (int e = lane; e < 3 * p; e += 32) {
        const int t = e / p, m = e - t * p;
        const int off = odd ? (t == 0 ? -3 : (t == 1 ? -2 : 2)) : (t == 0 ? -2 : (t == 1 ? 2 : 3));
        const int64_t I = (B + off + nb) & (nb - 1);
        const cplx<T>* fb = f + I * sl;
        // (two partial sums, the loads of several steps in flight: s_l >= 8, even)
        T ar = 0, ai = 0, br = 0, bi = 0;
#pragma unroll 4
        for (int o = 0; o < sl; o += 2) {
          const cplx<T> v0 = fb[o], v1 = fb[o + 1];
          const T w0 = rp[o * p + m], w1 = rp[(o + 1) * p + m];
          ar = fma(v0.x, w0, ar);
          ai = fma(v0.y, w0, ai);
          br = fma(v1.x, w1, br);
          bi = fma(v1.y, w1, bi);
        }
        mv[e] = mk<T>(ar + br, ai + bi);
      }
      __syncwarp();
      const cplx<T>* lpar = lpb + (level_off(l - 1) - 4 + (B >> 1)) * p;
      auto msrc = [&](int off) {
        const int t = odd ? (off == -3 ? 0 : (off == -2 ? 1 : 2)) : (off == -2 ? 0 : (off == 2 ? 1 : 2));
        return mv + t * p;
      };
      for (int n = lane; n < p; n += 32)
        lad[(level_off(l) - 4 + B) * p + n] = m2l_one<T>(Tm, Tl, p, n, odd, msrc, lpar, (T)0);
      __syncwarp();  // (mv is rewritten by the warp's next box)
    }
    __syncthreads();  // level l complete: the parents of level l + 1
  }
}

// expansion lengths with a compile-time instance of the one-launch tree
// passes (FP32); other lengths take the run-time instance
#define NUFFT_TREE_P_LIST(X) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(16)

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
// op: [4][nq][nq] = W1, W2, S-, S+.  out: [4][nq] then Q = sum of charges,
// in FP64 and (outf, optional) rounded to FP32.  One CTA.
template <class T>
__global__ void k_level2(TreeDims d, int nq, const double* __restrict__ op, double c1, double c2,
                         const cplx<T>* __restrict__ mexp, double2* __restrict__ out,
                         float2* __restrict__ outf) {
  pdl_wait();
  pdl_trigger();
  __shared__ double2 mu[4][66];
  __shared__ double2 A1[4][66];
  extern __shared__ double sop[];  // the four weight tables, staged once
  const cplx<T>* m2 = mexp + blockIdx.x * d.mstride;  // level 2 sits at offset 0
  out += blockIdx.x * (4 * nq + 1);
  if (outf) outf += blockIdx.x * (4 * nq + 1);
  for (int e = threadIdx.x; e < 4 * nq * nq; e += blockDim.x) sop[e] = op[e];
  for (int e = threadIdx.x; e < 4 * nq; e += blockDim.x) {
    int a = e / nq, i = e - a * nq;
    double2 v = to_d2(m2[a * d.pm + i]);
    double sc = ldexp((i & 1) ? -1.0 : 1.0, -i);
    mu[a][i] = make_double2(v.x * sc, v.y * sc);
  }
  __syncthreads();
  const double* W1 = sop;
  const double* W2 = sop + nq * nq;
  const double* Sm = sop + 2 * nq * nq;
  const double* Sp = sop + 3 * nq * nq;
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
    if (outf) outf[n * nq + l] = make_float2((float)acc.x, (float)acc.y);
  }
  if (threadIdx.x == 0) {
    double2 qs = make_double2(0, 0);
    for (int a = 0; a < 4; ++a) qs = cadd(qs, to_d2(m2[a * d.pm]));
    out[4 * nq] = qs;
    if (outf) outf[4 * nq] = make_float2((float)qs.x, (float)qs.y);
  }
}

// ---------------------------------------------------------------- evaluation helpers

template <class T>
__device__ inline cplx<T> horner(const cplx<T>* __restrict__ c, int n, T u) {
  cplx<T> acc = c[n - 1];
#pragma unroll 4
  for (int k = n - 2; k >= 0; --k) {
    cplx<T> v = c[k];
    acc.x = fma(acc.x, u, v.x);
    acc.y = fma(acc.y, u, v.y);
  }
  return acc;
}

// horner with the length n = NN a compile-time constant (NN > 0), else run time
template <class T, int NN>
__device__ inline cplx<T> horner_n(const cplx<T>* __restrict__ c, int n, T u) {
  if constexpr (NN > 0) {
    cplx<T> acc = c[NN - 1];
#pragma unroll
    for (int k = NN - 2; k >= 0; --k) {
      const cplx<T> v = c[k];
      acc.x = fma(acc.x, u, v.x);
      acc.y = fma(acc.y, u, v.y);
    }
    return acc;
  } else {
    return horner<T>(c, n, u);
  }
}

// store a result in the caller's element type (complex128 by integer widening)
__device__ inline void store_cplx(double2* p, float2 v) { *p = to_c128(v); }
__device__ inline void store_cplx(double2* p, double2 v) { *p = v; }
__device__ inline void store_cplx(float2* p, float2 v) { *p = v; }
__device__ inline void store_cplx(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

template <class V> __device__ inline void store_out(V* p, double2 v);
template <> __device__ inline void store_out<double2>(double2* p, double2 v) { *p = v; }
template <> __device__ inline void store_out<float2>(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}
template <class V> __device__ inline void store_out_f(V* p, float2 v);
template <> __device__ inline void store_out_f<double2>(double2* p, float2 v) {
  *p = make_double2(v.x, v.y);
}
template <> __device__ inline void store_out_f<float2>(float2* p, float2 v) { *p = v; }

// Exact conversion of a small integer (|D| < 2^22) to T: for FP32 through
// the bit pattern of 1.5 * 2^23 + D (an integer add and one subtraction,
// no conversion instruction).
__device__ inline float int_to_t(int D, float) {
  return __int_as_float(0x4B400000 + D) - 12582912.0f;
}
__device__ inline double int_to_t(int D, double) { return (double)D; }

// 1/t of a near-field pair: rcp_t (common.cuh).

// Near-field accumulation of q / t.  FP64 path: FP64 throughout.  FP32 path:
// FP32 partial sums of up to 16 terms folded into a compensated (Kahan) FP32
// total, so a sum of ~100 terms stays at the 1e-7 level without FP64
// instructions.  Callers add terms in chunks and call fold() between them.
template <class T> struct NearAcc;
template <> struct NearAcc<double> {
  double2 s = make_double2(0, 0);
  __device__ inline void add_r(double2 q, double r) {
    s.x = fma(q.x, r, s.x);
    s.y = fma(q.y, r, s.y);
  }
  __device__ inline void fold() {}
  __device__ inline double2 get() const { return s; }
};
template <> struct NearAcc<float> {
  float2 f = make_float2(0, 0), s = make_float2(0, 0), c = make_float2(0, 0);
  __device__ inline static void kahan(float& sum, float& comp, float v) {
    float y = v - comp;
    float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
  }
  __device__ inline void add_r(float2 q, float r) {
    f.x = fmaf(q.x, r, f.x);
    f.y = fmaf(q.y, r, f.y);
  }
  __device__ inline void fold() {
    kahan(s.x, c.x, f.x);
    kahan(s.y, c.y, f.y);
    f = make_float2(0, 0);
  }
  __device__ inline float2 get() { fold(); return s; }
};

// Two FP32 partial sums (the even and the odd term of each pair of terms),
// added together and folded into the compensated total after every chunk of
// 32 terms, so each partial holds 16 terms, as NearAcc's single partial does
// with chunks of 16.
struct NearAcc2f {
  float2 f = make_float2(0, 0), g = make_float2(0, 0);
  float2 s = make_float2(0, 0), c = make_float2(0, 0);
  __device__ inline void add0(float2 q, float r) {
    f.x = fmaf(q.x, r, f.x);
    f.y = fmaf(q.y, r, f.y);
  }
  __device__ inline void add1(float2 q, float r) {
    g.x = fmaf(q.x, r, g.x);
    g.y = fmaf(q.y, r, g.y);
  }
  __device__ inline void fold() {
    NearAcc<float>::kahan(s.x, c.x, f.x + g.x);
    NearAcc<float>::kahan(s.y, c.y, f.y + g.y);
    f = g = make_float2(0, 0);
  }
};

// ---------------------------------------------------------------- forward targets

// Packed source position for the adjoint / inverse near field: grid index k0
// and offset delta in one 8-byte (FP32) or 16-byte (FP64) load, shared by all
// signals.
template <class T> struct SrcPos;
template <> struct SrcPos<float> { int k0; float dl; };
template <> struct SrcPos<double> { long long k0; double dl; };

// Staged source of the two-point adjoint / inverse near field: position
// (x relative to the CTA, delta) and charge, one 16-byte load in FP32.
template <class T> struct __align__(16) SrcQ {
  cplx<T> rel, q;
};

// Targets per CTA and the capacity of the staged near-field windows.
constexpr int kTgtThreads = 256;
template <class T, int G> struct NearCap {
  // forward: grid samples per signal; adjoint / inverse: sources per chunk
  static constexpr int fwd = (sizeof(T) == 4 ? 2048 : 1024) / G;
  static constexpr int grid = (sizeof(T) == 4 ? 1024 : 512) / G;
  static constexpr size_t fwd_bytes = (size_t)fwd * G * sizeof(cplx<T>);
  static constexpr size_t grid_bytes = (size_t)grid * (1 + 2 * G) * sizeof(cplx<T>);
};

// Near-field sum of one target over window indices [lo, hi): full chunks of
// 16 terms (unrolled, no predicates), then the tail, each chunk folded into
// the compensated total (NearAcc).  term(i, u) adds term i + u; u is a
// compile-time constant inside full chunks.
template <class T, int G, class Term>
__device__ inline void near_window(int lo, int hi, NearAcc<T>* acc, Term term) {
  int i = lo;
  for (; i + 16 <= hi; i += 16) {
#pragma unroll
    for (int u = 0; u < 16; ++u) term(i, u);
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
  if (i < hi) {
    const int n = hi - i;
#pragma unroll
    for (int u = 0; u < 16; ++u)
      if (u < n) term(i, u);
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
}

// near_window with one known excluded index `ex`: term(i, u, check) gets
// std::true_type only in chunks holding the ex of some lane of the warp (a
// warp vote: lo and hi are the same for every lane, so the warp never runs
// both variants of a chunk) and in the tail; the other chunks carry no
// compare / select.
template <class T, int G, class Term>
__device__ inline void near_window_ex(int lo, int hi, int ex, NearAcc<T>* acc, Term term) {
  const unsigned mask = __activemask();
  int i = lo;
  for (; i + 16 <= hi; i += 16) {
    // (several signals per thread: one variant only, the code would not fit)
    if (G > 1 || __any_sync(mask, ex - i >= 0 && ex - i < 16)) {
#pragma unroll
      for (int u = 0; u < 16; ++u) term(i, u, std::true_type());
    } else if (G == 1) {
#pragma unroll
      for (int u = 0; u < 16; ++u) term(i, u, std::false_type());
    }
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
  if (i < hi) {
    for (int u = 0; u < hi - i; ++u) term(i, u, std::true_type());
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
}

// near_window_ex over [0, n), n even, two terms per call: term(i, u, check)
// adds terms i + u and i + u + 1 (u even), so a 16-byte load can fetch both
// FP32 samples.
template <class T, int G, class Term>
__device__ inline void near_window_ex2(int n, int ex, NearAcc<T>* acc, Term term) {
  int i = 0;
  for (; i + 16 <= n; i += 16) {
    if (G > 1 || (ex - i >= 0 && ex - i < 16)) {
#pragma unroll
      for (int u = 0; u < 16; u += 2) term(i, u, std::true_type());
    } else if (G == 1) {
#pragma unroll
      for (int u = 0; u < 16; u += 2) term(i, u, std::false_type());
    }
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
  if (i < n) {
    for (int u = 0; u < n - i; u += 2) term(i, u, std::true_type());
#pragma unroll
    for (int gg = 0; gg < G; ++gg) acc[gg].fold();
  }
}

// near_window_ex2 for one signal: chunks of 32 terms (16 calls), the
// compare variant taken by the whole warp whenever the chunk holds the
// excluded index of any of its lanes (a warp vote; n is the same for every
// lane), so a warp never runs the two variants one after the other.
template <class Term>
__device__ inline void near_window_ex2w(int n, int ex, NearAcc2f& acc, Term term) {
  const unsigned mask = __activemask();
  int i = 0;
  for (; i + 32 <= n; i += 32) {
    if (__any_sync(mask, ex - i >= 0 && ex - i < 32)) {
#pragma unroll
      for (int u = 0; u < 32; u += 2) term(i, u, std::true_type());
    } else {
#pragma unroll
      for (int u = 0; u < 32; u += 2) term(i, u, std::false_type());
    }
    acc.fold();
  }
  // (3s = 48 or 24 terms, the deeper classes of the adaptive tree: a half
  // chunk, voted the same way, before the tail)
  if (i + 16 <= n) {
    if (__any_sync(mask, ex - i >= 0 && ex - i < 16)) {
#pragma unroll
      for (int u = 0; u < 16; u += 2) term(i, u, std::true_type());
    } else {
#pragma unroll
      for (int u = 0; u < 16; u += 2) term(i, u, std::false_type());
    }
    acc.fold();
    i += 16;
  }
  if (i < n) {
    for (int u = 0; u < n - i; u += 2) term(i, u, std::true_type());
    acc.fold();
  }
}

// One thread per sorted target j and group of G signals (Eq. p4, p5, p20):
//   g_j = E_j f_{k0} - (F_j/2) (Q + i h'_j),
//   h'_j = (N/pi) [ (1/s) sum_n L_n u^n + sum_{near, k != k0} f_k / t ]
//          - (2/pi) sum_l D^(arc)_l uhat^l
// where the pair (y_j, x_k0) enters through E_j (its singular 2/t part in
// closed form) and through Q and the regular polynomial like every source.
// Near field: the CTA's 256 targets (sorted, so in leaves bl..bh) draw on the
// grid samples of leaves bl-1..bh+1, staged once in shared memory; a target
// in leaf b reads the 3s samples of leaves b-1, b, b+1 from there, with
// t = (D + delta), D = k0 - k an exact integer in T.  The reciprocals 1/t
// depend on the points only and are shared by the G signals.  A CTA whose
// window exceeds the capacity (sparse targets) reads the samples from global
// memory instead.  All arithmetic in T (F_j, E_j were formed in FP64 at plan
// time).  Signal g of the group: blockIdx.y * G + g; per-signal strides N
// (grid), M (output), d.lstride (locals), 4 (2q) + 1 (level-2 coefficients).
// Split evaluation: with hout set the kernel forms the near-field sums only
// and stores them to hout (it needs the grid samples alone, so it can run
// beside the tree passes); with hnear set it skips them and reads them there.
template <class T, class VO, int G>
__device__ inline void targets_fwd_tile(
    int tile, TreeDims d, int M, const SrcPos<T>* __restrict__ pos,
    const int32_t* __restrict__ perm, const cplx<T>* __restrict__ F,
    const cplx<T>* __restrict__ E, const cplx<T>* __restrict__ fgrid,
    const cplx<T>* __restrict__ lexp, const cplx<T>* __restrict__ lvl2,
    const cplx<T>* __restrict__ hnear, VO* __restrict__ g, cplx<T>* __restrict__ hout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* sf = reinterpret_cast<cplx<T>*>(smraw);  // [G][window]
  __shared__ int s_lo, s_hi;
  const int N = (int)d.N;
  const int s = d.s;
  const int sig0 = blockIdx.y * G;
  fgrid += (int64_t)sig0 * N;
  const int j0 = tile * kTgtThreads;
  const int j = j0 + threadIdx.x;
  const bool act = j < M;
  const int jl = (j0 + kTgtThreads < M ? j0 + kTgtThreads : M) - 1;
  int k0 = 0, b = 0, o = 0;
  T dt = 0;
  if (act) {  // (delta in T has the sign of the FP64 offset: the same leaf)
    const SrcPos<T> ps = pos[j];
    k0 = (int)ps.k0;
    dt = ps.dl;
    point_local(k0, (double)dt, N, s, &b, &o);
  }
  // hnear: near-field sums computed elsewhere (side branch or tensor cores):
  // no window, no barrier, every load of the far part can be in flight at once
  int bl = b, bh = b, nwin = 0;
  bool staged = false;
  if (!hnear) {
    if (threadIdx.x == 0) s_lo = b;
    if (j == jl) s_hi = b;
    __syncthreads();
    bl = s_lo;
    bh = s_hi;
    nwin = (bh - bl + 3) * s;  // samples of leaves bl-1 .. bh+1
    staged = nwin <= NearCap<T, G>::fwd;
    // (targets are sorted by leaf, so b lies in [bl, bh]; checked all the same)
    if (staged) {
      const int base = (bl - 1) * s;
      for (int e = threadIdx.x; e < nwin; e += kTgtThreads) {
        const int k = (base + e + N) & (N - 1);
#pragma unroll
        for (int gg = 0; gg < G; ++gg) sf[gg * nwin + e] = fgrid[(int64_t)gg * N + k];
      }
    }
    __syncthreads();
  }
  if (!act) return;
  NearAcc<T> acc[G];
  // c-th sample of the target's 3 leaves: D = k0 - k = (o + s) - c
  const T D0 = (T)(o + s);
  // per chunk: Di = D0 - i (exact); per term: t0 = Di - u (exact), t = t0 + delta
  // the pair with x_k0 (window index o + s, D = 0) is left out: E_j carries it
  const int ex = o + s;
  if (hnear) {
  } else if (std::is_same<T, float>::value && (s & 1) == 0 && staged && b >= bl && b <= bh) {
    // FP32, even s: samples c, c + 1 (c even) in one 16-byte load (nwin and
    // (b - bl) s are even, so every pair is 16-byte aligned)
    if constexpr (std::is_same<T, float>::value && G == 1) {
      const float2* w = sf + (b - bl) * s;
      NearAcc2f a2;
      near_window_ex2w(3 * s, ex, a2, [&](int i, int u, auto chk) {
        // t_b = t_a - 1 from the rounded t_a: for every included pair
        // |t_b| >= 1/2 and |t_a| <= |t_b| + 1, so t_b keeps a relative
        // error of at most two roundings
        const T ta = (D0 - (T)i) - (T)u, tb = ta - (T)1;
        const T xa = ta + dt;
        T ra = rcp_t(xa), rb = rcp_t(xa - (T)1);
        if (decltype(chk)::value) {
          ra = ta == (T)0 ? (T)0 : ra;
          rb = tb == (T)0 ? (T)0 : rb;
        }
        const float4 q = *reinterpret_cast<const float4*>(w + i + u);
        a2.add0(make_float2(q.x, q.y), ra);
        a2.add1(make_float2(q.z, q.w), rb);
      });
      acc[0].s = a2.s;
      acc[0].c = a2.c;
    } else if constexpr (std::is_same<T, float>::value) {
      const float2* w = sf + (b - bl) * s;
      near_window_ex2<T, G>(3 * s, ex, acc, [&](int i, int u, auto chk) {
        const T ta = (D0 - (T)i) - (T)u, tb = ta - (T)1;
        T ra = rcp_t(ta + dt), rb = rcp_t(tb + dt);
        if (decltype(chk)::value) {
          ra = ta == (T)0 ? (T)0 : ra;
          rb = tb == (T)0 ? (T)0 : rb;
        }
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
          const float4 q = *reinterpret_cast<const float4*>(w + gg * nwin + i + u);
          acc[gg].add_r(make_float2(q.x, q.y), ra);
          acc[gg].add_r(make_float2(q.z, q.w), rb);
        }
      });
    }
  } else if (staged && b >= bl && b <= bh) {
    const cplx<T>* w = sf + (b - bl) * s;  // leaf b - 1 of the window
    near_window_ex<T, G>(0, 3 * s, ex, acc, [&](int i, int u, auto chk) {
      const T t0 = (D0 - (T)i) - (T)u;
      T r = rcp_t(t0 + dt);
      if (decltype(chk)::value) r = t0 == (T)0 ? (T)0 : r;
#pragma unroll
      for (int gg = 0; gg < G; ++gg) acc[gg].add_r(w[gg * nwin + i + u], r);
    });
  } else {
    const int base = (b - 1) * s;
    near_window_ex<T, G>(0, 3 * s, ex, acc, [&](int i, int u, auto chk) {
      const T t0 = (D0 - (T)i) - (T)u;
      T r = rcp_t(t0 + dt);
      if (decltype(chk)::value) r = t0 == (T)0 ? (T)0 : r;
      const int k = (base + i + u + N) & (N - 1);
#pragma unroll
      for (int gg = 0; gg < G; ++gg) acc[gg].add_r(fgrid[(int64_t)gg * N + k], r);
    });
  }
  if (hout) {  // near field only: the rest runs once the tree passes are done
#pragma unroll
    for (int gg = 0; gg < G; ++gg) hout[(int64_t)(sig0 + gg) * M + j] = acc[gg].get();
    return;
  }
  const int base = b * s;
  const int Q2 = 2 * d.q;  // cot kernel: degree 2q-1
  const int arc = b >> (d.L - 2);
  const int I = base + o - arc * (N >> 2) - (N >> 3);
  const T uh = ((T)I + dt) * KConst<T>::two_n(d);
  const T ts = KConst<T>::inv_s(d);
  const T u = fma((T)o + dt, ts, (T)-0.5);
  const T cN = KConst<T>::n_pi(d), c2 = (T)(2.0 * kInvPi);
  const cplx<T> Fj = F[j], Ej = E[j];
  const int pj = perm[j];
#pragma unroll
  for (int gg = 0; gg < G; ++gg) {
    const int sig = sig0 + gg;
    cplx<T> far = mk<T>(0, 0);
    if (d.L >= 3)
      far = horner<T>(lexp + sig * d.lstride + ((int64_t)(level_off(d.L) - 4) + b) * d.p, d.p, u);
    const cplx<T>* l2 = lvl2 + (int64_t)sig * (4 * Q2 + 1);
    cplx<T> reg = horner<T>(l2 + arc * Q2, Q2, uh);
    cplx<T> Qs = l2[4 * Q2];
    cplx<T> nr = hnear ? hnear[(int64_t)sig * M + j] : acc[gg].get();
    T hr = cN * fma(far.x, ts, nr.x) - c2 * reg.x;
    T hi = cN * fma(far.y, ts, nr.y) - c2 * reg.y;
    // g = E f_k0 - (F/2)(Q + i h')
    cplx<T> wv = mk<T>(Qs.x - hi, Qs.y + hr);
    cplx<T> res = cscale(cmul(Fj, wv), (T)-0.5);
    res = cadd(res, cmul(Ej, fgrid[(int64_t)gg * N + k0]));
    store_cplx(g + (int64_t)sig * M + pj, res);
  }
}

// Tiles of 256 sorted targets; a grid of fewer CTAs than tiles loops over
// them (the near-field pass beside the tree passes runs a few CTAs per SM
// only, so the tree kernels keep room on every SM).
template <class T, class VO, int G>
__global__ void __launch_bounds__(kTgtThreads) k_targets_fwd(
    TreeDims d, int M, const SrcPos<T>* __restrict__ pos,
    const int32_t* __restrict__ perm, const cplx<T>* __restrict__ F,
    const cplx<T>* __restrict__ E, const cplx<T>* __restrict__ fgrid,
    const cplx<T>* __restrict__ lexp, const cplx<T>* __restrict__ lvl2,
    const cplx<T>* __restrict__ hnear, VO* __restrict__ g, cplx<T>* __restrict__ hout) {
  pdl_wait();
  pdl_trigger();
  const int ntiles = (M + kTgtThreads - 1) / kTgtThreads;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (tile != (int)blockIdx.x) __syncthreads();  // the previous tile's shared data are read
    targets_fwd_tile<T, VO, G>(tile, d, M, pos, perm, F, E, fgrid, lexp, lvl2, hnear, g, hout);
  }
}

// The far part of the forward targets after the near-field sums were formed
// on the side branch (hnear, sorted order): the same arithmetic as the end of
// k_targets_fwd for one signal, one target per thread with no barrier: every
// load but the target's leaf locals and the sample at k0 is independent of
// the target's position, and those read through L1 (the targets of a CTA
// share a few leaves, and the level-2 coefficients are common to all), so a
// thread waits for two memory latencies.  P > 0: the local expansion length
// as a compile-time constant (d.p == P).
template <class T, class VO, int P = 0>
__global__ void __launch_bounds__(kTgtThreads) k_far_fwd(
    TreeDims d, int M, const SrcPos<T>* __restrict__ pos,
    const int32_t* __restrict__ perm, const cplx<T>* __restrict__ F,
    const cplx<T>* __restrict__ E, const cplx<T>* __restrict__ fgrid,
    const cplx<T>* __restrict__ lexp, const cplx<T>* __restrict__ lvl2,
    const cplx<T>* __restrict__ hnear, VO* __restrict__ g) {
  pdl_wait();
  pdl_trigger();
  const int j = blockIdx.x * kTgtThreads + threadIdx.x;
  if (j >= M) return;
  const int p = P > 0 ? P : d.p;
  const int Q2 = 2 * d.q;
  const int N = (int)d.N;
  const int s = d.s;
  const SrcPos<T> ps = pos[j];
  const int pj = perm[j];
  const cplx<T> Fj = F[j], Ej = E[j], nr = hnear[j];
  const cplx<T> Qs = lvl2[4 * Q2];
  const int k0 = (int)ps.k0;
  const T dt = ps.dl;
  int b, o;
  point_local(k0, (double)dt, N, s, &b, &o);
  const cplx<T> fk = fgrid[k0];
  const int arc = b >> (d.L - 2);
  const int I = b * s + o - arc * (N >> 2) - (N >> 3);
  const T uh = ((T)I + dt) * KConst<T>::two_n(d);
  const T ts = KConst<T>::inv_s(d);
  const T u = fma((T)o + dt, ts, (T)-0.5);
  const T cN = KConst<T>::n_pi(d), c2 = (T)(2.0 * kInvPi);
  cplx<T> far = mk<T>(0, 0);
  if (d.L >= 3)
    far = horner_n<T, P>(lexp + ((int64_t)(level_off(d.L) - 4) + b) * p, p, u);
  const cplx<T> reg = horner<T>(lvl2 + arc * Q2, Q2, uh);
  const T hr = cN * fma(far.x, ts, nr.x) - c2 * reg.x;
  const T hi = cN * fma(far.y, ts, nr.y) - c2 * reg.y;
  const cplx<T> wv = mk<T>(Qs.x - hi, Qs.y + hr);
  cplx<T> res = cscale(cmul(Fj, wv), (T)-0.5);
  res = cadd(res, cmul(Ej, fk));
  store_cplx(g + pj, res);
}

// ---------------------------------------------------------------- adjoint / inverse targets

// Charges in sorted order: adjoint q_i = conj(F_i) g_perm(i);
// inverse q_i = Dt_i g_perm(i) (Eq. p6: D_j g_j, scaled by e^{-Lambda}).
// Signal blockIdx.y: samples and charges at stride M.

template <class T, class VI>
__global__ void k_charges(int64_t M, const int32_t* __restrict__ perm,
                          const cplx<T>* __restrict__ coef, int conj_coef,
                          const VI* __restrict__ gin, cplx<T>* __restrict__ charge) {
  pdl_wait();
  pdl_trigger();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= M) return;
  gin += blockIdx.y * M;
  charge += blockIdx.y * M;
  cplx<T> c = coef[i];
  if (conj_coef) c.y = -c.y;
  charge[i] = cmul(c, load_in<T>(gin + perm[i]));
}

// The pair (y_j, x_k0) of each source j with its nearest grid point, one
// thread per sorted source and signal:
//   adjoint: conj(E_j) g_j, the closed form of the pair's 2/t part (and
//            conj(F_j) G(x_k0 - y_j) -> 1 at an exact hit);
//   inverse: the pair's 2/t part times the target factor, q_j S_j with the
//            plan's per-point factor S_j = i C~_k0 (N / 2pi) / delta_j (finite,
//            as C~_k0 carries sin((x_k0 - y_j)/2); times the general-N phase),
//            1 / (N D~_j) at an exact hit, where C~_k0 = 0 removes every
//            other term (k_assemble_S, in FP64 with an FP32 copy).
// The same quantities for one sorted source i of one signal (the caller
// offsets gin by the signal), in a form the near-field kernels can also
// evaluate while staging their sources: the charge q_i = coef_i g_perm(i)
// (conj(coef_i) for the adjoint) and its self term.
struct SelfArgs {
  int inverse = 0;
  const int32_t* perm = nullptr;
  const void* gin = nullptr;  // caller samples: double2 (gin64) or float2
  int gin64 = 1;
};
template <class T> __device__ inline cplx<T> sample_in(const SelfArgs& a, int64_t idx) {
  return a.gin64 ? load_in<T>((const double2*)a.gin + idx) : load_in<T>((const float2*)a.gin + idx);
}
template <class T>
__device__ inline cplx<T> self_term_of(const SelfArgs& a, int i, cplx<T> q,
                                       const cplx<T>* __restrict__ E,
                                       const cplx<T>* __restrict__ S) {
  if (!a.inverse) return cmul(cconj(E[i]), sample_in<T>(a, a.perm[i]));
  return cmul(q, S[i]);
}

// Charges and self terms formed where they are used (coef non-null), or read
// from the arrays a charge / self-term kernel wrote.
template <class T> struct InlineSrc {
  SelfArgs a;
  const cplx<T>* coef = nullptr;
  const cplx<T>* E = nullptr;
  const cplx<T>* S = nullptr;  // the inverse's self-term factors S_j
};

// The charge of staged source i (returned) and, with need_self, its self
// term (to *st): the values of k_charges and self_term_of, with the caller's
// sample read once for both.
template <class T>
__device__ inline cplx<T> stage_charge_self(const InlineSrc<T>& is, int i, bool need_self,
                                            cplx<T>* st) {
  const SelfArgs& a = is.a;
  const cplx<T> gs = sample_in<T>(a, a.perm[i]);
  cplx<T> c = is.coef[i];
  if (!a.inverse) c.y = -c.y;  // the adjoint's conj(F_i)
  const cplx<T> q = cmul(c, gs);
  if (need_self) *st = a.inverse ? cmul(q, is.S[i]) : cmul(cconj(is.E[i]), gs);
  return q;
}

template <class T, class VI>
__global__ void k_self_terms(int M, int inverse, const int32_t* __restrict__ perm,
                             const cplx<T>* __restrict__ E, const cplx<T>* __restrict__ S,
                             const cplx<T>* __restrict__ charge, const VI* __restrict__ gin,
                             cplx<T>* __restrict__ st) {
  pdl_wait();
  pdl_trigger();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  gin += (int64_t)blockIdx.y * M;
  charge += (int64_t)blockIdx.y * M;
  st += (int64_t)blockIdx.y * M;
  SelfArgs a;
  a.inverse = inverse;
  a.perm = perm;
  a.gin = gin;
  a.gin64 = sizeof(VI) == sizeof(double2);
  st[i] = self_term_of<T>(a, i, inverse ? charge[i] : mk<T>(0, 0), E, S);
}


// Adaptive tree, adjoint / inverse: the multipoles of the deep boxes of
// level l (one warp per box S of the list; its sources are the class-major
// points [range[2i], range[2i + 1])): M_m = sum q rho^m, m < p, with
// rho = (o + delta) / s_l - 1/2 and o = (k0 - S s_l) mod N, the charges formed
// from the caller's samples as in the near-field staging (coef_i g_perm(i),
// conj(coef_i) for the adjoint).  A chunk of 32 sources writes q rho^m for up
// to 32 consecutive m into the warp's tile of shared memory, lanes then
// reduce rows (the P2M of the uniform tree's leaves, on a range).
template <class T>
__global__ void __launch_bounds__(kDeepWarps * 32) k_deep_p2m(
    TreeDims d, int l, int nbox, const int32_t* __restrict__ box,
    const int32_t* __restrict__ range, const SrcPos<T>* __restrict__ pos, InlineSrc<T> isrc,
    cplx<T>* __restrict__ mexp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  pdl_wait();
  pdl_trigger();
  const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int bi = blockIdx.x * kDeepWarps + w;
  if (bi >= nbox) return;
  cplx<T>* tile = reinterpret_cast<cplx<T>*>(smraw) + w * 32 * kP2mPitch;
  const int N = (int)d.N, p = d.p;
  const int sl = (int)(d.N >> l);
  const int bs = box[bi] * sl;
  const int a = range[2 * bi], e = range[2 * bi + 1];
  const T inv_s = (T)1 / (T)sl;
  const SelfArgs& sa = isrc.a;
  for (int mc = 0; mc < p; mc += 32) {
    const int nm = p - mc < 32 ? p - mc : 32;
    T accr = 0, acci = 0;
    for (int c0 = a; c0 < e; c0 += 32) {
      const int i = c0 + lane;
      cplx<T> q = mk<T>(0, 0);
      T rho = 0;
      if (i < e) {
        const SrcPos<T> ps = pos[i];
        rho = fma((T)(((int)ps.k0 - bs) & (N - 1)) + ps.dl, inv_s, (T)-0.5);
        cplx<T> c = isrc.coef[i];
        if (!sa.inverse) c.y = -c.y;  // the adjoint's conj(F_i)
        q = cmul(c, sample_in<T>(sa, sa.perm[i]));
      }
      T pw = 1;
      for (int m = 0; m < mc; ++m) pw *= rho;
      for (int m = 0; m < nm; ++m) {
        tile[m * kP2mPitch + lane] = mk<T>(q.x * pw, q.y * pw);
        pw *= rho;
      }
      __syncwarp();
      const int nk = e - c0 < 32 ? e - c0 : 32;
      if (lane < nm)
        for (int k = 0; k < nk; ++k) {
          const cplx<T> v = tile[lane * kP2mPitch + k];
          accr += v.x;
          acci += v.y;
        }
      __syncwarp();
    }
    if (lane < nm) mexp[(int64_t)bi * p + mc + lane] = mk<T>(accr, acci);
  }
}

// Adaptive tree, adjoint / inverse: grid box I of level l (one warp per box
// of the list `gbox`) receives the M2L of the deep boxes of its interaction
// list (gil: their indices among the level's deep boxes, -1 for a box that
// is not refined that far), and the local expansion is evaluated at its
// s_l grid points and added to their near-field sums in the units the far
// part reads them ((1/s_l) sum_n L_n u^n, u = o / s_l - 1/2): the pairs of
// grid points and sources that the sources' deeper near field no longer
// holds.  Levels run one launch after another, so the additions are ordered.
template <class T>
__global__ void __launch_bounds__(kDeepWarps * 32) k_deep_m2l_grid(
    TreeDims d, int l, int ngbox, const int32_t* __restrict__ gbox,
    const int32_t* __restrict__ gil, const T* __restrict__ op_m2l, const T* __restrict__ op_l2l,
    const cplx<T>* __restrict__ mexp, cplx<T>* __restrict__ hout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int p = d.p;
  T* Tm = reinterpret_cast<T*>(smraw);
  T* Tl = Tm + 4 * p * p;
  cplx<T>* Lw = reinterpret_cast<cplx<T>*>(Tl + 2 * p * p);  // [kDeepWarps][p]
  cplx<T>* Z = Lw + kDeepWarps * p;                            // [p] zeros
  for (int i = threadIdx.x; i < 4 * p * p; i += blockDim.x) Tm[i] = op_m2l[i];
  for (int i = threadIdx.x; i < 2 * p * p; i += blockDim.x) Tl[i] = op_l2l[i];
  for (int i = threadIdx.x; i < p; i += blockDim.x) Z[i] = mk<T>(0, 0);
  pdl_wait();
  pdl_trigger();
  __syncthreads();
  const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int gi = blockIdx.x * kDeepWarps + w;
  if (gi >= ngbox) return;
  const int64_t I = gbox[gi];
  const int odd = (int)(I & 1);
  const int s0 = gil[3 * gi], s1 = gil[3 * gi + 1], s2 = gil[3 * gi + 2];
  auto msrc = [&](int off) {
    const int t = odd ? (off == -3 ? 0 : (off == -2 ? 1 : 2)) : (off == -2 ? 0 : (off == 2 ? 1 : 2));
    const int si = t == 0 ? s0 : (t == 1 ? s1 : s2);
    return si >= 0 ? mexp + (int64_t)si * p : (const cplx<T>*)Z;
  };
  cplx<T>* lw = Lw + w * p;
  for (int n = lane; n < p; n += 32) lw[n] = m2l_one<T>(Tm, Tl, p, n, odd, msrc, nullptr, (T)0);
  __syncwarp();
  const int sl = (int)(d.N >> l);
  const T ts = (T)1 / (T)sl;
  for (int o = lane; o < sl; o += 32) {
    const T u = fma((T)o, ts, (T)-0.5);
    const cplx<T> v = horner<T>(lw, p, u);
    const int64_t k = I * sl + o;
    cplx<T> h = hout[2 * k];
    h.x = fma(v.x, ts, h.x);
    h.y = fma(v.y, ts, h.y);
    hout[2 * k] = h;
  }
}

template <class T>
__global__ void k_pack_positions(int M, const int32_t* __restrict__ k0s,
                                 const double* __restrict__ dels, SrcPos<T>* __restrict__ pos) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  SrcPos<T> r;
  r.k0 = k0s[i];
  r.dl = (T)dels[i];
  pos[i] = r;
}

// One thread per grid point k and group of G signals (Eq. p4 transposed, Eq. p6):
//   h_k = sum_j q_j cot((x_k - y_j)/2)   by the same FMM, then
//   adjoint: u_k   = -(Q + i h'_k)/2 + sum_{j: k0_j = k} st_j
//   inverse: f_k/N = Ct_k (-(Q + i h'_k)/2) + sum_{j: k0_j = k} st_j
// where h' leaves out the 2/t part of the pairs with k0_j = k (their st_j
// terms above); Ct_k = C_k e^Lambda / N carries the 1/N of Eq. p1.
// Near field: the CTA's 256 grid points lie in leaves bl..bh; the sources of
// leaves bl-1..bh+1 (consecutive in sorted order, leaf by leaf, inside a
// leaf by nearest grid point) are staged in shared memory in chunks, each
// with its position x relative to the CTA's first grid point kb (an exact
// integer in T, unwrapped through its leaf slot, non-decreasing along the
// window) and offset delta, its charges and self terms.  A grid point in
// leaf b sums over the sources of leaves b-1, b, b+1: t = (k - kb - x) -
// delta with the first difference exact; the run of sources with x = k - kb
// (found by binary search) contributes its self terms instead.  The
// reciprocals 1/t are shared by the G signals.  All arithmetic in T (Ct in
// FP32 for the mixed path).
template <class T, int G>
__global__ void __launch_bounds__(kTgtThreads) k_targets_grid(
    TreeDims d, int inverse, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, const cplx<T>* __restrict__ lexp,
    const cplx<T>* __restrict__ lvl2, const T* __restrict__ Ct, cplx<T>* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  constexpr int CAP = NearCap<T, G>::grid;
  constexpr int kMaxSlots = kTgtThreads + 3;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* srel = reinterpret_cast<cplx<T>*>(smraw);  // [CAP] (x, delta)
  cplx<T>* sq = srel + CAP;                            // [G][CAP] charges
  cplx<T>* sst = sq + G * CAP;                         // [G][CAP] self terms
  __shared__ int s_off[kMaxSlots + 1];                 // window offsets of the leaf slots
  const int N = (int)d.N;
  const int64_t M = d.M_;
  const int sig0 = blockIdx.y * G;
  charge += sig0 * M;
  st += sig0 * M;
  const int s = d.s;
  const int B = 1 << d.L;
  const int kb = blockIdx.x * kTgtThreads;
  const int k = kb + threadIdx.x;
  const bool act = k < N;
  const int bl = kb / s;
  const int bh = ((kb + kTgtThreads < N ? kb + kTgtThreads : N) - 1) / s;
  const int nslot = bh - bl + 3;  // leaves bl-1 .. bh+1 (<= kMaxSlots)
  // slot sizes, then their offsets in the window (one warp, shuffle scan)
  if (threadIdx.x < 32) {
    int carry = 0;
    for (int c0 = 0; c0 < nslot; c0 += 32) {
      const int js = c0 + threadIdx.x;
      int cnt = 0;
      if (js < nslot) {
        const int bb = (bl - 1 + js + B) & (B - 1);
        cnt = start[bb + 1] - start[bb];
      }
      int v = cnt;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, v, sh);
        if ((int)threadIdx.x >= sh) v += n;
      }
      if (js < nslot) s_off[js + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (threadIdx.x == 0) s_off[0] = 0;
  }
  __syncthreads();
  const int total = s_off[nslot];
  const int b = act ? k / s : bl;
  const int wlo = s_off[b - bl], whi = s_off[b - bl + 3];  // this point's 3 leaves
  const T kf = (T)(k - kb);
  NearAcc<T> acc[G];
  cplx<T> self[G];
#pragma unroll
  for (int gg = 0; gg < G; ++gg) self[gg] = mk<T>(0, 0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < total; c0 += CAP) {
    const int c1 = total - c0 < CAP ? total : c0 + CAP;
    __syncthreads();  // the previous chunk is consumed
    // stage: warp w copies slots w, w + 8, ... (their part inside [c0, c1))
    for (int js = warp; js < nslot; js += kTgtThreads / 32) {
      const int lo = s_off[js] > c0 ? s_off[js] : c0;
      const int hi = s_off[js + 1] < c1 ? s_off[js + 1] : c1;
      if (lo >= hi) continue;
      const int bu = bl - 1 + js;  // unwrapped leaf of the slot
      const int bb = (bu + B) & (B - 1);
      const int g0 = start[bb] - s_off[js];  // global index of window index e: g0 + e
      for (int e = lo + lane; e < hi; e += 32) {
        const int gi = g0 + e;
        const SrcPos<T> ps = pos[gi];
        const int xu = bu * s + (((int)ps.k0 - bb * s) & (N - 1)) - kb;
        srel[e - c0] = mk<T>((T)xu, ps.dl);
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
          sq[gg * CAP + e - c0] = charge[gg * M + gi];
          sst[gg * CAP + e - c0] = st[gg * M + gi];
        }
      }
    }
    __syncthreads();
    const int lo = (wlo > c0 ? wlo : c0) - c0, hi = (whi < c1 ? whi : c1) - c0;
    if (act && lo < hi) {
      // sources with k0_j = k (x = k - kb) form one run of the window, which
      // is sorted by x: their self terms replace their pairs
      int ha = lo, hb = hi;
      while (ha < hb) {
        const int mid = (ha + hb) >> 1;
        if (srel[mid].x < kf) ha = mid + 1; else hb = mid;
      }
      int he = ha;
      while (he < hi && srel[he].x == kf) {
#pragma unroll
        for (int gg = 0; gg < G; ++gg) self[gg] = cadd(self[gg], sst[gg * CAP + he]);
        ++he;
      }
      auto term = [&](int i, int u) {
        const cplx<T> rp = srel[i + u];
        const T r = rcp_t((kf - rp.x) - rp.y);
#pragma unroll
        for (int gg = 0; gg < G; ++gg) acc[gg].add_r(sq[gg * CAP + i + u], r);
      };
      near_window<T, G>(lo, ha, acc, term);
      near_window<T, G>(he, hi, acc, term);
    }
  }
  if (!act) return;
  const int o = k - b * s;
  const int Q2 = 2 * d.q;
  const int arc = b >> (d.L - 2);
  const int I = k - arc * (N >> 2) - (N >> 3);
  const T uh = (T)I * KConst<T>::two_n(d);
  const T ts = KConst<T>::inv_s(d);
  const T u = fma((T)o, ts, (T)-0.5);
  const T cN = KConst<T>::n_pi(d), c2 = (T)(2.0 * kInvPi);
#pragma unroll
  for (int gg = 0; gg < G; ++gg) {
    const int sig = sig0 + gg;
    cplx<T> far = mk<T>(0, 0);
    if (d.L >= 3)
      far = horner<T>(lexp + sig * d.lstride + ((int64_t)(level_off(d.L) - 4) + b) * d.p, d.p, u);
    const cplx<T>* l2 = lvl2 + (int64_t)sig * (4 * Q2 + 1);
    cplx<T> reg = horner<T>(l2 + arc * Q2, Q2, uh);
    cplx<T> Qs = l2[4 * Q2];
    cplx<T> nr = acc[gg].get();
    T hr = cN * fma(far.x, ts, nr.x) - c2 * reg.x;
    T hi = cN * fma(far.y, ts, nr.y) - c2 * reg.y;
    cplx<T> res = mk<T>((T)-0.5 * (Qs.x - hi), (T)-0.5 * (Qs.y + hr));
    if (inverse) {
      res = cscale(res, Ct[k]);
      if (d.nc) res = cmul(res, from_d2<T>(inv_phase(d, k)));
    }
    out[(int64_t)sig * N + k] = cadd(res, self[gg]);
  }
}

// k_targets_grid for one signal with two adjacent grid points k, k + 1 per
// thread (same leaf: s is even); isrc.coef set: the staged sources' charges
// and self terms are formed while staging (from the caller's samples), so
// no kernel needs to run before this one: every staged source (position and charge
// in one record) is read once for both points, which halves the
// shared-memory instructions of the pair loop.  The
// window is sorted by x, so the sources with k0 = k and those with
// k0 = k + 1 are two consecutive runs: each point takes the self terms of its
// own run and the pair of the other's.  Same arithmetic per pair as
// k_targets_grid.
// MODE 0: the whole evaluation; 1: near field only (to hout), with the
// charges and self terms formed while staging (isrc); 2: far part only (hin).
template <class T, int MODE, int P = 0>
__device__ inline void grid2_tile(
    int tile, TreeDims d, int inverse, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, const cplx<T>* __restrict__ lexp,
    const cplx<T>* __restrict__ lvl2, const T* __restrict__ Ct, cplx<T>* __restrict__ out,
    cplx<T>* __restrict__ hout, const cplx<T>* __restrict__ hin, const InlineSrc<T>& isrc) {
  constexpr int CAP = NearCap<T, 1>::grid;
  constexpr int kPts = 2 * kTgtThreads;
  constexpr int kMaxSlots = kTgtThreads + 3;  // kPts / s + 3 with s >= 2
  extern __shared__ __align__(16) unsigned char smraw[];
  SrcQ<T>* sw = reinterpret_cast<SrcQ<T>*>(smraw);          // [CAP] (x, delta), charge
  cplx<T>* sst = reinterpret_cast<cplx<T>*>(sw + CAP);      // [CAP] self terms
  __shared__ int s_off[kMaxSlots + 1];
  const int N = (int)d.N;
  const int s = d.s;
  const int B = 1 << d.L;
  const int kb = tile * kPts;
  const int k = kb + 2 * threadIdx.x;  // and k + 1
  const bool act = k < N;
  const int bl = kb / s;
  const int bh = ((kb + kPts < N ? kb + kPts : N) - 1) / s;
  const int nslot = bh - bl + 3;
  const int b = act ? k / s : bl;
  NearAcc<T> acc0, acc1;
  cplx<T> self0 = mk<T>(0, 0), self1 = mk<T>(0, 0);
  cplx<T> nr0 = mk<T>(0, 0), nr1 = mk<T>(0, 0);
  // the far part's tables: the CTA's leaf locals and the level-2
  // coefficients, staged in shared memory when only the far part runs here
  const int p = P > 0 ? P : d.p;  // (P > 0: d.p as a compile-time constant)
  const cplx<T>* lxg = lexp + (int64_t)(level_off(d.L) - 4) * p;
  const cplx<T>* lx = lxg;  // locals of leaf b at lx + (b - lxb) p
  int lxb = 0;
  const cplx<T>* l2 = lvl2;
  if constexpr (MODE == 2) {  // near-field sums and self terms formed by an earlier launch
    // (the leaf locals and level-2 coefficients read through L1: every load
    // of this part is independent of the others, no barrier)
    if (!act) return;
    nr0 = hin[2 * (int64_t)k];
    self0 = hin[2 * (int64_t)k + 1];
    if (k + 1 < N) {
      nr1 = hin[2 * (int64_t)k + 2];
      self1 = hin[2 * (int64_t)k + 3];
    }
  } else {
  if (threadIdx.x < 32) {
    int carry = 0;
    for (int c0 = 0; c0 < nslot; c0 += 32) {
      const int js = c0 + threadIdx.x;
      int cnt = 0;
      if (js < nslot) {
        const int bb = (bl - 1 + js + B) & (B - 1);
        cnt = start[bb + 1] - start[bb];
      }
      int v = cnt;
#pragma unroll
      for (int sh = 1; sh < 32; sh <<= 1) {
        int n = __shfl_up_sync(0xffffffffu, v, sh);
        if ((int)threadIdx.x >= sh) v += n;
      }
      if (js < nslot) s_off[js + 1] = carry + v;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (threadIdx.x == 0) s_off[0] = 0;
  }
  __syncthreads();
  const int total = s_off[nslot];
  const int wlo = s_off[b - bl], whi = s_off[b - bl + 3];
  const T kf0 = (T)(k - kb), kf1 = kf0 + (T)1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // both points' pairs with source i: t0 = (k - x) - delta, t1 = t0 + 1
  // from the rounded t0 (for every included pair |t1| >= 1/2 and |t0| <=
  // |t1| + 1, so t1 keeps a relative error of at most two roundings)
  // (MODE 0, the whole evaluation at five CTAs per SM, keeps the exact
  // t1 = (e0 + 1) - delta: its register budget has no room for the other form)
  auto both = [&](int i) {
    const SrcQ<T> v = sw[i];  // one 16-byte load (FP32)
    const T e0 = kf0 - v.rel.x;
    const T t0 = e0 - v.rel.y;
    const T t1 = MODE == 0 ? (e0 + (T)1) - v.rel.y : t0 + (T)1;
    const T r0 = rcp_t(t0), r1 = rcp_t(t1);
    acc0.add_r(v.q, r0);
    acc1.add_r(v.q, r1);
  };
  // the same for a source that may lie in one of the lane's own runs (e0 =
  // 0: no pair with k; e0 = -1: no pair with k + 1; those enter through the
  // self terms), and (both_checked) also outside its window [lo, hi)
  auto both_own = [&](int i) {
    const SrcQ<T> v = sw[i];
    const T e0 = kf0 - v.rel.x;
    const T t0 = e0 - v.rel.y;
    const T t1 = MODE == 0 ? (e0 + (T)1) - v.rel.y : t0 + (T)1;
    T r0 = rcp_t(t0), r1 = rcp_t(t1);
    r0 = e0 != (T)0 ? r0 : (T)0;
    r1 = e0 != (T)-1 ? r1 : (T)0;
    acc0.add_r(v.q, r0);
    acc1.add_r(v.q, r1);
  };
  auto both_checked = [&](int i, int lo, int hi) {
    const SrcQ<T> v = sw[i];
    const T e0 = kf0 - v.rel.x;
    const T t0 = e0 - v.rel.y;
    const T t1 = MODE == 0 ? (e0 + (T)1) - v.rel.y : t0 + (T)1;
    T r0 = rcp_t(t0), r1 = rcp_t(t1);
    const bool in = i >= lo && i < hi;
    r0 = in && e0 != (T)0 ? r0 : (T)0;
    r1 = in && e0 != (T)-1 ? r1 : (T)0;
    acc0.add_r(v.q, r0);
    acc1.add_r(v.q, r1);
  };
  for (int c0 = 0; c0 < total; c0 += CAP) {
    const int c1 = total - c0 < CAP ? total : c0 + CAP;
    __syncthreads();
    for (int js = warp; js < nslot; js += kTgtThreads / 32) {
      const int lo = s_off[js] > c0 ? s_off[js] : c0;
      const int hi = s_off[js + 1] < c1 ? s_off[js + 1] : c1;
      if (lo >= hi) continue;
      const int bu = bl - 1 + js;
      const int bb = (bu + B) & (B - 1);
      const int g0 = start[bb] - s_off[js];
      for (int e = lo + lane; e < hi; e += 32) {
        const int gi = g0 + e;
        const SrcPos<T> ps = pos[gi];
        const int xu = bu * s + (((int)ps.k0 - bb * s) & (N - 1)) - kb;
        SrcQ<T> v;
        v.rel = mk<T>((T)xu, ps.dl);
        if constexpr (MODE == 1) {  // charge and self term formed here (no kernel before)
          // (only a source whose nearest grid point lies in this tile's
          // range can be in a tile point's own run: the halo's sources need
          // no self term)
          v.q = stage_charge_self<T>(isrc, gi, xu >= 0 && xu < kPts, &sst[e - c0]);
        } else {
          v.q = charge[gi];
          sst[e - c0] = st[gi];
        }
        sw[e - c0] = v;
      }
    }
    __syncthreads();
    const int lo = (wlo > c0 ? wlo : c0) - c0, hi = (whi < c1 ? whi : c1) - c0;
    const bool has = act && lo < hi;
    int ha = lo, h2 = lo;
    if (has) {
      // runs x = k - kb and x = k + 1 - kb: [ha, h1), [h1, h2): self terms
      int hb = hi;
      while (ha < hb) {
        const int mid = (ha + hb) >> 1;
        if (sw[mid].rel.x < kf0) ha = mid + 1; else hb = mid;
      }
      h2 = ha;
      for (; h2 < hi && sw[h2].rel.x == kf0; ++h2) self0 = cadd(self0, sst[h2]);
      for (; h2 < hi && sw[h2].rel.x == kf1; ++h2) self1 = cadd(self1, sst[h2]);
    }
    // pairs: the warp walks the union of its lanes' windows in chunks of 16
    // sources; a chunk that is not inside every active lane's window, or
    // that meets a lane's own runs, is taken by the whole warp in the
    // corresponding checked form (warp votes), so no lane waits on another's
    // different bounds
    const int ulo = __reduce_min_sync(0xffffffffu, has ? lo : INT_MAX);
    const int uhi = __reduce_max_sync(0xffffffffu, has ? hi : INT_MIN);
    for (int i = ulo; i < uhi; i += 16) {
      const int n = uhi - i < 16 ? uhi - i : 16;
      const bool edge = act && (i < lo || i + 16 > hi);
      const bool own = act && i < h2 && i + 16 > ha;
      if (n < 16 || __any_sync(0xffffffffu, edge)) {
#pragma unroll
        for (int u = 0; u < 16; ++u)
          if (u < n) both_checked(i + u, lo, hi);
      } else if (__any_sync(0xffffffffu, own)) {
        // inside every active lane's window: only the own runs are left out
#pragma unroll
        for (int u = 0; u < 16; ++u) both_own(i + u);
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) both(i + u);
      }
      acc0.fold();
      acc1.fold();
    }
  }
  if (!act) return;
  nr0 = acc0.get();
  nr1 = acc1.get();
  if constexpr (MODE == 1) {  // near field only: the far part follows the tree passes
    hout[2 * (int64_t)k] = nr0;
    hout[2 * (int64_t)k + 1] = self0;
    if (k + 1 < N) {
      hout[2 * (int64_t)k + 2] = nr1;
      hout[2 * (int64_t)k + 3] = self1;
    }
    return;
  }
  }
  const int Q2 = 2 * d.q;
  const int arc = b >> (d.L - 2);
  const T ts = KConst<T>::inv_s(d);
  const T cN = KConst<T>::n_pi(d), c2 = (T)(2.0 * kInvPi);
  const cplx<T> Qs = l2[4 * Q2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int kk = k + h;
    if (kk >= N) break;
    const int o = kk - b * s;
    const int I = kk - arc * (N >> 2) - (N >> 3);
    const T uh = (T)I * KConst<T>::two_n(d);
    const T u = fma((T)o, ts, (T)-0.5);
    cplx<T> far = mk<T>(0, 0);
    if (d.L >= 3) far = horner_n<T, P>(lx + (int64_t)(b - lxb) * p, p, u);
    const cplx<T> reg = horner<T>(l2 + arc * Q2, Q2, uh);
    const cplx<T> nr = h ? nr1 : nr0;
    const T hr = cN * fma(far.x, ts, nr.x) - c2 * reg.x;
    const T hi = cN * fma(far.y, ts, nr.y) - c2 * reg.y;
    cplx<T> res = mk<T>((T)-0.5 * (Qs.x - hi), (T)-0.5 * (Qs.y + hr));
    if (inverse) {
      res = cscale(res, Ct[kk]);
      if (d.nc) res = cmul(res, from_d2<T>(inv_phase(d, kk)));
    }
    out[kk] = cadd(res, h ? self1 : self0);
  }
}

template <class T, int MODE, int P = 0>
__global__ void __launch_bounds__(kTgtThreads, (sizeof(T) == 4 && MODE == 0) ? 5 : 4) k_targets_grid2(
    TreeDims d, int inverse, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, const cplx<T>* __restrict__ lexp,
    const cplx<T>* __restrict__ lvl2, const T* __restrict__ Ct, cplx<T>* __restrict__ out,
    cplx<T>* __restrict__ hout, const cplx<T>* __restrict__ hin, InlineSrc<T> isrc) {
  pdl_wait();
  pdl_trigger();
  const int ntiles = (int)((d.N + 2 * kTgtThreads - 1) / (2 * kTgtThreads));
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    if (tile != (int)blockIdx.x) __syncthreads();  // the previous tile's shared data are read
    grid2_tile<T, MODE, P>(tile, d, inverse, start, pos, charge, st, lexp, lvl2, Ct, out, hout, hin,
                        isrc);
  }
}

// Adjoint / inverse near field for one signal when each grid point meets
// many sources (M >> N, or clustered sources): one warp per G consecutive
// grid points of one leaf b (G divides s), so all G share the window of
// leaves b - 1 .. b + 1.  The lanes stride over the window's sources (loads
// of consecutive sources are coalesced and shared by the G targets), each
// lane keeps G compensated partial sums; a reduce-scatter across the lanes
// (log2 G halving exchanges, then full exchanges: 5 shuffle rounds) leaves
// target g's sum in the lanes g * 32 / G .. (g + 1) * 32 / G - 1, the first of
// which finishes it: the sources whose nearest grid point is the target (a
// run of the sorted leaf, found by binary search) add their self terms, the
// far field, the regular part (Eq. p20) and C_k complete it as in
// k_targets_grid2.  Grid size N / (8 G) CTAs of 8 warps.  With hout set
// only the near-field sums and self terms are formed (two per grid point,
// the layout k_targets_grid2 reads with hin).
template <class T>
__device__ inline T int_small_to_t(int v) { return int_to_t(v, T()); }

// One warp's G grid points kb .. kb + G - 1 (AD: the near-field sums of a
// deeper class of the adaptive tree, added to the earlier classes').
template <class T, int G, int AD>
__device__ inline void gridw_group(
    int kb, const TreeDims& d, int inverse, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, const cplx<T>* __restrict__ lexp,
    const cplx<T>* __restrict__ lvl2, const T* __restrict__ Ct, cplx<T>* __restrict__ out,
    cplx<T>* __restrict__ hout) {
  constexpr int LOGG = G == 8 ? 3 : (G == 4 ? 2 : 1);
  const int N = (int)d.N;
  const int s = d.s;
  const int B = 1 << d.L;
  const int lane = threadIdx.x & 31;
  const int b = kb / s;
  NearAcc<T> acc[G];
  for (int nb = -1; nb <= 1; ++nb) {
    const int bu = b + nb;
    const int bb = bu & (B - 1);
    const int i0 = start[bb], i1 = start[bb + 1];
    const int xbase = bu * s - kb;  // source position relative to kb: xbase + (k0 - bb s) mod N
    int cnt = 0;
    for (int i = i0 + lane; i < i1; i += 32) {
      const SrcPos<T> ps = pos[i];
      const cplx<T> q = charge[i];
      const int xi = xbase + (((int)ps.k0 - bb * s) & (N - 1));
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const T e = int_small_to_t<T>(g - xi);  // exact small integer
        T r = rcp_t(e - ps.dl);
        r = e != (T)0 ? r : (T)0;  // the nearest grid point: self term below
        acc[g].add_r(q, r);
      }
      if (++cnt == 16) {
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g].fold();
        cnt = 0;
      }
    }
  }
  // reduce-scatter over the lanes
  cplx<T> v[G];
#pragma unroll
  for (int g = 0; g < G; ++g) v[g] = acc[g].get();
#pragma unroll
  for (int st_ = 0; st_ < LOGG; ++st_) {
    const int mask = 16 >> st_;
    const int half = G >> (st_ + 1);
    const bool upper = (lane & mask) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const cplx<T> send = upper ? v[i] : v[i + half];
      const cplx<T> keep = upper ? v[i + half] : v[i];
      cplx<T> got;
      got.x = __shfl_xor_sync(0xffffffffu, send.x, mask);
      got.y = __shfl_xor_sync(0xffffffffu, send.y, mask);
      v[i] = cadd(keep, got);
    }
  }
#pragma unroll
  for (int mask = 16 >> LOGG; mask > 0; mask >>= 1) {
    v[0].x += __shfl_xor_sync(0xffffffffu, v[0].x, mask);
    v[0].y += __shfl_xor_sync(0xffffffffu, v[0].y, mask);
  }
  if ((lane & ((32 >> LOGG) - 1)) != 0) return;
  const int g = lane >> (5 - LOGG);
  const int k = kb + g;
  // self terms: the run of leaf b with k0 = k, and for the leaf's first grid
  // point the sources at the end of leaf b - 1 that round up to it
  cplx<T> self = mk<T>(0, 0);
  {
    const int want = k - b * s;  // (k0 - b s) mod N of the run, in [0, s)
    int lo = start[b], hi = start[b + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((((int)pos[mid].k0 - b * s) & (N - 1)) < want) lo = mid + 1; else hi = mid;
    }
    for (int i = lo; i < start[b + 1] && (((int)pos[i].k0 - b * s) & (N - 1)) == want; ++i)
      self = cadd(self, st[i]);
    if (want == 0) {
      const int bp = (b - 1) & (B - 1);
      for (int i = start[bp + 1] - 1; i >= start[bp] && (((int)pos[i].k0 - bp * s) & (N - 1)) == s; --i)
        self = cadd(self, st[i]);
    }
  }
  if (hout) {  // near field only (the two-point kernel's far part follows)
    if constexpr (AD) {
      v[0] = cadd(v[0], hout[2 * (int64_t)k]);
      self = cadd(self, hout[2 * (int64_t)k + 1]);
    }
    hout[2 * (int64_t)k] = v[0];
    hout[2 * (int64_t)k + 1] = self;
    return;
  }
  const int Q2 = 2 * d.q;
  const int arc = b >> (d.L - 2);
  const T ts = KConst<T>::inv_s(d);
  const T cN = KConst<T>::n_pi(d), c2 = (T)(2.0 * kInvPi);
  const cplx<T> Qs = lvl2[4 * Q2];
  const int o = k - b * s;
  const int I = k - arc * (N >> 2) - (N >> 3);
  const T uh = (T)I * KConst<T>::two_n(d);
  const T u = fma((T)o, ts, (T)-0.5);
  cplx<T> far = mk<T>(0, 0);
  if (d.L >= 3) far = horner<T>(lexp + ((int64_t)(level_off(d.L) - 4) + b) * d.p, d.p, u);
  const cplx<T> reg = horner<T>(lvl2 + arc * Q2, Q2, uh);
  const T hr = cN * fma(far.x, ts, v[0].x) - c2 * reg.x;
  const T hi = cN * fma(far.y, ts, v[0].y) - c2 * reg.y;
  cplx<T> res = mk<T>((T)-0.5 * (Qs.x - hi), (T)-0.5 * (Qs.y + hr));
  if (inverse) {
    res = cscale(res, Ct[k]);
    if (d.nc) res = cmul(res, from_d2<T>(inv_phase(d, k)));
  }
  out[k] = cadd(res, self);
}

template <class T, int G>
__global__ void __launch_bounds__(kTgtThreads) k_targets_gridw(
    TreeDims d, int inverse, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, const cplx<T>* __restrict__ lexp,
    const cplx<T>* __restrict__ lvl2, const T* __restrict__ Ct, cplx<T>* __restrict__ out,
    cplx<T>* __restrict__ hout) {
  pdl_wait();
  pdl_trigger();
  const int kb = (int)((blockIdx.x * (unsigned)kTgtThreads + threadIdx.x) >> 5) * G;
  if (kb >= (int)d.N) return;  // the same for the whole warp
  gridw_group<T, G, 0>(kb, d, inverse, start, pos, charge, st, lexp, lvl2, Ct, out, hout);
}

// The near-field sums of one deeper class of the adaptive tree (its sources
// alone, the tree of depth d.L; charges and self terms in class order),
// added to the earlier classes', on the grid tiles of 2 kTgtThreads points of
// the list `tiles`: kGridwTileCtas CTAs of 8 warps x 8 grid points per tile.
constexpr int kGridwTileCtas = 2 * kTgtThreads / (kTgtThreads / 32 * 8);
template <class T>
__global__ void __launch_bounds__(kTgtThreads) k_targets_gridw_ad(
    TreeDims d, int inverse, const int32_t* __restrict__ tiles, const int32_t* __restrict__ start,
    const SrcPos<T>* __restrict__ pos, const cplx<T>* __restrict__ charge,
    const cplx<T>* __restrict__ st, cplx<T>* __restrict__ hout) {
  pdl_wait();
  pdl_trigger();
  const int tile = tiles[blockIdx.x / kGridwTileCtas];
  const int kb = tile * 2 * kTgtThreads +
                 (int)(((blockIdx.x % kGridwTileCtas) * (unsigned)kTgtThreads + threadIdx.x) >> 5) * 8;
  if (kb >= (int)d.N) return;  // the same for the whole warp
  gridw_group<T, 8, 1>(kb, d, inverse, start, pos, charge, st, nullptr, nullptr, nullptr, nullptr,
                       hout);
}

}  // namespace nufft

using namespace nufft;

// ---------------------------------------------------------------- host drivers

static inline unsigned nblk(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }

// persistent grids: at most kPersistCtas CTAs, each looping over its share
// tree passes: levels <= kTopLevel (at most 32 boxes) run in one CTA, finer
// levels in subtrees of at most kSubDepth levels (64 boxes) per CTA
static constexpr int kTopLevel = 5;
static constexpr int kSubDepth = 6;
static constexpr size_t kSmemBudget = 220 * 1024;

template <class T>
static size_t up_sub_smem(int pm, int depth) {
  return (size_t)2 * pm * pm * sizeof(T) + (size_t)3 * ((size_t)pm << depth) / 2 * sizeof(cplx<T>);
}
// Stages of k_up_fused for a plan (depth per stage as large as shared
// memory allows, at most kSubDepth); returns the counters it needs per signal.
template <class T>
static int up_fused_stages(int pm, int L, UpStages* sg) {
  int dep = kSubDepth;
  while (dep > 1 && up_sub_smem<T>(pm, dep) > kSmemBudget) --dep;
  sg->n = 0;
  sg->dmax = 0;
  sg->lev[0] = L;
  int lev = L;
  while (lev > 2 && sg->n < 15) {
    const int lt = lev - dep > 2 ? lev - dep : 2;
    if (lev - lt > sg->dmax) sg->dmax = lev - lt;
    sg->lev[++sg->n] = lt;
    lev = lt;
  }
  if (lev > 2) return -1;
  // counters of the boxes of level lev[2] and coarser (indexed like multipoles)
  return sg->n >= 2 ? (int)(int64_t(2) << sg->lev[2]) : 0;
}

int fmm_up_counters(int prec, int pm, int L) {
  UpStages sg;
  return prec == NUFFT_FP64 ? up_fused_stages<double>(pm, L, &sg)
                            : up_fused_stages<float>(pm, L, &sg);
}

template <class T>
static size_t down_sub_smem(int p, int depth) {
  size_t nbx = (size_t)1 << depth;
  return (size_t)6 * p * p * sizeof(T) + (nbx + 6 + 2 * nbx) * p * sizeof(cplx<T>);
}

template <class T>
static size_t down_fused_smem(int p, int depth, int lt) {
  const size_t nlam = (((size_t)2 << depth) - 2) * p;
  return (size_t)6 * p * p * sizeof(T) +
         (2 * nlam + (size_t)6 * depth * p + (size_t)(lt - 2) * 4 * p) * sizeof(cplx<T>);
}

int m2l_tc_level(const TreeDims& d, int l, int nsig, const float* bops, const float2* mexp,
                 float2* lexp, int* status, cudaStream_t st);

template <class T>
static cudaError_t down_fused_attrs(int big) {
  cudaError_t e = cudaSuccess;
  if constexpr (std::is_same<T, float>::value) {
#define NUFFT_DOWN_ATTR(PV)                                                                   \
  if (e == cudaSuccess)                                                                      \
    e = cudaFuncSetAttribute(k_down_fused<T, PV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             big);
    NUFFT_TREE_P_LIST(NUFFT_DOWN_ATTR)
#undef NUFFT_DOWN_ATTR
  }
  return e;
}

// the one-launch upward pass (P2M from SRC 1 or 2), at the compile-time
// instance for pm where there is one
template <class T, int SRC, class VI, class... A>
static void launch_up_fused(int pm, dim3 grid, size_t smem, cudaStream_t st, A... args) {
  if constexpr (std::is_same<T, float>::value) {
    switch (pm) {
#define NUFFT_UP_CASE(PV)                                                            \
  case PV:                                                                          \
    launch_pdl(k_up_fused<T, SRC, VI, PV>, grid, kUpThreads, smem, st, args...);    \
    return;
      NUFFT_TREE_P_LIST(NUFFT_UP_CASE)
#undef NUFFT_UP_CASE
      default: break;
    }
  }
  launch_pdl(k_up_fused<T, SRC, VI>, grid, kUpThreads, smem, st, args...);
}

template <class T, int SRC, class VI>
static cudaError_t up_fused_attrs(int big) {
  cudaError_t e = cudaSuccess;
  if constexpr (std::is_same<T, float>::value) {
#define NUFFT_UP_ATTR(PV)                                                                  \
  if (e == cudaSuccess)                                                                   \
    e = cudaFuncSetAttribute(k_up_fused<T, SRC, VI, PV>,                                  \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    NUFFT_TREE_P_LIST(NUFFT_UP_ATTR)
#undef NUFFT_UP_ATTR
  }
  return e;
}

// the one-launch downward pass, at the compile-time instance for p where
// there is one
template <class T, class... A>
static void launch_down_fused(int p, dim3 grid, size_t smem, cudaStream_t st, A... args) {
  if constexpr (std::is_same<T, float>::value) {
    switch (p) {
#define NUFFT_DOWN_CASE(PV)                                                          \
  case PV:                                                                          \
    launch_pdl(k_down_fused<T, PV>, grid, kDownThreads, smem, st, args...);         \
    return;
      NUFFT_TREE_P_LIST(NUFFT_DOWN_CASE)
#undef NUFFT_DOWN_CASE
      default: break;
    }
  }
  launch_pdl(k_down_fused<T>, grid, kDownThreads, smem, st, args...);
}

template <class T>
int fmm_configure() {
  int big = 220 * 1024;
  if (cudaFuncSetAttribute(k_up_sub<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_up_top<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 0, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 1, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 0, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 1, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_up_fused<T, 2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_p2m_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_down_top<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_down_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      down_fused_attrs<T>(big) != cudaSuccess ||
      up_fused_attrs<T, 1, float2>(big) != cudaSuccess ||
      up_fused_attrs<T, 2, float2>(big) != cudaSuccess ||
      up_fused_attrs<T, 2, double2>(big) != cudaSuccess ||
      cudaFuncSetAttribute(k_down_sub<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_down_deep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_deep_p2m<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_deep_m2l_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           big) != cudaSuccess ||
      cudaFuncSetAttribute(k_level2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           4 * 66 * 66 * (int)sizeof(double)) != cudaSuccess ||
      cudaFuncSetAttribute(k_p2m_chunks<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)p2m_smem<T>(32)) != cudaSuccess ||
      cudaFuncSetAttribute(k_p2m_nonuniform<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)p2m_smem<T>(32)) != cudaSuccess)
    return NUFFT_ECUDA;
  return NUFFT_OK;
}

TreeDims dims_of(const nufft_plan_s* pl) {
  TreeDims d{pl->N, pl->L, pl->s, pl->p, pl->q, pl->pm};
  d.mstride = ((int64_t(2) << pl->L) - 4) * pl->pm;
  int64_t nl = (int64_t(2) << pl->L) - 8;
  d.lstride = (nl > 0 ? nl : 1) * pl->p;
  d.M_ = pl->M;
  d.two_n = 2.0 / (double)pl->N;
  d.inv_s = 1.0 / (double)pl->s;
  d.n_pi = (double)pl->N * kInvPi;
  d.two_n_f = (float)d.two_n;
  d.inv_s_f = (float)d.inv_s;
  d.n_pi_f = (float)d.n_pi;
  d.nc = pl->inv_nc;
  return d;
}

// the plan's per-point data in the arithmetic type T
template <class T> struct PlanT;
template <> struct PlanT<double> {
  static const double* delta(nufft_plan_s* pl) { return pl->delta; }
  static const double2* D(nufft_plan_s* pl) { return pl->Dt; }
  static const double2* F(nufft_plan_s* pl) { return pl->F; }
  static const double2* E(nufft_plan_s* pl) { return pl->E; }
  static const double2* lvl2(nufft_plan_s* pl) { return pl->lvl2; }
  static const double* Ct(nufft_plan_s* pl) { return pl->Ct; }
  static const double2* S(nufft_plan_s* pl) { return pl->Sinv; }
};
template <> struct PlanT<float> {
  static const float* delta(nufft_plan_s* pl) { return pl->delta_f; }
  static const float2* D(nufft_plan_s* pl) { return pl->Dtf; }
  static const float2* F(nufft_plan_s* pl) { return pl->Ff; }
  static const float2* E(nufft_plan_s* pl) { return pl->Ef; }
  static const float2* lvl2(nufft_plan_s* pl) { return pl->lvl2f; }
  static const float* Ct(nufft_plan_s* pl) { return pl->Ctf; }
  static const float2* S(nufft_plan_s* pl) { return pl->Sinvf; }
};

// Upward pass (P2M, M2M) for all signals of the plan at once (grid y =
// signal), then the level-2 coefficients on a side branch.  Sources:
// uniform (the grid samples `charge`, [batch][N]) or the sorted non-uniform
// points (`charge`, [batch][M]); with `gin` set (non-uniform sources only),
// the charges are formed from the caller's samples as coef_i g_perm(i)
// (conj(coef_i) when conj) and stored to `charge`: inside the upward kernel
// where it forms the leaves' multipoles itself, else by k_charges first;
// *charges_done then reports that the charges are in place.
template <class T, class VI>
int fmm_upward(nufft_plan_s* pl, const FmmOps& ops, bool uniform_sources, const cplx<T>* charge,
               const cplx<T>* coef, int conj, const VI* gin, bool* charges_done, double2* lvl2,
               float2* lvl2f) {
  cudaStream_t st = pl->stream;
  const TreeDims d = dims_of(pl);
  const unsigned nsig = (unsigned)pl->batch;
  int64_t B = pl->B;
  cplx<T>* mexp = (cplx<T>*)pl->mexp;
  cplx<T>* mleaf = mexp + level_off(pl->L) * pl->pm;
  const int pm = pl->pm, L = pl->L;
  // the one-launch upward pass, with P2M inside where shared memory allows
  UpStages sg;
  // (non-uniform sources: a shallower first stage, one leaf per warp, so
  // the per-leaf P2M loops run on as many warps as a separate P2M would)
  const int ncnt = L > 2 && pl->upcnt && fused_up_enabled() && !ops.leaf_shift
                       ? up_fused_stages<T>(pm, L, &sg) : -1;
  const bool fused = ncnt >= 0 && ncnt <= pl->upcnt_n;
  int src = 0;
  // (clustered sources: the chunked P2M before the pass instead of one warp
  // per leaf inside it)
  const bool chunked = !uniform_sources && pl->p2m_part != nullptr && !ops.leaf_shift;
  if (fused) {
    if (uniform_sources && up_fused_smem<T>(pm, sg, 1, pl->s) <= kSmemBudget) src = 1;
    if (!uniform_sources && !chunked && up_fused_smem<T>(pm, sg, 2, pl->s) <= kSmemBudget)
      src = 2;
  }
  if (gin && src != 2) {  // charges first, by their own kernel
    prof_begin(pl, NUFFT_STAGE_P2M);
    launch_pdl(k_charges<T, VI>, dim3(nblk(pl->M, 256), nsig), 256, 0, st, pl->M, pl->perm, coef,
               conj, gin, (cplx<T>*)charge);
    prof_end(pl, 1);
  }
  if (charges_done) *charges_done = gin != nullptr;
  if (src) {
    prof_begin(pl, NUFFT_STAGE_M2M);
    UpSrc<T, VI> us;
    us.q = charge;
    us.rp = (const T*)pl->op_p2m;
    us.start = pl->leaf_start;
    us.k0 = pl->k0;
    us.delta_t = PlanT<T>::delta(pl);
    if (src == 2 && gin) {
      us.perm = pl->perm;
      us.coef = coef;
      us.conj = conj;
      us.gin = gin;
      us.charge = (cplx<T>*)charge;
    }
    const size_t sm = up_fused_smem<T>(pm, sg, src, pl->s);
    const dim3 grid(1u << sg.lev[1], nsig);
    if (src == 1) {  // (the input type does not enter SRC 1)
      UpSrc<T, float2> u1;
      u1.q = us.q;
      u1.rp = us.rp;
      u1.start = us.start;
      u1.k0 = us.k0;
      u1.delta_t = us.delta_t;
      launch_up_fused<T, 1, float2>(pm, grid, sm, st, d, sg, (const T*)pl->op_m2m, mexp,
                                    pl->upcnt, pl->upcnt_n, u1);
    } else {
      launch_up_fused<T, 2, VI>(pm, grid, sm, st, d, sg, (const T*)pl->op_m2m, mexp, pl->upcnt,
                                pl->upcnt_n, us);
    }
    prof_end(pl, 1);
  } else {
    prof_begin(pl, NUFFT_STAGE_P2M);
    if (uniform_sources && pl->N >= kP2mChunk && pl->s <= kP2mChunk &&
        p2m_grid_smem<T>(pl->s, pl->pm) <= kSmemBudget) {
      launch_pdl(k_p2m_grid<T>, dim3((unsigned)(pl->N / kP2mChunk), nsig), 256,
                 p2m_grid_smem<T>(pl->s, pl->pm), st, d, charge, (const T*)pl->op_p2m, mleaf);
    } else if (uniform_sources) {
      launch_pdl(k_p2m_uniform<T>, dim3(nblk(B * pl->pm, 256), nsig), 256, 0, st, d, charge,
                 (const T*)pl->op_p2m, mleaf);
    } else if (chunked) {
      constexpr int WPB = P2mWarps<T>::value;
      const int nc = (int)pl->p2m_nchunk;
      cplx<T>* part = (cplx<T>*)pl->p2m_part;
      launch_pdl(k_p2m_chunks<T>, dim3(nblk(nc, WPB), nsig), 32 * WPB, p2m_smem<T>(pl->pm), st,
                 d, nc, (const int32_t*)pl->p2m_chunk, (const int32_t*)pl->k0,
                 PlanT<T>::delta(pl), charge, part);
      launch_pdl(k_p2m_chunk_sum<T>, dim3(nblk(B * pl->pm, 256), nsig), 256, 0, st, d, nc,
                 (const int32_t*)pl->p2m_cfirst, (const cplx<T>*)part, mleaf);
    } else {
      constexpr int WPB = P2mWarps<T>::value;
      launch_pdl(k_p2m_nonuniform<T>, dim3(nblk(B, WPB), nsig), 32 * WPB, p2m_smem<T>(pl->pm),
                 st, d, pl->leaf_start, pl->k0, PlanT<T>::delta(pl), charge, mleaf);
    }
    if (ops.leaf_shift)
      launch_pdl(k_leaf_shift<T>, nblk(B * pl->pm, 256), 256, 0, st, B, pl->pm, ops.leaf_shift,
                 mleaf);
    prof_end(pl, ops.leaf_shift || chunked ? 2 : 1);
    // upward: one launch, or subtrees of up to kSubDepth levels down to level
    // kTopLevel, then one CTA
    prof_begin(pl, NUFFT_STAGE_M2M);
    int nl = 0;
    int lev = L;
    if (fused) {
      launch_pdl(k_up_fused<T, 0, VI>, dim3(1u << sg.lev[1], nsig), kUpThreads,
                 up_fused_smem<T>(pm, sg, 0, pl->s), st, d, sg, (const T*)pl->op_m2m, mexp,
                 pl->upcnt, pl->upcnt_n, UpSrc<T, VI>());
      ++nl;
      lev = 2;
    }
    while (lev > kTopLevel) {
      int dep = kSubDepth;
      while (dep > 1 && up_sub_smem<T>(pm, dep) > kSmemBudget) --dep;
      int lt = lev - dep > kTopLevel ? lev - dep : kTopLevel;
      launch_pdl(k_up_sub<T>, dim3(1u << lt, nsig), 512, up_sub_smem<T>(pm, lev - lt), st, d,
                 lev, lt, (const T*)pl->op_m2m, mexp);
      ++nl;
      lev = lt;
    }
    if (lev > 2) {
      size_t sm = (size_t)2 * pm * pm * sizeof(T) +
                  (size_t)3 * ((size_t)pm << lev) / 2 * sizeof(cplx<T>);
      launch_pdl(k_up_top<T>, dim3(1, nsig), 512, sm, st, d, lev, (const T*)pl->op_m2m, mexp);
      ++nl;
    }
    prof_end(pl, nl);
  }
  // level-2 coefficients on the side branch (only the targets need them)
  prof_begin(pl, NUFFT_STAGE_LEVEL2);
  {
    cudaStream_t s2 = side_begin(pl, 0);
    launch_pdl(k_level2<T>, nsig, 256, (size_t)4 * ops.nq * ops.nq * sizeof(double), s2, d,
               ops.nq, ops.reg, ops.c1, ops.c2, mexp, lvl2, lvl2f);
    side_end(pl, 0, s2);
  }
  prof_end(pl, 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// Downward pass (M2L, L2L) to the leaves' local expansions, then joins the
// level-2 side branch.
template <class T>
int fmm_downward(nufft_plan_s* pl, const FmmOps& ops) {
  cudaStream_t st = pl->stream;
  const TreeDims d = dims_of(pl);
  const unsigned nsig = (unsigned)pl->batch;
  cplx<T>* mexp = (cplx<T>*)pl->mexp;
  cplx<T>* lexp = (cplx<T>*)pl->lexp;
  const int p = pl->p, L = pl->L;
  int nl = 0;
  // without tensor-core levels the whole pass in one launch; with them,
  // levels 3..kTopLevel in one CTA, then subtrees (cut from the finest level
  // up so the costly fine levels get the most CTAs) down to the first
  // tensor-core level
  prof_begin(pl, NUFFT_STAGE_M2L);
  int log2N = 0;
  while ((int64_t(1) << log2N) < pl->N) ++log2N;
  if (L >= 3) {
    int top = L < kTopLevel ? L : kTopLevel;
    auto top_smem = [&](int t) {
      return (size_t)6 * p * p * sizeof(T) + (size_t)3 * ((size_t)p << t) * sizeof(cplx<T>);
    };
    while (top > 3 && top_smem(top) > kSmemBudget) --top;
    size_t smt = top_smem(top);
    // levels lc..L as one tensor-core GEMM each (FP32 data, cot kernel only)
    int lc = L + 1;
    if constexpr (std::is_same<T, float>::value)
      if (!ops.log_kernel && pl->op_tc && pl->tc_level >= 4 && pl->tc_level <= L)
        lc = pl->tc_level > top + 1 ? pl->tc_level : top + 1;
    // no tensor-core levels: the whole downward pass in one launch, where its
    // shared memory fits (else, as with tensor-core levels, the banded form)
    int fdep = kSubDepth;
    while (fdep > 1 && down_fused_smem<T>(p, fdep, L) > kSmemBudget) --fdep;
    const int flt = L - fdep > 3 ? L - fdep : 3;  // subtree roots
    if (lc > L && down_fused_smem<T>(p, L - flt, flt) <= kSmemBudget) {
      if (L > 3) {
        launch_down_fused<T>(p, dim3(1u << flt, nsig), down_fused_smem<T>(p, L - flt, flt), st,
                             d, flt, L, (const T*)ops.m2l, (const T*)ops.l2l,
                             (const cplx<T>*)mexp, lexp, ops.log_kernel, log2N);
      } else {  // L = 3: level 3 alone
        launch_pdl(k_down_top<T>, dim3(1, nsig), 512, smt, st, d, 3, (const T*)ops.m2l,
                   (const T*)ops.l2l, mexp, lexp, ops.log_kernel, log2N);
      }
      ++nl;
    } else {
      launch_pdl(k_down_top<T>, dim3(1, nsig), 512, smt, st, d, top, (const T*)ops.m2l,
                 (const T*)ops.l2l, mexp, lexp, ops.log_kernel, log2N);
      ++nl;
      int dep = kSubDepth;
      while (dep > 1 && down_sub_smem<T>(p, dep) > kSmemBudget) --dep;
      int cuts[32], nc = 0;
      for (int lb = lc - 1; lb > top; lb -= dep) cuts[nc++] = lb;
      int lt = top;
      for (int c = nc - 1; c >= 0; --c) {
        int lb = cuts[c];
        launch_pdl(k_down_sub<T>, dim3(1u << lt, nsig), 512, down_sub_smem<T>(p, lb - lt), st, d,
                   lt, lb, (const T*)ops.m2l, (const T*)ops.l2l, mexp, lexp, ops.log_kernel,
                   log2N);
        ++nl;
        lt = lb;
      }
    }
    if constexpr (std::is_same<T, float>::value) {
      for (int l = lc; l <= L; ++l) {
        int rc = m2l_tc_level(d, l, (int)nsig, pl->op_tc, (const float2*)mexp, (float2*)lexp,
                              pl->status, st);
        if (rc) return rc;
        ++nl;
      }
    }
  }
  prof_end(pl, nl);
  side_join(pl, 0);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template <class T>
int fmm_upward_downward(nufft_plan_s* pl, const FmmOps& ops, bool uniform_sources,
                        const cplx<T>* charge, double2* lvl2, float2* lvl2f) {
  int rc = fmm_upward<T, float2>(pl, ops, uniform_sources, charge, nullptr, 0,
                                 (const float2*)nullptr, nullptr, lvl2, lvl2f);
  return rc ? rc : fmm_downward<T>(pl, ops);
}

static FmmOps cot_ops(nufft_plan_s* pl) {
  FmmOps o;
  o.m2l = pl->op_m2l;
  o.l2l = pl->op_l2l;
  o.reg = pl->op_reg;
  o.nq = 2 * pl->q;
  return o;
}

// CTAs of a near-field pass beside the tree passes: one per target tile (0),
// or r per SM looping over the tiles (NUFFT_NEAR_FWD_CTAS / NUFFT_NEAR_GRID_CTAS
// = r), which keeps room for the tree kernels' CTAs on every SM; measured at
// 2^20: every r tried (2..8) lost more near-field throughput than the tree
// passes gained, so one CTA per tile is the default.
static int near_ctas_per_sm(bool grid) {
  static const int f = [] { const char* e = std::getenv("NUFFT_NEAR_FWD_CTAS"); return e ? std::atoi(e) : 0; }();
  static const int g = [] { const char* e = std::getenv("NUFFT_NEAR_GRID_CTAS"); return e ? std::atoi(e) : 0; }();
  return grid ? g : f;
}
static unsigned near_grid(int64_t tiles, bool grid) {
  static const int nsm = [] {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    return n;
  }();
  const int r = near_ctas_per_sm(grid);
  if (r <= 0 || nsm <= 0) return (unsigned)tiles;
  const int64_t cap = (int64_t)r * nsm;
  return (unsigned)(tiles < cap ? tiles : cap);
}

// k_targets_grid2's far part (MODE 2) at the compile-time instance for p
template <class T, class... A>
static void launch_far_grid2(int p, unsigned nb, size_t sm, cudaStream_t st, A... args) {
  if constexpr (std::is_same<T, float>::value) {
    switch (p) {
#define NUFFT_FARG_CASE(PV)                                                   \
  case PV:                                                                   \
    launch_pdl(k_targets_grid2<T, 2, PV>, nb, kTgtThreads, sm, st, args...); \
    return;
      NUFFT_TREE_P_LIST(NUFFT_FARG_CASE)
#undef NUFFT_FARG_CASE
      default: break;
    }
  }
  launch_pdl(k_targets_grid2<T, 2>, nb, kTgtThreads, sm, st, args...);
}

// k_far_fwd at the compile-time instance for p where there is one
template <class T, class VO, class... A>
static void launch_far_fwd(int p, unsigned nb, size_t sm, cudaStream_t st, A... args) {
  if constexpr (std::is_same<T, float>::value) {
    switch (p) {
#define NUFFT_FAR_CASE(PV)                                                  \
  case PV:                                                                 \
    launch_pdl(k_far_fwd<T, VO, PV>, nb, kTgtThreads, sm, st, args...);    \
    return;
      NUFFT_TREE_P_LIST(NUFFT_FAR_CASE)
#undef NUFFT_FAR_CASE
      default: break;
    }
  }
  launch_pdl(k_far_fwd<T, VO>, nb, kTgtThreads, sm, st, args...);
}

template <class T, class VO, int G>
static void launch_targets_fwd(nufft_plan_s* pl, const TreeDims& d, const cplx<T>* f,
                               const cplx<T>* hnear, void* g, cplx<T>* hout = nullptr,
                               cudaStream_t st = nullptr) {
  const int64_t tiles = nblk(pl->M, kTgtThreads);
  dim3 grid(hout ? near_grid(tiles, false) : (unsigned)tiles, (unsigned)(pl->batch / G));
  launch_pdl(k_targets_fwd<T, VO, G>, grid, kTgtThreads, hnear ? 0 : NearCap<T, G>::fwd_bytes,
             st ? st : pl->stream, d, (int)pl->M, (const SrcPos<T>*)pl->srcpos,
             pl->perm, PlanT<T>::F(pl), PlanT<T>::E(pl), f, (const cplx<T>*)pl->lexp,
             PlanT<T>::lvl2(pl), hnear, (VO*)g, hout);
}

// Split target evaluation: the near-field sums on side branch 2 while the
// tree passes run (one signal, no tensor-core near field; NUFFT_NO_SPLIT_NEAR
// keeps the single fused launch after the tree passes).
static bool split_near(const nufft_plan_s* pl) {
  static const bool off = std::getenv("NUFFT_NO_SPLIT_NEAR") != nullptr;
  return !off && pl->batch == 1 && pl->tc_near <= 0 && pl->hnear && pl->side_ok;
}

int near_tc_forward(const TreeDims& d, int M, int batch, const int32_t* k0s, const double* dels,
                    const float* dels_f, const float2* fgrid, float2* hnear, int* status,
                    cudaStream_t st);

// the per-point data of the adaptive classes in the arithmetic type T
template <class T> struct AdT;
template <> struct AdT<double> {
  static const double2* F(nufft_plan_s* pl) { return pl->ad_F; }
  static const double2* E(nufft_plan_s* pl) { return pl->ad_E; }
};
template <> struct AdT<float> {
  static const float2* F(nufft_plan_s* pl) { return pl->ad_Ff; }
  static const float2* E(nufft_plan_s* pl) { return pl->ad_Ef; }
};

// The tree of depth class c: leaves at level L + c, s >> c grid points each.
static TreeDims class_dims(const nufft_plan_s* pl, int c) {
  TreeDims d = dims_of(pl);
  d.L += c;
  d.s >>= c;
  d.inv_s = 1.0 / (double)d.s;
  d.inv_s_f = (float)d.inv_s;
  d.lstride = ((int64_t(2) << d.L) - 8) * d.p;
  return d;
}

// Forward with the adaptive tree (one signal): the targets of depth class c
// (stored class after class) are the uniform tree's targets at depth L + c.
// Their near-field sums (grid samples only) run on side branch 2 beside the
// tree passes, class after class; the main chain runs the uniform upward and
// downward passes, then the deeper levels (k_down_deep: one launch, one CTA
// per refined leaf); the far parts of the classes follow the join.
template <class T>
static int fmm_forward_adaptive(nufft_plan_s* pl, void* g) {
  const cplx<T>* f = (const cplx<T>*)pl->grid;
  const bool c64 = (pl->flags & NUFFT_IO_C64) != 0;
  const int D = pl->ad_D, p = pl->p;
  const SrcPos<T>* pos = (const SrcPos<T>*)pl->ad_pos;
  const cplx<T>* F = AdT<T>::F(pl);
  const cplx<T>* E = AdT<T>::E(pl);
  cplx<T>* hn = (cplx<T>*)pl->hnear;
  const cplx<T>* l2 = PlanT<T>::lvl2(pl);
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  cudaStream_t s2 = side_begin(pl, 2);
  int nn = 0;
  {
    LowPriority lp;
    for (int c = 0; c <= D; ++c) {
      const int64_t o = pl->ad_off[c], mc = pl->ad_off[c + 1] - o;
      if (mc == 0) continue;
      const TreeDims dc = class_dims(pl, c);
      const unsigned nb = near_grid(nblk(mc, kTgtThreads), false);
      if (c64)
        launch_pdl(k_targets_fwd<T, float2, 1>, dim3(nb, 1), kTgtThreads,
                   NearCap<T, 1>::fwd_bytes, s2, dc, (int)mc, pos + o, pl->ad_perm + o, F + o,
                   E + o, f, (const cplx<T>*)nullptr, l2, (const cplx<T>*)nullptr,
                   (float2*)g, hn + o);
      else
        launch_pdl(k_targets_fwd<T, double2, 1>, dim3(nb, 1), kTgtThreads,
                   NearCap<T, 1>::fwd_bytes, s2, dc, (int)mc, pos + o, pl->ad_perm + o, F + o,
                   E + o, f, (const cplx<T>*)nullptr, l2, (const cplx<T>*)nullptr,
                   (double2*)g, hn + o);
      ++nn;
    }
  }
  side_end(pl, 2, s2);
  prof_end(pl, nn);
  const FmmOps ops = cot_ops(pl);
  int rc = fmm_upward_downward<T>(pl, ops, true, f, pl->lvl2,
                                  sizeof(T) == 4 ? pl->lvl2f : nullptr);
  if (rc) return rc;
  prof_begin(pl, NUFFT_STAGE_M2L);
  const size_t sm = (size_t)6 * p * p * sizeof(T) + (size_t)kDeepWarps * 3 * p * sizeof(cplx<T>);
  cplx<T>* lad = (cplx<T>*)pl->ad_lexp;
  DeepTabs<T> tabs;
  for (int c = 1; c <= 3; ++c)
    tabs.rp[c - 1] = (const T*)pl->ad_p2m + pl->ad_toff[c <= D ? c - 1 : 0];
  launch_pdl(k_down_deep<T>, dim3((unsigned)pl->ad_nrleaf), kDeepWarps * 32, sm, pl->stream,
             dims_of(pl), (const int32_t*)pl->ad_rleaf, tabs, (const T*)ops.m2l,
             (const T*)ops.l2l, f, (const cplx<T>*)pl->lexp, lad);
  prof_end(pl, 1);
  side_join(pl, 2);
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  int nf = 0;
  for (int c = 0; c <= D; ++c) {
    const int64_t o = pl->ad_off[c], mc = pl->ad_off[c + 1] - o;
    if (mc == 0) continue;
    const TreeDims dc = class_dims(pl, c);
    const cplx<T>* lx = c == 0 ? (const cplx<T>*)pl->lexp : lad;
    const unsigned nb = nblk(mc, kTgtThreads);
    if (c64)
      launch_far_fwd<T, float2>(p, nb, 0, pl->stream, dc, (int)mc, pos + o,
                                (const int32_t*)pl->ad_perm + o, F + o, E + o, f, lx, l2,
                                (const cplx<T>*)hn + o, (float2*)g);
    else
      launch_far_fwd<T, double2>(p, nb, 0, pl->stream, dc, (int)mc, pos + o,
                                 (const int32_t*)pl->ad_perm + o, F + o, E + o, f, lx, l2,
                                 (const cplx<T>*)hn + o, (double2*)g);
    ++nf;
  }
  prof_end(pl, nf);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// forward: grid samples f (cplx<T>, in pl->grid, [batch][N]) -> g ([batch][M], original order)
template <class T>
int fmm_forward(nufft_plan_s* pl, void* g) {
  if (pl->ad_D > 0 && pl->batch == 1 && pl->hnear) return fmm_forward_adaptive<T>(pl, g);
  const cplx<T>* f = (const cplx<T>*)pl->grid;
  const TreeDims d = dims_of(pl);
  const bool split = split_near(pl);
  const bool c64 = (pl->flags & NUFFT_IO_C64) != 0;
  if (split) {  // near field beside the tree passes (it needs f only)
    prof_begin(pl, NUFFT_STAGE_TARGETS);
    cudaStream_t s2 = side_begin(pl, 2);
    {
      LowPriority lp;
      if (c64) launch_targets_fwd<T, float2, 1>(pl, d, f, nullptr, g, (cplx<T>*)pl->hnear, s2);
      else launch_targets_fwd<T, double2, 1>(pl, d, f, nullptr, g, (cplx<T>*)pl->hnear, s2);
    }
    side_end(pl, 2, s2);
    prof_end(pl, 1);
  }
  int rc = fmm_upward_downward<T>(pl, cot_ops(pl), true, f, pl->lvl2,
                                  sizeof(T) == 4 ? pl->lvl2f : nullptr);
  if (rc) return rc;
  const bool g4 = (pl->batch % 4) == 0;
  if (split) side_join(pl, 2);
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  // batches of 64 signals: near-field sums on the tensor cores first
  const cplx<T>* hnear = split ? (const cplx<T>*)pl->hnear : nullptr;
  if constexpr (std::is_same<T, float>::value) {
    if (pl->tc_near > 0) {
      int rc2 = near_tc_forward(d, (int)pl->M, pl->batch, pl->k0, pl->delta, pl->delta_f,
                                (const float2*)f, (float2*)pl->charge, pl->status, pl->stream);
      if (rc2) return rc2;
      hnear = (const cplx<T>*)pl->charge;
    }
  }
  if (split) {
    const size_t sm = 0;
    const unsigned nb = nblk(pl->M, kTgtThreads);
    if (c64)
      launch_far_fwd<T, float2>(pl->p, nb, sm, pl->stream, d, (int)pl->M,
                              (const SrcPos<T>*)pl->srcpos, (const int32_t*)pl->perm,
                              PlanT<T>::F(pl), PlanT<T>::E(pl), f, (const cplx<T>*)pl->lexp,
                              PlanT<T>::lvl2(pl), hnear, (float2*)g);
    else
      launch_far_fwd<T, double2>(pl->p, nb, sm, pl->stream, d, (int)pl->M,
                              (const SrcPos<T>*)pl->srcpos, (const int32_t*)pl->perm,
                              PlanT<T>::F(pl), PlanT<T>::E(pl), f, (const cplx<T>*)pl->lexp,
                              PlanT<T>::lvl2(pl), hnear, (double2*)g);
  } else if (pl->flags & NUFFT_IO_C64) {
    if (g4) launch_targets_fwd<T, float2, 4>(pl, d, f, hnear, g);
    else launch_targets_fwd<T, float2, 1>(pl, d, f, hnear, g);
  } else {
    if (g4) launch_targets_fwd<T, double2, 4>(pl, d, f, hnear, g);
    else launch_targets_fwd<T, double2, 1>(pl, d, f, hnear, g);
  }
  prof_end(pl, hnear ? 2 : 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// The warp-per-G-grid-points near field pays when the two-point kernel's
// CTAs (512 grid points each) would not fill the GPU or each grid point meets
// more than twice the sources of a uniform grid (M > 2N); NUFFT_NEAR_GRID2=1
// (environment) keeps the two-point kernel, NUFFT_NEAR_GRIDW=1 forces this one.
static bool gridw_wanted(const nufft_plan_s* pl) {
  static const int force = std::getenv("NUFFT_NEAR_GRIDW") ? 1 : (std::getenv("NUFFT_NEAR_GRID2") ? -1 : 0);
  if (force) return force > 0;
  return pl->N / (2 * kTgtThreads) < 2 * 152 || pl->M > 2 * pl->N ||
         (pl->M > 0 && (int64_t)pl->max_leaf * pl->B >= 4 * pl->M);
}

// adjoint / inverse: samples g ([batch][M], original order) -> values on the
// grid (cplx<T>, in pl->grid, [batch][N])
// near-field part of the adjoint / inverse targets for one signal (hout: the
// near-field sums and self terms only), or the whole evaluation (hout null)
template <class T>
static void launch_targets_grid1(nufft_plan_s* pl, const TreeDims& d, int inverse,
                                 const SrcPos<T>* pos, const cplx<T>* charge, const cplx<T>* stt,
                                 cplx<T>* hout, cudaStream_t st,
                                 InlineSrc<T> isrc = InlineSrc<T>()) {
  const cplx<T>* lexp_c = (const cplx<T>*)pl->lexp;
  if (gridw_wanted(pl)) {
    // many sources per grid point: one warp per G grid points (see k_targets_gridw)
    const unsigned nb = nblk(pl->N, (int64_t)(kTgtThreads / 32) * (pl->s >= 8 ? 8 : pl->s));
    if (pl->s >= 8)
      launch_pdl(k_targets_gridw<T, 8>, nb, kTgtThreads, 0, st, d, inverse, pl->leaf_start, pos,
                 charge, stt, lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid,
                 hout);
    else if (pl->s == 4)
      launch_pdl(k_targets_gridw<T, 4>, nb, kTgtThreads, 0, st, d, inverse, pl->leaf_start, pos,
                 charge, stt, lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid,
                 hout);
    else
      launch_pdl(k_targets_gridw<T, 2>, nb, kTgtThreads, 0, st, d, inverse, pl->leaf_start, pos,
                 charge, stt, lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid,
                 hout);
  } else {
    if (hout)
      launch_pdl(k_targets_grid2<T, 1>, near_grid(nblk(pl->N, 2 * kTgtThreads), true), kTgtThreads,
                 NearCap<T, 1>::grid_bytes, st, d, inverse, pl->leaf_start, pos, charge, stt,
                 lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid, hout,
                 (const cplx<T>*)nullptr, isrc);
    else
      launch_pdl(k_targets_grid2<T, 0>, nblk(pl->N, 2 * kTgtThreads), kTgtThreads,
                 NearCap<T, 1>::grid_bytes, st, d, inverse, pl->leaf_start, pos, charge, stt,
                 lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid, hout,
                 (const cplx<T>*)nullptr, isrc);
  }
}

template <class T, class VI>
static void launch_self_terms(nufft_plan_s* pl, const TreeDims& d, int inverse, const VI* g,
                              const cplx<T>* charge, cplx<T>* stt, cudaStream_t s1) {
  const dim3 gm(nblk(pl->M, 256), (unsigned)pl->batch);
  launch_pdl(k_self_terms<T, VI>, gm, 256, 0, s1, (int)pl->M, inverse, pl->perm, PlanT<T>::E(pl),
             inverse ? PlanT<T>::S(pl) : (const cplx<T>*)nullptr, charge, g, stt);
}

template <class T> struct AdInvT;
template <> struct AdInvT<double> {
  static const double2* D(nufft_plan_s* pl) { return pl->ad_Dt; }
  static const double2* S(nufft_plan_s* pl) { return pl->ad_S; }
};
template <> struct AdInvT<float> {
  static const float2* D(nufft_plan_s* pl) { return pl->ad_Dtf; }
  static const float2* S(nufft_plan_s* pl) { return pl->ad_Sf; }
};

// Adjoint / inverse with the adaptive tree (one signal).  Side branch 2,
// beside the uniform tree passes (which take every source, as before): the
// near-field sums of class 0 on every grid tile (charges and self terms
// formed inline), those of each deeper class (the uniform tree of depth
// L + d over its own sources, one warp per 8 grid points, its charges and
// self terms formed first in class order) added on the tiles it reaches,
// then level by level the deep boxes' multipoles and their M2L into the grid
// boxes of their interaction lists, added at those grid points.  After the join the far
// part reads the sums as with the uniform tree.
template <class T>
static int fmm_to_grid_adaptive(nufft_plan_s* pl, const void* g, int inverse) {
  cudaStream_t st = pl->stream;
  const bool c64 = (pl->flags & NUFFT_IO_C64) != 0;
  const int D = pl->ad_D, p = pl->p;
  const TreeDims d = dims_of(pl);
  const SrcPos<T>* pos = (const SrcPos<T>*)pl->ad_pos;
  const cplx<T>* coef = inverse ? AdInvT<T>::D(pl) : AdT<T>::F(pl);
  const cplx<T>* E = AdT<T>::E(pl);
  const cplx<T>* S = inverse ? AdInvT<T>::S(pl) : (const cplx<T>*)nullptr;
  if (inverse && !S) return NUFFT_EINVAL;
  cplx<T>* hn = (cplx<T>*)pl->hnear;
  const cplx<T>* l2 = PlanT<T>::lvl2(pl);
  const cplx<T>* lad = (const cplx<T>*)pl->ad_lexp;
  const FmmOps ops = cot_ops(pl);
  auto isrc_of = [&](int64_t o) {
    InlineSrc<T> is;
    is.a.inverse = inverse;
    is.a.perm = pl->ad_perm + o;
    is.a.gin = g;
    is.a.gin64 = c64 ? 0 : 1;
    is.coef = coef + o;
    is.E = E + o;
    if (S) is.S = S + o;
    return is;
  };
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  cudaStream_t s2 = side_begin(pl, 2);
  int nn = 0;
  {
    LowPriority lp;
    const int64_t o0 = pl->ad_off[0];
    launch_pdl(k_targets_grid2<T, 1>, near_grid(nblk(pl->N, 2 * kTgtThreads), true), kTgtThreads,
               NearCap<T, 1>::grid_bytes, s2, d, inverse,
               (const int32_t*)pl->ad_start + pl->ad_soff[0], pos + o0, (const cplx<T>*)nullptr,
               (const cplx<T>*)nullptr, (const cplx<T>*)pl->lexp, l2, PlanT<T>::Ct(pl),
               (cplx<T>*)pl->grid, hn, (const cplx<T>*)nullptr, isrc_of(o0));
    ++nn;
    // the deeper classes' charges and self terms in class order, then their
    // near fields one warp per 8 grid points (a refined leaf's grid points
    // each meet many sources)
    const int64_t o1 = pl->ad_off[1], m1 = pl->M - o1;
    cplx<T>* qa = (cplx<T>*)pl->ad_charge + o1;
    cplx<T>* sa = (cplx<T>*)pl->ad_st + o1;
    if (m1 > 0) {
      if (c64) {
        launch_pdl(k_charges<T, float2>, dim3(nblk(m1, 256), 1), 256, 0, s2, m1, pl->ad_perm + o1,
                   coef + o1, (int)!inverse, (const float2*)g, qa);
        launch_pdl(k_self_terms<T, float2>, dim3(nblk(m1, 256), 1), 256, 0, s2, (int)m1, inverse,
                   pl->ad_perm + o1, E + o1, S ? S + o1 : S, (const cplx<T>*)qa,
                   (const float2*)g, sa);
      } else {
        launch_pdl(k_charges<T, double2>, dim3(nblk(m1, 256), 1), 256, 0, s2, m1,
                   pl->ad_perm + o1, coef + o1, (int)!inverse, (const double2*)g, qa);
        launch_pdl(k_self_terms<T, double2>, dim3(nblk(m1, 256), 1), 256, 0, s2, (int)m1,
                   inverse, pl->ad_perm + o1, E + o1, S ? S + o1 : S, (const cplx<T>*)qa,
                   (const double2*)g, sa);
      }
      nn += 2;
    }
    for (int c = 1; c <= D; ++c) {
      const int64_t o = pl->ad_off[c], nt = pl->ad_tioff[c] - pl->ad_tioff[c - 1];
      if (nt == 0) continue;
      launch_pdl(k_targets_gridw_ad<T>, dim3((unsigned)(nt * kGridwTileCtas)), kTgtThreads, 0, s2,
                 class_dims(pl, c), inverse, (const int32_t*)pl->ad_tiles + pl->ad_tioff[c - 1],
                 (const int32_t*)pl->ad_start + pl->ad_soff[c], pos + o,
                 (const cplx<T>*)pl->ad_charge + o, (const cplx<T>*)pl->ad_st + o, hn);
      ++nn;
    }
    const size_t smp = (size_t)kDeepWarps * 32 * kP2mPitch * sizeof(cplx<T>);
    const size_t sml = (size_t)6 * p * p * sizeof(T) + (size_t)(kDeepWarps + 1) * p * sizeof(cplx<T>);
    for (int c = 1; c <= D; ++c) {
      const int64_t b0 = pl->ad_boff[c - 1], nbox = pl->ad_boff[c] - b0;
      const int64_t g0 = pl->ad_goff[c - 1], ng = pl->ad_goff[c] - g0;
      cplx<T>* mx = (cplx<T>*)pl->ad_mexp + b0 * p;
      launch_pdl(k_deep_p2m<T>, dim3(nblk(nbox, kDeepWarps)), kDeepWarps * 32, smp, s2, d,
                 pl->L + c, (int)nbox, (const int32_t*)pl->ad_box + b0,
                 (const int32_t*)pl->ad_srange + 2 * b0, pos, isrc_of(0), mx);
      if (ng > 0)
        launch_pdl(k_deep_m2l_grid<T>, dim3(nblk(ng, kDeepWarps)), kDeepWarps * 32, sml, s2, d,
                   pl->L + c, (int)ng, (const int32_t*)pl->ad_gbox + g0,
                   (const int32_t*)pl->ad_gil + 3 * g0, (const T*)ops.m2l, (const T*)ops.l2l,
                   (const cplx<T>*)mx, hn);
      nn += 2;
    }
  }
  side_end(pl, 2, s2);
  prof_end(pl, nn);
  cplx<T>* charge = (cplx<T>*)pl->charge;
  const cplx<T>* coef_u = inverse ? PlanT<T>::D(pl) : PlanT<T>::F(pl);
  double2* lv2 = pl->lvl2;
  float2* lv2f = sizeof(T) == 4 ? pl->lvl2f : nullptr;
  int rc = c64 ? fmm_upward<T, float2>(pl, ops, false, charge, coef_u, (int)!inverse,
                                       (const float2*)g, nullptr, lv2, lv2f)
               : fmm_upward<T, double2>(pl, ops, false, charge, coef_u, (int)!inverse,
                                        (const double2*)g, nullptr, lv2, lv2f);
  if (rc) return rc;
  rc = fmm_downward<T>(pl, ops);
  if (rc) return rc;
  side_join(pl, 2);
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  launch_far_grid2<T>(pl->p, nblk(pl->N, 2 * kTgtThreads), (size_t)0, st, d, inverse,
                      (const int32_t*)pl->leaf_start, (const SrcPos<T>*)pl->srcpos,
                      (const cplx<T>*)charge, (const cplx<T>*)pl->selft,
                      (const cplx<T>*)pl->lexp, l2, PlanT<T>::Ct(pl), (cplx<T>*)pl->grid,
                      (cplx<T>*)nullptr, (const cplx<T>*)hn, InlineSrc<T>());
  prof_end(pl, 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// adjoint / inverse: samples g ([batch][M], original order) -> values on the
// grid (cplx<T>, in pl->grid, [batch][N])
template <class T>
int fmm_to_grid(nufft_plan_s* pl, const void* g, int inverse) {
  if (pl->ad_D > 0 && pl->batch == 1 && pl->hnear) return fmm_to_grid_adaptive<T>(pl, g, inverse);
  cudaStream_t st = pl->stream;
  bool c64 = (pl->flags & NUFFT_IO_C64) != 0;
  const cplx<T>* coef = inverse ? PlanT<T>::D(pl) : PlanT<T>::F(pl);
  cplx<T>* charge = (cplx<T>*)pl->charge;
  const unsigned nsig = (unsigned)pl->batch;
  const TreeDims d = dims_of(pl);
  cplx<T>* stt = (cplx<T>*)pl->selft;
  SrcPos<T>* pos = (SrcPos<T>*)pl->srcpos;
  // charges q_i = coef_i g_perm(i) (conj(F_i) for the adjoint) and the
  // upward pass; the charges are formed inside the upward kernel when it
  // forms the leaf multipoles itself
  const FmmOps ops = cot_ops(pl);
  double2* l2 = pl->lvl2;
  float2* l2f = sizeof(T) == 4 ? pl->lvl2f : nullptr;
  int rc;
  const bool split = split_near(pl) && pl->s >= 2;
  if (split) {
    // on side branch 2 the near-field sums (with the self terms), which need
    // nothing from the tree passes: the two-point kernel forms the charges
    // and self terms of its staged sources itself, so it starts at once
    // beside the upward pass (which forms the charges it needs too); the
    // warp-per-grid-points kernel reads them from a charge kernel and a
    // self-term kernel run first
    const bool inl = !gridw_wanted(pl);
    InlineSrc<T> isrc;
    if (inl) {
      isrc.a.inverse = inverse;
      isrc.a.perm = pl->perm;
      isrc.a.gin = g;
      isrc.a.gin64 = c64 ? 0 : 1;
      isrc.coef = coef;
      isrc.E = PlanT<T>::E(pl);
      if (inverse) isrc.S = PlanT<T>::S(pl);
    } else {
      prof_begin(pl, NUFFT_STAGE_P2M);
      if (c64)
        launch_pdl(k_charges<T, float2>, dim3(nblk(pl->M, 256), nsig), 256, 0, st, pl->M,
                   pl->perm, coef, (int)!inverse, (const float2*)g, charge);
      else
        launch_pdl(k_charges<T, double2>, dim3(nblk(pl->M, 256), nsig), 256, 0, st, pl->M,
                   pl->perm, coef, (int)!inverse, (const double2*)g, charge);
      prof_end(pl, 1);
    }
    prof_begin(pl, NUFFT_STAGE_TARGETS);
    cudaStream_t s2 = side_begin(pl, 2);
    {
      LowPriority lp;
      if (!inl) {
        if (c64) launch_self_terms<T, float2>(pl, d, inverse, (const float2*)g, charge, stt, s2);
        else launch_self_terms<T, double2>(pl, d, inverse, (const double2*)g, charge, stt, s2);
      }
      launch_targets_grid1<T>(pl, d, inverse, pos, charge, stt, (cplx<T>*)pl->hnear, s2, isrc);
    }
    side_end(pl, 2, s2);
    prof_end(pl, inl ? 1 : 2);
    if (inl)
      rc = c64 ? fmm_upward<T, float2>(pl, ops, false, charge, coef, (int)!inverse,
                                       (const float2*)g, nullptr, l2, l2f)
               : fmm_upward<T, double2>(pl, ops, false, charge, coef, (int)!inverse,
                                        (const double2*)g, nullptr, l2, l2f);
    else
      rc = fmm_upward<T, float2>(pl, ops, false, charge, coef, (int)!inverse,
                                 (const float2*)nullptr, nullptr, l2, l2f);
    if (rc) return rc;
    rc = fmm_downward<T>(pl, ops);
    if (rc) return rc;
    side_join(pl, 2);
    prof_begin(pl, NUFFT_STAGE_TARGETS);
    launch_far_grid2<T>(pl->p, nblk(pl->N, 2 * kTgtThreads),
                        (size_t)0, st, d,
                        inverse, (const int32_t*)pl->leaf_start, (const SrcPos<T>*)pos,
                        (const cplx<T>*)charge, (const cplx<T>*)stt, (const cplx<T>*)pl->lexp,
                        PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid,
                        (cplx<T>*)nullptr, (const cplx<T>*)pl->hnear, InlineSrc<T>());
    prof_end(pl, 1);
    return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
  }
  bool done = false;
  rc = c64 ? fmm_upward<T, float2>(pl, ops, false, charge, coef, (int)!inverse,
                                   (const float2*)g, &done, l2, l2f)
           : fmm_upward<T, double2>(pl, ops, false, charge, coef, (int)!inverse,
                                    (const double2*)g, &done, l2, l2f);
  if (rc) return rc;
  if (!done) return NUFFT_ECUDA;
  // self terms on the side branch (they need the charges; only the targets
  // kernel needs them), overlapping the downward pass
  prof_begin(pl, NUFFT_STAGE_OTHER);
  cudaStream_t s1 = side_begin(pl, 1);
  if (c64) launch_self_terms<T, float2>(pl, d, inverse, (const float2*)g, charge, stt, s1);
  else launch_self_terms<T, double2>(pl, d, inverse, (const double2*)g, charge, stt, s1);
  side_end(pl, 1, s1);
  prof_end(pl, 1);
  rc = fmm_downward<T>(pl, ops);
  if (rc) return rc;
  side_join(pl, 1);
  prof_begin(pl, NUFFT_STAGE_TARGETS);
  const cplx<T>* lexp_c = (const cplx<T>*)pl->lexp;
  if (pl->batch % 4 == 0)
    launch_pdl(k_targets_grid<T, 4>, dim3(nblk(pl->N, kTgtThreads), nsig / 4), kTgtThreads,
               NearCap<T, 4>::grid_bytes, st, d, inverse, pl->leaf_start, pos, charge, stt,
               lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid);
  else if (nsig == 1 && pl->s >= 2)
    launch_targets_grid1<T>(pl, d, inverse, pos, charge, stt, nullptr, st);
  else
    launch_pdl(k_targets_grid<T, 1>, dim3(nblk(pl->N, kTgtThreads), nsig), kTgtThreads,
               NearCap<T, 1>::grid_bytes, st, d, inverse, pl->leaf_start, pos, charge, stt,
               lexp_c, PlanT<T>::lvl2(pl), PlanT<T>::Ct(pl), (cplx<T>*)pl->grid);
  prof_end(pl, 1);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template int fmm_configure<double>();
template int fmm_configure<float>();
// Source positions of the adjoint / inverse near field, packed once per plan.
int fmm_pack_positions(nufft_plan_s* pl) {
  if (pl->prec == NUFFT_FP64)
    k_pack_positions<double><<<nblk(pl->M, 256), 256, 0, pl->stream>>>(
        (int)pl->M, pl->k0, pl->delta, (SrcPos<double>*)pl->srcpos);
  else
    k_pack_positions<float><<<nblk(pl->M, 256), 256, 0, pl->stream>>>(
        (int)pl->M, pl->k0, pl->delta, (SrcPos<float>*)pl->srcpos);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template int fmm_forward<double>(nufft_plan_s*, void*);
template int fmm_forward<float>(nufft_plan_s*, void*);
template int fmm_to_grid<double>(nufft_plan_s*, const void*, int);
template int fmm_to_grid<float>(nufft_plan_s*, const void*, int);
template int fmm_upward_downward<double>(nufft_plan_s*, const FmmOps&, bool, const double2*,
                                         double2*, float2*);
