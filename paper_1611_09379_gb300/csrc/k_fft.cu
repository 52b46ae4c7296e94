// Stockham auto-sort FFT for the c_n <-> f_k step (Eq. p1, Sec. 2):
//   out_n = sum_k in_k e^{sign 2 pi i n k / N},  N = 2^L, no scaling.
// Each pass is one radix-R Stockham iteration,
//   a_r = in[j + r N/R] * w^{sign r (j mod Ns) / (Ns R)},  A = DFT_R(a),
//   out[(j/Ns) Ns R + (j mod Ns) + r' Ns] = A_r',
// with the size-R DFTs of J adjacent columns j done by one CTA (so the
// strided global reads and writes move J contiguous elements).  Passes
// multiply Ns by R until it reaches N.  Inside a CTA the size-R DFT is
// itself a Stockham sequence of radix-8 stages (the last one radix 2 or 4
// when 3 does not divide log2 R), each thread holding 8 elements in
// registers between stages, which exchange through shared memory.
// Twiddles come from two small tables, w^{m/N} = T_hi[m >> b] *
// T_lo[m & (2^b - 1)], filled once per plan with sincospi of exact
// arguments.
#include <cstdint>
#include <cstdlib>

#include "common.cuh"

namespace nufft {

constexpr int kFftSmemElems = 4096;  // R * J complex elements per CTA (at most)
constexpr int kFftMaxThreads = 512;

// Twiddle tables of a plan: w_N^m = T_hi[m >> b] T_lo[m & (2^b - 1)] (T_lo
// first, 2^b entries, then T_hi, N / 2^b entries), then the radix-1024 pass
// table w_1024^{ka t} at [ka 32 + t] (ka, t < 32).
__global__ void k_fft_tables(double2* __restrict__ tw, int64_t N, int lo_bits) {
  int64_t nlo = int64_t(1) << lo_bits, nhi = N >> lo_bits;
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double s, c;
  if (i < nlo) {
    sincospi(2.0 * (double)i / (double)N, &s, &c);
    tw[i] = make_double2(c, s);
  } else if (i < nlo + nhi) {
    int64_t h = i - nlo;
    // 2 h 2^b / N reduced mod 2 exactly (all powers of two)
    sincospi(2.0 * (double)(h << lo_bits) / (double)N, &s, &c);
    tw[i] = make_double2(c, s);
  } else if (i < nlo + nhi + 1024) {
    const int e = (int)(i - nlo - nhi);
    sincospi((double)((e >> 5) * (e & 31)) / 512.0, &s, &c);  // exact argument
    tw[i] = make_double2(c, s);
  }
}

template <int LOG> __device__ constexpr int brev_c(int x) {
  int r = 0;
  for (int i = 0; i < LOG; ++i) r |= ((x >> i) & 1) << (LOG - 1 - i);
  return r;
}

// Shared-memory slot of element e = r J + c of the CTA's columns: one spare
// slot per 32, so the stage writes with stride 8 J spread over the banks.
__device__ inline int fft_pad(int e) { return e + (e >> 5); }

// x * (sg i), sg = +-1
template <class T> __device__ inline cplx<T> mul_si(cplx<T> x, T sg) { return mk<T>(-sg * x.y, sg * x.x); }

// Size-2^LOGRAD DFT in registers, decimation in frequency: a in natural
// order, X_k = sum_m a_m e^{sg 2 pi i m k / RAD} left in a[brev(k)].  The
// twiddles of radix 8 are the constants (+-1 +- i) / sqrt 2 and +-i.
template <class T, int LOGRAD>
__device__ inline void dft_small(cplx<T>* a, T sg) {
  if constexpr (LOGRAD == 3) {
    const T h = (T)0.70710678118654752440;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const cplx<T> u = a[k], v = a[k + 4];
      a[k] = cadd(u, v);
      cplx<T> d = csub(u, v);
      if (k == 1) d = mk<T>(h * (d.x - sg * d.y), h * (d.y + sg * d.x));
      if (k == 2) d = mul_si(d, sg);
      if (k == 3) d = mk<T>(-h * (d.x + sg * d.y), h * (sg * d.x - d.y));
      a[k + 4] = d;
    }
#pragma unroll
    for (int hh = 0; hh < 8; hh += 4)
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const cplx<T> u = a[hh + k], v = a[hh + k + 2];
        a[hh + k] = cadd(u, v);
        const cplx<T> d = csub(u, v);
        a[hh + k + 2] = k ? mul_si(d, sg) : d;
      }
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      const cplx<T> u = a[k], v = a[k + 1];
      a[k] = cadd(u, v);
      a[k + 1] = csub(u, v);
    }
  } else if constexpr (LOGRAD == 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const cplx<T> u = a[k], v = a[k + 2];
      a[k] = cadd(u, v);
      const cplx<T> d = csub(u, v);
      a[k + 2] = k ? mul_si(d, sg) : d;
    }
#pragma unroll
    for (int k = 0; k < 4; k += 2) {
      const cplx<T> u = a[k], v = a[k + 1];
      a[k] = cadd(u, v);
      a[k + 1] = csub(u, v);
    }
  } else {
    const cplx<T> u = a[0], v = a[1];
    a[0] = cadd(u, v);
    a[1] = csub(u, v);
  }
}

// Shape of a pass kernel for R = 2^LOGR: E elements per thread, TPC
// threads per column, at most JMAX columns (kFftMaxThreads threads,
// kFftSmemElems elements); buffers: two (FP32: one barrier per stage) or one.
template <class T, int LOGR> struct FftShape {
  static constexpr int R = 1 << LOGR, LOGE = LOGR < 3 ? LOGR : 3, E = 1 << LOGE, TPC = R / E;
  static constexpr int JT = kFftMaxThreads / TPC, JS = kFftSmemElems / R;
  static constexpr int JMAX = JT < JS ? JT : JS;
  static constexpr int NBUF = sizeof(T) == 4 ? 2 : 1;
};

// Slot of element e + K (K >= 0) given the slot of e: for K a multiple of
// 32 (compile-time after unrolling when J is) the padding shifts by K / 32.
template <int JC>
__device__ inline int pad_add(int e, int pe, int K) {
  if (JC != 0 && (K & 31) == 0) return pe + K + (K >> 5);
  return fft_pad(e + K);
}

// One radix-2^LOGRAD Stockham stage of the R-point DFTs of the CTA's J
// columns (element r of column c in buffer[fft_pad(r J + c)]), Ns = 2^LOGNS
// the length of the sub-DFTs done so far.  Thread (c, q), q < TPC, does the
// butterflies b = q + i TPC, i < E / 2^LOGRAD:
//   x_m = src[b + m R / 2^LOGRAD] w^m,  w = w_{Ns 2^LOGRAD}^{b mod Ns},  A = DFT(x),
//   dst[(b / Ns) Ns 2^LOGRAD + (b mod Ns) + k Ns] = A_k.
// w is read from the table once per butterfly, its powers formed by
// products (w^2 = w w, w^3 = w^2 w, w^4 = w^2 w^2, ...: at most three
// roundings deep).  IN_REGS: the inputs are already in v (the first stage,
// straight from the loads); src == dst (one buffer) needs a barrier between
// the reads and the writes.  LAST (Ns 2^LOGRAD = R): the outputs stay in
// registers, v[m] = element q + m TPC (butterfly i, output k: m = i + k E /
// 2^LOGRAD), which is the thread's share of the pass output.
template <class T, int LOGR, int LOGRAD, int LOGNS, int JC, bool IN_REGS, bool LAST = false>
__device__ inline void fft_stage(cplx<T>* v, const cplx<T>* src, cplx<T>* dst,
                                 const cplx<T>* __restrict__ wR, int J, int c, int q, T sg) {
  using S = FftShape<T, LOGR>;
  constexpr int R = S::R, E = S::E, TPC = S::TPC;
  constexpr int RAD = 1 << LOGRAD, NB = E / RAD, NS = 1 << LOGNS;
  if (!IN_REGS) {
    const int e0 = q * J + c, p0 = fft_pad(e0);
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
      for (int m = 0; m < RAD; ++m)
        v[i * RAD + m] = src[pad_add<JC>(e0, p0, (i * TPC + m * (R / RAD)) * J)];
    if (!LAST && src == dst) __syncthreads();  // every input read before any output is written
  }
  cplx<T> o[E];  // LAST: outputs by row
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = q + i * TPC, j = b & (NS - 1);
    cplx<T>* a = v + i * RAD;
    if (LOGNS > 0 && j != 0) {
      const cplx<T> w1 = wR[j << (LOGR - LOGNS - LOGRAD)];
      a[1] = cmul(a[1], w1);
      if constexpr (RAD >= 4) {
        const cplx<T> w2 = cmul(w1, w1), w3 = cmul(w2, w1);
        a[2] = cmul(a[2], w2);
        a[3] = cmul(a[3], w3);
        if constexpr (RAD == 8) {
          const cplx<T> w4 = cmul(w2, w2);
          a[4] = cmul(a[4], w4);
          a[5] = cmul(a[5], cmul(w4, w1));
          a[6] = cmul(a[6], cmul(w4, w2));
          a[7] = cmul(a[7], cmul(w4, w3));
        }
      }
    }
    dft_small<T, LOGRAD>(a, sg);
    if constexpr (LAST) {
#pragma unroll
      for (int k = 0; k < RAD; ++k) o[i + k * NB] = a[brev_c<LOGRAD>(k)];
      continue;
    }
    const int e0 = (((b >> LOGNS) << (LOGNS + LOGRAD)) + j) * J + c, p0 = fft_pad(e0);
    // the butterfly's outputs span Ns RAD J slots from a multiple of that
    // span: inside one 32-slot row when the span is at most 32
    const bool one_row = JC != 0 && NS * RAD * JC <= 32;
#pragma unroll
    for (int k = 0; k < RAD; ++k) {
      const int K = (k << LOGNS) * J;
      dst[one_row ? p0 + K : pad_add<JC>(e0, p0, K)] = a[brev_c<LOGRAD>(k)];
    }
  }
  if constexpr (LAST) {
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = o[m];
  } else {
    __syncthreads();
  }
}

// Stages ST = 1, 2, ... after the first: radix 8 while at least 3 bits are
// left, then radix 2 or 4; buffers alternate when there are two.
template <class T, int LOGR, int JC, int ST>
__device__ inline void fft_stages(cplx<T>* v, cplx<T>* X0, cplx<T>* X1,
                                  const cplx<T>* __restrict__ wR, int J, int c, int q, T sg) {
  using S = FftShape<T, LOGR>;
  constexpr int LOGNS = S::LOGE + 3 * (ST - 1);
  if constexpr (LOGNS < LOGR) {
    constexpr int LEFT = LOGR - LOGNS, LOGRAD = LEFT < 3 ? LEFT : 3;
    cplx<T>* src = (S::NBUF == 2 && (ST & 1) == 0) ? X1 : X0;
    cplx<T>* dst = (S::NBUF == 2 && (ST & 1) == 1) ? X1 : X0;
    fft_stage<T, LOGR, LOGRAD, LOGNS, JC, false, LOGNS + LOGRAD == LOGR>(v, src, dst, wR, J, c, q,
                                                                         sg);
    fft_stages<T, LOGR, JC, ST + 1>(v, X0, X1, wR, J, c, q, sg);
  }
}

// One radix-R Stockham pass (R = 2^LOGR) for J columns j per CTA (JC: J at
// compile time, 0 = Jrt at run time), J TPC threads; thread (c, q) =
// (tid mod J, tid / J) loads elements r = q + m TPC (m < E) of column c
// with the pass twiddle, runs the first stage from registers and the rest
// through shared memory; the result goes to
// out[(j / Ns) Ns R + (j mod Ns) + r' Ns] in contiguous runs (J per r' for
// Ns >= J, else R per j).
// e^{sign 2 pi i m / N} from the two tables, 32-bit exponent m < N
template <class T>
__device__ inline cplx<T> twiddle32(const cplx<T>* __restrict__ tw, uint32_t m, int lo_bits,
                                    uint32_t lo_mask, T sg) {
  const cplx<T> a = tw[m & lo_mask], b = tw[(lo_mask + 1) + (m >> lo_bits)];
  cplx<T> r = cmul(a, b);
  r.y *= sg;
  return r;
}

template <class T>
__device__ inline cplx<T> ld_cv(const float2* p) {
  const float2 v = *p;
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ inline cplx<T> ld_cv(const double2* p) {
  return c128_to<T>(*p);
}

// loads of a pass: element r = q + m TPC of column jg at in[jg + r NR],
// times w^{(r jm N / (Ns R)) mod N}, the exponent advancing by
// de = TPC jm N / (Ns R) per m (32-bit offsets: N < 2^31).  All E loads are
// issued before the first twiddle is applied, so they are in flight together.
template <class T, int E, class V>
__device__ inline void fft_load(cplx<T>* v, const V* __restrict__ in, uint32_t idx,
                                uint32_t stride, uint32_t n_in, uint32_t ex, uint32_t de,
                                uint32_t nmask, const cplx<T>* __restrict__ tw, int lo_bits,
                                uint32_t lo_mask, T sg) {
  V raw[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const uint32_t e = idx + m * stride;
    if (e < n_in) raw[m] = in[e];  // elements n_in .. N - 1 are the zero padding
    else { raw[m].x = 0; raw[m].y = 0; }
  }
  if (de == 0 && ex == 0) {  // first pass (Ns = 1) and column 0: no twiddles
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = ld_cv<T>(&raw[m]);
    return;
  }
  cplx<T> w[E];
#pragma unroll
  for (int m = 0; m < E; ++m) {
    w[m] = twiddle32<T>(tw, ex, lo_bits, lo_mask, sg);  // w^0 = 1 exactly from the tables
    ex = (ex + de) & nmask;
  }
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = cmul(ld_cv<T>(&raw[m]), w[m]);
}

template <class T>
__device__ inline void st_cv(float2* p, cplx<T> v) {
  *p = make_float2((float)v.x, (float)v.y);
}
template <class T>
__device__ inline void st_cv(double2* p, cplx<T> v) {
  *p = to_c128(v);
}

// One radix-R Stockham pass (R = 2^LOGR) for J columns j per CTA (JC: J at
// compile time, 0 = Jrt at run time), J TPC threads; thread (c, q) =
// (tid mod J, tid / J) loads elements r = q + m TPC (m < E) of column c
// with the pass twiddle, runs the first stage from registers and the rest
// through shared memory; the result goes to
// out[(j / Ns) Ns R + (j mod Ns) + r' Ns] in contiguous runs (J per r' for
// Ns >= J, else R per j).  N = 2^logN < 2^31, Ns = 2^logNs.  The input holds
// n_in <= N elements per signal (signal stride n_in; the rest read as zero)
// and the output keeps the first n_out <= N (signal stride n_out): both N for
// the passes between two work buffers.
template <class T, int LOGR, int JC>
__global__ void __launch_bounds__(kFftMaxThreads, sizeof(T) == 4 ? 3 : 2) k_fft_st(
    const void* __restrict__ in, int in_f64, void* __restrict__ out, int out_f64, int logN,
    int logNs, int Jrt, int logJrt, int sign, const cplx<T>* __restrict__ tw, int lo_bits,
    uint32_t n_in, uint32_t n_out) {
  using S = FftShape<T, LOGR>;
  constexpr int R = S::R, LOGE = S::LOGE, E = S::E, TPC = S::TPC;
  const int J = JC ? JC : Jrt;
  int logJ = logJrt;
  if (JC) {
    logJ = 0;
    while ((1 << logJ) < JC) ++logJ;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* wR = reinterpret_cast<cplx<T>*>(smraw);  // [R] w_R^e
  cplx<T>* X0 = wR + R;                             // [fft_pad(R J) + 1] columns
  cplx<T>* X1 = X0 + (S::NBUF == 2 ? R * J + (R * J >> 5) + 1 : 0);
  const uint32_t N = 1u << logN, nmask = N - 1, Ns = 1u << logNs;
  const int lognr = logN - LOGR;  // NR = N / R
  const uint32_t lo_mask = (1u << lo_bits) - 1;
  const int tid = threadIdx.x, nth = blockDim.x;
  const T sg = (T)sign;
  for (int e = tid; e < R; e += nth)
    wR[e] = twiddle32<T>(tw, (uint32_t)e << lognr, lo_bits, lo_mask, sg);
  // (the twiddle tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  const int c = tid & (J - 1), q = tid >> logJ;
  const uint32_t j0 = blockIdx.x * (uint32_t)J;
  const uint32_t jg = j0 + c, jm = jg & (Ns - 1);
  cplx<T> v[E];
  {
    const int lstep = logN - logNs - LOGR;  // N / (Ns R) = 2^lstep
    const uint32_t idx = jg + ((uint32_t)q << lognr), stride = (uint32_t)TPC << lognr;
    const uint32_t ex = ((q * jm) << lstep) & nmask, de = ((TPC * jm) << lstep) & nmask;
    const size_t sig = (size_t)blockIdx.y * n_in;
    if (in_f64)
      fft_load<T, E>(v, reinterpret_cast<const double2*>(in) + sig, idx, stride, n_in, ex, de,
                     nmask, tw, lo_bits, lo_mask, sg);
    else
      fft_load<T, E>(v, reinterpret_cast<const float2*>(in) + sig, idx, stride, n_in, ex, de,
                     nmask, tw, lo_bits, lo_mask, sg);
  }
  __syncthreads();  // wR ready
  fft_stage<T, LOGR, LOGE, 0, JC, true, LOGE == LOGR>(v, X0, X0, wR, J, c, q, sg);
  fft_stages<T, LOGR, JC, 1>(v, X0, X1, wR, J, c, q, sg);
  // v[m] = A_r' of column c, r' = q + m TPC -> out[(j / Ns) Ns R + (j mod Ns) + r' Ns]
  // (J contiguous per r' for Ns >= J; runs of TPC per column for Ns = 1)
  const size_t sig = (size_t)blockIdx.y * n_out;
  const uint32_t d0 = ((jg >> logNs) << (logNs + LOGR)) + jm + ((uint32_t)q << logNs);
  const uint32_t dstep = (uint32_t)TPC << logNs;
  if (out_f64) {
    double2* o = reinterpret_cast<double2*>(out) + sig;
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (d0 + m * dstep < n_out) st_cv<T>(o + d0 + m * dstep, v[m]);
  } else {
    float2* o = reinterpret_cast<float2*>(out) + sig;
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (d0 + m * dstep < n_out) st_cv<T>(o + d0 + m * dstep, v[m]);
  }
}

// ------------------------------------------- radix-1024 pass, one warp per column (FP32)
//
// The same pass as k_fft_st for R = 1024 = 32 x 32, with r = t + 32 m (t the
// lane, m a register index) and r' = ka + 32 kb:
//   A_{ka + 32 kb} = sum_t w_32^{t kb} [ w_1024^{t ka} sum_m a_{t + 32 m} w_32^{m ka} ]:
// stage A is lane t's 32-point DFT over m in registers, then the twiddle
// w_1024^{t ka} from a [ka][t] table in shared memory (conflict-free: the
// lanes read consecutive entries), a transpose through shared memory inside
// the warp (no CTA barrier), stage B lane ka's 32-point DFT over t.  The
// CTA's four warps take four adjacent columns j; their strided rows are
// loaded (and, for Ns > 1, stored) by the whole CTA as runs of four adjacent
// elements through shared memory.  The pass twiddle w_{Ns R}^{r jm} factors
// into w^{t jm} (per lane) times w^{32 m jm} (per warp, from shared memory).

// COLS columns (warps) per CTA: rows of the strided passes move as runs of
// COLS adjacent elements (32, 64 or 128 bytes)
template <int COLS> struct W32Shape {
  static constexpr int threads = 32 * COLS;
  // column stride in shared memory: rows 33 m + t, then 16 / COLS slots so
  // the staging accesses (COLS columns x 32 / COLS rows per half-warp) fall
  // in different banks
  static constexpr int stride = 1056 + 16 / COLS;
  static constexpr size_t smem = (size_t)(COLS * stride + 1024 + COLS * 32) * sizeof(float2);
};

// cos and sin of 2 pi e / 32 (the exact values rounded to FP32), e in [0, 32)
__host__ __device__ constexpr float w32_cos(int e) {
  constexpr float q[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f,
                          0.83146961230254523708f, 0.70710678118654752440f,
                          0.55557023301960222474f, 0.38268343236508977173f,
                          0.19509032201612826785f, 0.0f};
  return e <= 8 ? q[e] : e <= 16 ? -q[16 - e] : e <= 24 ? -q[e - 16] : q[32 - e];
}
__host__ __device__ constexpr float w32_sin(int e) { return w32_cos((e + 24) & 31); }

// x e^{sg 2 pi i e / 32}, e a compile-time constant after unrolling
__device__ inline float2 w32_mul(float2 x, int e, float sg) {
  e &= 31;
  if (e == 0) return x;
  if (e == 8) return mul_si<float>(x, sg);
  if (e == 16) return make_float2(-x.x, -x.y);
  if (e == 24) return mul_si<float>(x, -sg);
  const float c = w32_cos(e), s = sg * w32_sin(e);
  return make_float2(x.x * c - x.y * s, x.x * s + x.y * c);
}

// X_k = sum_n a_n e^{sg 2 pi i n k / 32} in place, natural order in and out:
// n = n1 + 4 n2, k = 8 k1 + k2, four radix-8 DFTs over n2, the twiddles
// w_32^{n1 k2}, eight radix-4 DFTs over n1.
__device__ inline void dft32(float2* a, float sg) {
  float2 y[32];  // y[n1 8 + k2]
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) {
    float2 b[8];
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2) b[n2] = a[n1 + 4 * n2];
    dft_small<float, 3>(b, sg);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) y[n1 * 8 + k2] = w32_mul(b[brev_c<3>(k2)], n1 * k2, sg);
  }
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    float2 c[4];
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) c[n1] = y[n1 * 8 + k2];
    dft_small<float, 2>(c, sg);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[8 * k1 + k2] = c[brev_c<2>(k1)];
  }
}

// One radix-1024 Stockham pass (the k_fft_st pass with R = 1024) for
// N = 2^logN >= 4096 and Ns = 1 or Ns >= 4: 128 threads, four columns
// j = 4 blockIdx.x + warp, signal blockIdx.y.  tw: the two-level FP32
// twiddle tables of w_N; tw32: w_1024^{ka t} at [ka 32 + t] (sign +1).
template <int COLS>
__global__ void __launch_bounds__(32 * COLS, 16 / COLS) k_fft_w32(
    const void* __restrict__ in, int in_f64, void* __restrict__ out, int out_f64, int logN,
    int logNs, int sign, const float2* __restrict__ tw, const float2* __restrict__ tw32,
    int lo_bits, uint32_t n_in, uint32_t n_out) {
  using S = W32Shape<COLS>;
  constexpr int kW32Cols = COLS, kW32Stride = S::stride, NT = S::threads;
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* X = reinterpret_cast<float2*>(smraw);  // [COLS][stride]
  float2* TW = X + kW32Cols * kW32Stride;        // [32 ka][32 t]
  float2* BM = TW + 1024;                        // [COLS warps][32 m]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const float sg = (float)sign;
  const uint32_t N = 1u << logN, nmask = N - 1, Ns = 1u << logNs;
  const int lognr = logN - 10;
  const uint32_t lo_mask = (1u << lo_bits) - 1;
  const uint32_t j0 = blockIdx.x * (uint32_t)kW32Cols, j = j0 + w, jm = j & (Ns - 1);
  float2 At = make_float2(1.0f, 0.0f);
  {
    // all table loads in flight together (a loop of load-store pairs would
    // wait for each load in turn)
    float2 tv[1024 / NT];
#pragma unroll
    for (int u = 0; u < 1024 / NT; ++u) tv[u] = tw32[tid + NT * u];
    if (Ns > 1) {  // w_{Ns R}^{e} = w_N^{e N / (Ns R)}, N / (Ns R) = 2^lstep
      const int lstep = logN - logNs - 10;
      At = twiddle32<float>(tw, ((lane * jm) << lstep) & nmask, lo_bits, lo_mask, sg);
      BM[w * 32 + lane] =
          twiddle32<float>(tw, ((32u * lane * jm) << lstep) & nmask, lo_bits, lo_mask, sg);
    }
#pragma unroll
    for (int u = 0; u < 1024 / NT; ++u) {
      tv[u].y *= sg;
      TW[tid + NT * u] = tv[u];
    }
  }
  // (the twiddle tables are plan constants: read before the predecessor ends)
  pdl_wait();
  pdl_trigger();
  const int c4 = tid % COLS, q4 = tid / COLS;  // staging: column j0 + c4, rows q4 + 32 i
  {
    float2* xc = X + c4 * kW32Stride + q4;
    const uint32_t e0 = j0 + c4 + ((uint32_t)q4 << lognr), de = 32u << lognr;
    if (in_f64) {
      const double2* src = reinterpret_cast<const double2*>(in) + (size_t)blockIdx.y * n_in;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        double2 raw[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const uint32_t e = e0 + (uint32_t)(h + i) * de;
          if (e < n_in) raw[i] = src[e];  // elements n_in .. N - 1 are the zero padding
          else raw[i] = make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i)
          xc[33 * (h + i)] = make_float2((float)raw[i].x, (float)raw[i].y);
      }
    } else {
      const float2* src = reinterpret_cast<const float2*>(in) + (size_t)blockIdx.y * n_in;
      float2 raw[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const uint32_t e = e0 + (uint32_t)i * de;
        raw[i] = e < n_in ? src[e] : make_float2(0.0f, 0.0f);
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) xc[33 * i] = raw[i];
    }
  }
  __syncthreads();
  float2* xw = X + w * kW32Stride;
  float2 a[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) a[m] = xw[33 * m + lane];
  if (Ns > 1) {
#pragma unroll
    for (int m = 0; m < 32; ++m) a[m] = cmul(a[m], cmul(At, BM[w * 32 + m]));
  }
  dft32(a, sg);  // a[ka] = sum_m a_{t + 32 m} w_32^{m ka}
#pragma unroll
  for (int ka = 1; ka < 32; ++ka) a[ka] = cmul(a[ka], TW[ka * 32 + lane]);
  __syncwarp();  // every lane's stage-A reads are done
#pragma unroll
  for (int ka = 0; ka < 32; ++ka) xw[33 * ka + lane] = a[ka];
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 32; ++t) a[t] = xw[33 * lane + t];
  dft32(a, sg);  // a[kb] = A_{lane + 32 kb}
  const size_t so = (size_t)blockIdx.y * n_out;
  if (Ns == 1) {  // out[j R + r']: 32 consecutive elements per kb
    const uint32_t base = (j << 10) + lane;
    if (out_f64) {
      double2* o = reinterpret_cast<double2*>(out) + so;
#pragma unroll
      for (int kb = 0; kb < 32; ++kb)
        if (base + 32u * kb < n_out) o[base + 32u * kb] = make_double2(a[kb].x, a[kb].y);
    } else {
      float2* o = reinterpret_cast<float2*>(out) + so;
#pragma unroll
      for (int kb = 0; kb < 32; ++kb)
        if (base + 32u * kb < n_out) o[base + 32u * kb] = a[kb];
    }
    return;
  }
  // out[(j / Ns) Ns R + jm + r' Ns]: rows of the four adjacent columns
  __syncwarp();
#pragma unroll
  for (int kb = 0; kb < 32; ++kb) xw[33 * kb + lane] = a[kb];
  __syncthreads();
  const float2* xc = X + c4 * kW32Stride + q4;
  const uint32_t base = ((j0 >> logNs) << (logNs + 10)) + (j0 & (Ns - 1)) + c4 + q4 * Ns;
  const uint32_t ds = 32u * Ns;
  if (out_f64) {
    double2* o = reinterpret_cast<double2*>(out) + so;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float2 v = xc[33 * i];
      if (base + i * ds < n_out) o[base + i * ds] = make_double2(v.x, v.y);
    }
  } else {
    float2* o = reinterpret_cast<float2*>(out) + so;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (base + i * ds < n_out) o[base + i * ds] = xc[33 * i];
  }
}

__global__ void k_tw_to_float(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

}  // namespace nufft

using namespace nufft;

int fft_lo_bits(int64_t N) {
  int L = 0;
  while ((int64_t(1) << L) < N) ++L;
  return (L + 1) / 2;
}

// entries of the two-level tables of w_N (the radix-1024 table follows them)
static size_t fft_table_base(int64_t N) {
  int b = fft_lo_bits(N);
  return (size_t)(int64_t(1) << b) + (size_t)(N >> b);
}

size_t fft_table_elems(int64_t N) { return fft_table_base(N) + 1024; }

// tw: double2 tables, twf: float2 copy (may be null)
int fft_init_tables(double2* tw, float2* twf, int64_t N, cudaStream_t st) {
  int b = fft_lo_bits(N);
  int64_t n = (int64_t)fft_table_elems(N);
  k_fft_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tw, N, b);
  if (twf) k_tw_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tw, twf, n);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// Split L into the fewest passes of at most 10 bits: as evenly as possible,
// or (radix10) 10-bit passes first and the remainder last, for the
// one-warp-per-column radix-1024 pass.
static int fft_plan_passes(int L, int* logR, bool radix10 = false) {
  int np = (L + 9) / 10;
  if (np == 0) np = 1;
  if (radix10 && L > 10) {
    for (int i = 0; i < np - 1; ++i) logR[i] = 10;
    logR[np - 1] = L - 10 * (np - 1);
    return np;
  }
  int base = L / np, extra = L % np;
  for (int i = 0; i < np; ++i) logR[i] = base + (i < extra ? 1 : 0);
  return np;
}

int fft_num_passes(int64_t N) {
  int L = 0;
  while ((int64_t(1) << L) < N) ++L;
  int logR[8];
  return fft_plan_passes(L, logR);
}

template <class T, int LR>
static void fft_launch(dim3 grid, int threads, size_t smem, cudaStream_t st, uint32_t n_in,
                       uint32_t n_out, const void* in,
                       int in_f64, void* out, int out_f64, int logN, int logNs, int J, int logJ,
                       int sign, const cplx<T>* tw, int lo_bits) {
  constexpr int JMAX = FftShape<T, LR>::JMAX;
  constexpr int JHALF = JMAX > 1 ? JMAX / 2 : JMAX;
  if (J == JMAX)
    launch_pdl(k_fft_st<T, LR, JMAX>, grid, threads, smem, st, in, in_f64, out, out_f64, logN,
               logNs, J, logJ, sign, tw, lo_bits, n_in, n_out);
  else if (J == JHALF)
    launch_pdl(k_fft_st<T, LR, JHALF>, grid, threads, smem, st, in, in_f64, out, out_f64, logN,
               logNs, J, logJ, sign, tw, lo_bits, n_in, n_out);
  else
    launch_pdl(k_fft_st<T, LR, 0>, grid, threads, smem, st, in, in_f64, out, out_f64, logN, logNs,
               J, logJ, sign, tw, lo_bits, n_in, n_out);
}

// the pass kernel for logR
template <class T>
static int fft_pass(int logR, dim3 grid, int threads, size_t smem, cudaStream_t st,
                    uint32_t n_in, uint32_t n_out, const void* in, int in_f64, void* out,
                    int out_f64, int logN, int logNs, int J, int logJ, int sign,
                    const cplx<T>* tw, int lo_bits) {
#define NUFFT_FFT_CASE(LR)                                                                  \
  case LR:                                                                                 \
    fft_launch<T, LR>(grid, threads, smem, st, n_in, n_out, in, in_f64, out, out_f64, logN, \
                      logNs, J, logJ, sign, tw, lo_bits);                                  \
    return NUFFT_OK;
  switch (logR) {
    NUFFT_FFT_CASE(1)
    NUFFT_FFT_CASE(2)
    NUFFT_FFT_CASE(3)
    NUFFT_FFT_CASE(4)
    NUFFT_FFT_CASE(5)
    NUFFT_FFT_CASE(6)
    NUFFT_FFT_CASE(7)
    NUFFT_FFT_CASE(8)
    NUFFT_FFT_CASE(9)
    NUFFT_FFT_CASE(10)
    default: return NUFFT_EINVAL;
  }
#undef NUFFT_FFT_CASE
}

static int g_fft_sms = 0;

// Columns per CTA of the radix-1024 pass: the widest of 16, 8, 4 (longest
// row runs) that still gives about one CTA per SM (at least 4/5 of the SMs)
// over the grid: measured at 2^20 (8: 14.4 us per transform, 4: 15.0, 16:
// 23.3), 2^21 (16: 29.8, 4: 31.3) and 2^24 (16: 276, 4: 292);
// NUFFT_FFT_W32_COLS (4, 8 or 16) fixes it, for measurements.
constexpr int kW32MinCols = 4;
static int w32_cols(int64_t NR, int64_t Ns, int batch, int64_t nsm) {
  static const int forced = [] {
    const char* e = std::getenv("NUFFT_FFT_W32_COLS");
    const int x = e ? std::atoi(e) : 0;
    return (x == 4 || x == 8 || x == 16) ? x : 0;
  }();
  int c = forced ? forced : 16;
  while (!forced && c > kW32MinCols && 5 * (NR / c) * batch < 4 * nsm) c >>= 1;
  while (c > kW32MinCols && (NR < c || (Ns > 1 && Ns < c))) c >>= 1;
  return c;
}

// The one-warp-per-column radix-1024 pass (FP32) where it applies;
// NUFFT_FFT_NO_W32=1 keeps every pass on k_fft_st, for measurements.
static bool fft_w32_enabled() {
  static const bool v = [] {
    const char* e = std::getenv("NUFFT_FFT_NO_W32");
    return !(e && std::atoi(e) == 1);
  }();
  return v;
}

// Fewest columns per CTA the pass planner goes down to when the grid of
// CTAs is small (4: every strided row is a full 32-byte sector of complex64);
// NUFFT_FFT_MIN_COLS (1, 2, 4 or 8) overrides it for measurements.
static int fft_min_cols() {
  static const int v = [] {
    const char* e = std::getenv("NUFFT_FFT_MIN_COLS");
    const int x = e ? std::atoi(e) : 4;
    return (x == 1 || x == 2 || x == 4 || x == 8) ? x : 4;
  }();
  return v;
}

// out = FFT(in) in arithmetic T for `batch` signals of N elements each
// (signal-major); in / out are complex128 (f64 = 1) or complex64.  Intermediate passes alternate between the scratch vectors buf
// and buf2 (batch x N cplx<T> each; buf2 is used only with three or more passes), so
// they keep T precision and never touch `out`.  `in` is only read.  in holds
// n_in <= N elements per signal, zero padded to N (the first pass reads
// nothing beyond n_in), and out keeps the first n_out <= N of the N outputs
// (signal strides n_in and n_out); 0 = N.
template <class T>
int fft_run(const void* in, int in_f64, void* out, int out_f64, cplx<T>* buf, cplx<T>* buf2,
            int64_t N, int batch, int sign, const cplx<T>* tw, cudaStream_t st, int64_t n_in,
            int64_t n_out) {
  if (n_in <= 0) n_in = N;
  if (n_out <= 0) n_out = N;
  if (n_in > N || n_out > N) return NUFFT_EINVAL;
  int L = 0;
  while ((int64_t(1) << L) < N) ++L;
  const int tf64 = sizeof(T) == 8;
  const int64_t nsm = g_fft_sms > 0 ? g_fft_sms : 152;
  // the radix-1024 pass where its grid (four columns per CTA) fills every SM
  const bool w32 = !tf64 && fft_w32_enabled() && L >= 12 &&
                   ((int64_t(1) << (L - 10)) / kW32MinCols) * batch >= nsm;
  int logR[8];
  int np = fft_plan_passes(L, logR, w32);
  if (np >= 3 && !buf2) return NUFFT_EINVAL;
  int b = fft_lo_bits(N);
  const void* src = in;
  int src_f64 = in_f64;
  int64_t Ns = 1;
  const int64_t target = 2 * nsm;
  for (int i = 0; i < np; ++i) {
    bool last = (i == np - 1);
    void* dst = last ? out : (void*)((i & 1) ? buf2 : buf);
    int dst_f64 = last ? out_f64 : tf64;
    const int lr = logR[i];
    const int R = 1 << lr, TPC = R >= 8 ? R / 8 : 1;
    const int64_t NR = N >> lr;
    const uint32_t pin = (uint32_t)(i == 0 ? n_in : N), pout = (uint32_t)(last ? n_out : N);
    if (w32 && lr == 10 && NR >= kW32MinCols && (Ns == 1 || Ns >= kW32MinCols)) {
      int logNs = 0;
      while ((int64_t(1) << logNs) < Ns) ++logNs;
      const int cols = w32_cols(NR, Ns, batch, nsm);
      const float2* twf = reinterpret_cast<const float2*>(tw);
      const float2* tw32 = twf + fft_table_base(N);
      const dim3 grid((unsigned)(NR / cols), (unsigned)batch);
      if (cols == 16)
        launch_pdl(k_fft_w32<16>, grid, W32Shape<16>::threads, W32Shape<16>::smem, st, src,
                   src_f64, dst, dst_f64, L, logNs, sign, twf, tw32, b, pin, pout);
      else if (cols == 8)
        launch_pdl(k_fft_w32<8>, grid, W32Shape<8>::threads, W32Shape<8>::smem, st, src,
                   src_f64, dst, dst_f64, L, logNs, sign, twf, tw32, b, pin, pout);
      else
        launch_pdl(k_fft_w32<4>, grid, W32Shape<4>::threads, W32Shape<4>::smem, st, src,
                   src_f64, dst, dst_f64, L, logNs, sign, twf, tw32, b, pin, pout);
      src = dst;
      src_f64 = dst_f64;
      Ns <<= lr;
      continue;
    }
    // columns per CTA: at most kFftMaxThreads threads and kFftSmemElems
    // elements, at least fft_min_cols() (contiguous runs), fewer while the
    // grid is small
    int J = kFftMaxThreads / TPC;
    while (J > 1 && (int64_t)R * J > kFftSmemElems) J >>= 1;
    while (J > fft_min_cols() && (NR / J) * batch < target) J >>= 1;
    if (J > NR) J = (int)NR;
    int logJ = 0;
    while ((1 << logJ) < J) ++logJ;
    const size_t nbuf = sizeof(T) == 4 ? 2 : 1;
    const size_t smem =
        ((size_t)R + nbuf * ((size_t)R * J + (size_t)R * J / 32 + 1)) * sizeof(cplx<T>);
    unsigned grid = (unsigned)(NR / J);
    int logNs = 0;
    while ((int64_t(1) << logNs) < Ns) ++logNs;
    int rc = fft_pass<T>(lr, dim3(grid, (unsigned)batch), J * TPC, smem, st, pin, pout, src,
                         src_f64, dst, dst_f64, L, logNs, J, logJ, sign, tw, b);
    if (rc) return rc;
    src = dst;
    src_f64 = dst_f64;
    Ns <<= lr;
  }
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template <class T, int LR>
static int fft_attr() {
  const int nbuf = sizeof(T) == 4 ? 2 : 1;
  const int big =
      (int)((1024 + nbuf * (kFftSmemElems + kFftSmemElems / 32 + 1)) * sizeof(cplx<T>));
  constexpr int JMAX = FftShape<T, LR>::JMAX;
  constexpr int JHALF = JMAX > 1 ? JMAX / 2 : JMAX;
  return cudaFuncSetAttribute(k_fft_st<T, LR, JMAX>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, big) == cudaSuccess &&
                 cudaFuncSetAttribute(k_fft_st<T, LR, JHALF>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      big) == cudaSuccess &&
                 cudaFuncSetAttribute(k_fft_st<T, LR, 0>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      big) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}

template <class T>
static int fft_attrs() {
  int rc = fft_attr<T, 1>();
  if (!rc) rc = fft_attr<T, 2>();
  if (!rc) rc = fft_attr<T, 3>();
  if (!rc) rc = fft_attr<T, 4>();
  if (!rc) rc = fft_attr<T, 5>();
  if (!rc) rc = fft_attr<T, 6>();
  if (!rc) rc = fft_attr<T, 7>();
  if (!rc) rc = fft_attr<T, 8>();
  if (!rc) rc = fft_attr<T, 9>();
  if (!rc) rc = fft_attr<T, 10>();
  return rc;
}

int fft_configure() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&g_fft_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NUFFT_ECUDA;
  int rc = fft_attrs<double>();
  if (!rc) rc = fft_attrs<float>();
  if (!rc && (cudaFuncSetAttribute(k_fft_w32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)W32Shape<8>::smem) != cudaSuccess ||
              cudaFuncSetAttribute(k_fft_w32<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)W32Shape<16>::smem) != cudaSuccess))
    rc = NUFFT_ECUDA;
  return rc;
}

template int fft_run<double>(const void*, int, void*, int, double2*, double2*, int64_t, int, int,
                             const double2*, cudaStream_t, int64_t, int64_t);
template int fft_run<float>(const void*, int, void*, int, float2*, float2*, int64_t, int, int,
                            const float2*, cudaStream_t, int64_t, int64_t);
