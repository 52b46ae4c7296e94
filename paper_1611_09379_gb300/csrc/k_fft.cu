// Stockham auto-sort FFT for the c_n <-> f_k step (Eq. p1, Sec. 2):
//   out_n = sum_k in_k e^{sign 2 pi i n k / N},  N = 2^L, no scaling.
// Each pass is one radix-R Stockham iteration,
//   a_r = in[j + r N/R] * w^{sign r (j mod Ns) / (Ns R)},  A = DFT_R(a),
//   out[(j/Ns) Ns R + (j mod Ns) + r' Ns] = A_r',
// with the size-R DFT done in shared memory by a CTA for J adjacent j (so
// the strided global reads and writes move J contiguous elements).  Passes
// multiply Ns by R until it reaches N.  Twiddles come from two small tables,
// w^{m/N} = T_hi[m >> b] * T_lo[m & (2^b - 1)], filled once per plan with
// sincospi of exact arguments.
#include <cstdint>

#include "common.cuh"

namespace nufft {

constexpr int kFftSmemElems = 4096;  // R * J complex elements staged per CTA (at most)

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
  }
}

// e^{sign 2 pi i m / N}, 0 <= m < N, from the two tables
template <class T>
__device__ inline cplx<T> twiddle_t(const cplx<T>* __restrict__ tw, int64_t m, int lo_bits,
                                    int sign) {
  int64_t nlo = int64_t(1) << lo_bits;
  cplx<T> a = tw[m & (nlo - 1)], b = tw[nlo + (m >> lo_bits)];
  cplx<T> r = cmul(a, b);
  if (sign < 0) r.y = -r.y;
  return r;
}

// in / out element type chosen at run time (uniform branch): complex128 when
// *_f64 != 0, complex64 otherwise; arithmetic in T.
template <class T>
__device__ inline cplx<T> load_c(const void* p, int64_t i, int f64) {
  if (f64) return c128_to<T>(reinterpret_cast<const double2*>(p)[i]);
  float2 v = reinterpret_cast<const float2*>(p)[i];
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ inline void store_c(void* p, int64_t i, int f64, cplx<T> v) {
  if (f64) reinterpret_cast<double2*>(p)[i] = to_c128(v);
  else reinterpret_cast<float2*>(p)[i] = make_float2((float)v.x, (float)v.y);
}

// Size-S DFT of v[0..S) in registers (S = 2^LOGS <= 32), radix-2
// decimation in time: v holds the input in bit-reversed order and receives
// the output in natural order.  Twiddles w_S^e = wR[e * (R / S)] from the
// pass's table in shared memory (broadcast reads).
template <class T, int LOGS>
__device__ inline void dft_reg(cplx<T>* v, const cplx<T>* __restrict__ wR, int rs) {
  constexpr int S = 1 << LOGS;
#pragma unroll
  for (int h = 1; h < S; h <<= 1) {
#pragma unroll
    for (int grp = 0; grp < S; grp += 2 * h) {
#pragma unroll
      for (int pos = 0; pos < h; ++pos) {
        cplx<T> a = v[grp + pos], bb = v[grp + pos + h];
        if (pos != 0) bb = cmul(bb, wR[pos * (S / (2 * h)) * rs]);
        v[grp + pos] = cadd(a, bb);
        v[grp + pos + h] = csub(a, bb);
      }
    }
  }
}

template <int LOG> __device__ constexpr int brev_c(int x) {
  int r = 0;
  for (int i = 0; i < LOG; ++i) r |= ((x >> i) & 1) << (LOG - 1 - i);
  return r;
}

// One radix-R Stockham pass, R = R1 R2 (R1 = 2^LOG1 >= R2 = 2^LOG2), for J
// columns j per CTA (blockDim = J R2 threads; thread (c, t) = (tid mod J,
// tid / J)).  Column j transforms a_r = in[j + r N/R] w^{sign r (j mod Ns) /
// (Ns R)}, r = t + R2 m, as
//   X[k1 + R1 k2] = sum_t w_R2^{t k2} w_R^{t k1} sum_m a[t + R2 m] w_R1^{m k1}:
// thread t does the inner size-R1 DFT over m in registers, multiplies by
// w_R^{t k1} and writes Y[k1][t] to shared memory; then thread u does the
// size-R2 DFTs over t for k1 = u, u + R2, ...; the result goes back through
// shared memory to out[(j / Ns) Ns R + (j mod Ns) + r' Ns] with contiguous
// runs (J per r' for Ns >= J, else R per j).
__device__ inline void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

template <class T, int LOG1, int LOG2>
__global__ void __launch_bounds__(256) k_fft_reg(const void* __restrict__ in, int in_f64,
                                                 void* __restrict__ out, int out_f64, int64_t N,
                                                 int64_t Ns, int J, int logJ, int sign,
                                                 const cplx<T>* __restrict__ tw, int lo_bits,
                                                 int staged) {
  constexpr int R1 = 1 << LOG1, R2 = 1 << LOG2, R = R1 * R2, LOGR = LOG1 + LOG2;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<T>* wR = reinterpret_cast<cplx<T>*>(smraw);  // [R] w_R^e
  cplx<T>* S = wR + R;                              // [R][J] (Y[k1][t] / X[r'] by column)
  const int64_t NR = N >> LOGR;
  const int64_t j0 = (int64_t)blockIdx.x * J;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int esz = in_f64 ? 16 : 8;
  in = (const char*)in + (size_t)blockIdx.y * N * esz;
  out = (char*)out + (size_t)blockIdx.y * N * (out_f64 ? 16 : 8);
  // staged: the tile's R rows of J contiguous inputs go to shared memory by
  // 16-byte asynchronous copies (the whole tile in flight at once); the
  // region holds R J inputs of esz bytes, reused for Y / X afterwards
  const int lpr = (J * esz) >> 4;  // 16-byte pieces per row (power of two)
  if (staged) {
    int lg = 0;
    while ((1 << lg) < lpr) ++lg;
    const char* src = (const char*)in + j0 * esz;
    char* dstb = reinterpret_cast<char*>(S);
    for (int e = tid; e < R * lpr; e += nth) {
      const int r = e >> lg, pc = e & (lpr - 1);
      cp_async16(dstb + ((size_t)r * J * esz + pc * 16), src + ((size_t)r * NR * esz + pc * 16));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int e = tid; e < R; e += nth) wR[e] = twiddle_t<T>(tw, (int64_t)e * NR, lo_bits, sign);
  const int c = tid & (J - 1), t = tid >> logJ;
  const int64_t j = j0 + c;
  const int64_t jm = j & (Ns - 1);
  int logNs = 0;
  while ((int64_t(1) << logNs) < Ns) ++logNs;
  int logN = 0;
  while ((int64_t(1) << logN) < N) ++logN;
  const int lstep = logN - logNs - LOGR;  // tstep = N / (Ns R) = 2^lstep
  if (staged) asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();  // wR and the staged tile ready
  // load (columns fastest: J contiguous elements per r) with the pass twiddle
  cplx<T> v[R1];
#pragma unroll
  for (int m = 0; m < R1; ++m) {
    const int r = t + R2 * m;
    cplx<T> x = staged ? load_c<T>(S, (int64_t)r * J + c, in_f64)
                       : load_c<T>(in, j + (int64_t)r * NR, in_f64);
    if (jm != 0 && r != 0) x = cmul(x, twiddle_t<T>(tw, (((int64_t)r * jm) << lstep) & (N - 1), lo_bits, sign));
    v[brev_c<LOG1>(m)] = x;
  }
  __syncthreads();  // all staged inputs read before S is reused
  dft_reg<T, LOG1>(v, wR, R / R1);
  // Y[k1][t] = v[k1] w_R^{t k1}
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cplx<T> y = v[k1];
    if (LOG2 > 0 && k1 != 0 && t != 0) y = cmul(y, wR[(t * k1) & (R - 1)]);
    S[(k1 * R2 + t) * J + c] = y;
  }
  __syncthreads();
  if (LOG2 > 0) {
    // thread u = t: size-R2 DFTs over t for k1 = u + R2 i, i < R1 / R2
#pragma unroll
    for (int i = 0; i < R1 / R2; ++i) {
      const int k1 = t + R2 * i;
      cplx<T> w[R2];
#pragma unroll
      for (int tt = 0; tt < R2; ++tt) w[brev_c<LOG2>(tt)] = S[(k1 * R2 + tt) * J + c];
      dft_reg<T, LOG2>(w, wR, R / R2);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[i * R2 + k2] = w[k2];
    }
    __syncthreads();  // all reads of Y done
#pragma unroll
    for (int i = 0; i < R1 / R2; ++i) {
      const int k1 = t + R2 * i;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) S[(k1 + R1 * k2) * J + c] = v[i * R2 + k2];
    }
    __syncthreads();
  }
  // S[r'][c] = X_{r'} of column c -> out
  for (int e = tid; e < R * J; e += nth) {
    int r, jj;
    if (Ns >= J) { r = e >> logJ; jj = e & (J - 1); }  // J contiguous per r
    else { jj = e >> LOGR; r = e & (R - 1); }           // small Ns: R contiguous per j
    const int64_t jg = j0 + jj;
    const int64_t jmg = jg & (Ns - 1);
    const int64_t dst = ((jg >> logNs) << (logNs + LOGR)) + jmg + ((int64_t)r << logNs);
    store_c<T>(out, dst, out_f64, S[r * J + jj]);
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

size_t fft_table_elems(int64_t N) {
  int b = fft_lo_bits(N);
  return (size_t)(int64_t(1) << b) + (size_t)(N >> b);
}

// tw: double2 tables, twf: float2 copy (may be null)
int fft_init_tables(double2* tw, float2* twf, int64_t N, cudaStream_t st) {
  int b = fft_lo_bits(N);
  int64_t n = (int64_t(1) << b) + (N >> b);
  k_fft_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tw, N, b);
  if (twf) k_tw_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tw, twf, n);
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

// Split L into passes of at most 10 bits, as evenly as possible.
static int fft_plan_passes(int L, int* logR) {
  int np = (L + 9) / 10;
  if (np == 0) np = 1;
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

// out = FFT(in) in arithmetic T for `batch` signals of N elements each
// (signal-major); in / out are complex128 (f64 = 1) or complex64.  Intermediate passes alternate between the scratch vectors buf
// and buf2 (batch x N cplx<T> each; buf2 is used only with three or more passes), so
// they keep T precision and never touch `out`.  `in` is only read.
using FftKernel = void (*)(const void*, int, void*, int, int64_t, int64_t, int, int, int,
                          const void*, int);

template <class T, int LOG1, int LOG2>
static void fft_launch(dim3 grid, int threads, size_t smem, cudaStream_t st, const void* in,
                       int in_f64, void* out, int out_f64, int64_t N, int64_t Ns, int J, int logJ,
                       int sign, const cplx<T>* tw, int lo_bits, int staged) {
  k_fft_reg<T, LOG1, LOG2><<<grid, threads, smem, st>>>(in, in_f64, out, out_f64, N, Ns, J, logJ,
                                                         sign, tw, lo_bits, staged);
}

// the pass kernel for logR = LOG1 + LOG2 (LOG1 = ceil(logR / 2))
template <class T>
static int fft_pass(int logR, dim3 grid, int threads, size_t smem, cudaStream_t st,
                    const void* in, int in_f64, void* out, int out_f64, int64_t N, int64_t Ns,
                    int J, int logJ, int sign, const cplx<T>* tw, int lo_bits, int staged) {
#define NUFFT_FFT_CASE(L1, L2)                                                                 \
  case L1 + L2:                                                                                \
    fft_launch<T, L1, L2>(grid, threads, smem, st, in, in_f64, out, out_f64, N, Ns, J, logJ, \
                          sign, tw, lo_bits, staged);                                          \
    return NUFFT_OK;
  switch (logR) {
    NUFFT_FFT_CASE(1, 0)
    NUFFT_FFT_CASE(1, 1)
    NUFFT_FFT_CASE(2, 1)
    NUFFT_FFT_CASE(2, 2)
    NUFFT_FFT_CASE(3, 2)
    NUFFT_FFT_CASE(3, 3)
    NUFFT_FFT_CASE(4, 3)
    NUFFT_FFT_CASE(4, 4)
    NUFFT_FFT_CASE(5, 4)
    NUFFT_FFT_CASE(5, 5)
    default: return NUFFT_EINVAL;
  }
#undef NUFFT_FFT_CASE
}

static int g_fft_sms = 0;

// out = FFT(in) in arithmetic T for `batch` signals of N elements each
// (signal-major); in / out are complex128 (f64 = 1) or complex64.  Intermediate passes alternate between the scratch vectors buf
// and buf2 (batch x N cplx<T> each; buf2 is used only with three or more passes), so
// they keep T precision and never touch `out`.  `in` is only read.
template <class T>
int fft_run(const void* in, int in_f64, void* out, int out_f64, cplx<T>* buf, cplx<T>* buf2,
            int64_t N, int batch, int sign, const cplx<T>* tw, cudaStream_t st) {
  int L = 0;
  while ((int64_t(1) << L) < N) ++L;
  int logR[8];
  int np = fft_plan_passes(L, logR);
  if (np >= 3 && !buf2) return NUFFT_EINVAL;
  int b = fft_lo_bits(N);
  const int tf64 = sizeof(T) == 8;
  const void* src = in;
  int src_f64 = in_f64;
  int64_t Ns = 1;
  const int64_t target = 2 * (int64_t)(g_fft_sms > 0 ? g_fft_sms : 152);
  for (int i = 0; i < np; ++i) {
    bool last = (i == np - 1);
    void* dst = last ? out : (void*)((i & 1) ? buf2 : buf);
    int dst_f64 = last ? out_f64 : tf64;
    const int lr = logR[i];
    const int R = 1 << lr, R2 = 1 << (lr / 2);
    const int64_t NR = N >> lr;
    // columns per CTA: at most 256 threads and kFftSmemElems staged
    // elements, at least 4 (contiguous runs), fewer while the grid is small
    int J = 256 / R2;
    while (J > 1 && (int64_t)R * J > kFftSmemElems) J >>= 1;
    while (J > 4 && (NR / J) * batch < target) J >>= 1;
    if (J > NR) J = (int)NR;
    int logJ = 0;
    while ((1 << logJ) < J) ++logJ;
    // staged input: 16-byte aligned rows of at least 16 bytes
    const size_t esz = src_f64 ? 16 : 8;
    const int staged = ((uintptr_t)src % 16 == 0) && (J * esz >= 16);
    const size_t elem = staged && esz > sizeof(cplx<T>) ? esz : sizeof(cplx<T>);
    size_t smem = (size_t)R * sizeof(cplx<T>) + (size_t)R * J * elem;
    unsigned grid = (unsigned)(NR / J);
    int rc = fft_pass<T>(lr, dim3(grid, (unsigned)batch), J * R2, smem, st, src, src_f64, dst,
                         dst_f64, N, Ns, J, logJ, sign, tw, b, staged);
    if (rc) return rc;
    src = dst;
    src_f64 = dst_f64;
    Ns <<= lr;
  }
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

template <class T, int LOG1, int LOG2>
static int fft_attr() {
  const int big = (int)(kFftSmemElems * 16 + 1024 * sizeof(cplx<T>));
  return cudaFuncSetAttribute(k_fft_reg<T, LOG1, LOG2>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, big) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}

template <class T>
static int fft_attrs() {
  int rc = fft_attr<T, 1, 0>();
  if (!rc) rc = fft_attr<T, 1, 1>();
  if (!rc) rc = fft_attr<T, 2, 1>();
  if (!rc) rc = fft_attr<T, 2, 2>();
  if (!rc) rc = fft_attr<T, 3, 2>();
  if (!rc) rc = fft_attr<T, 3, 3>();
  if (!rc) rc = fft_attr<T, 4, 3>();
  if (!rc) rc = fft_attr<T, 4, 4>();
  if (!rc) rc = fft_attr<T, 5, 4>();
  if (!rc) rc = fft_attr<T, 5, 5>();
  return rc;
}

int fft_configure() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&g_fft_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return NUFFT_ECUDA;
  int rc = fft_attrs<double>();
  if (!rc) rc = fft_attrs<float>();
  return rc;
}

template int fft_run<double>(const void*, int, void*, int, double2*, double2*, int64_t, int, int,
                             const double2*, cudaStream_t);
template int fft_run<float>(const void*, int, void*, int, float2*, float2*, int64_t, int, int,
                            const float2*, cudaStream_t);
