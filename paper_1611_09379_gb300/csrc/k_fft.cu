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
#include "common.cuh"

namespace nufft {

constexpr int kFftSmemElems = 4096;  // R * J complex elements staged per CTA

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
  if (f64) {
    double2 v = reinterpret_cast<const double2*>(p)[i];
    return mk<T>((T)v.x, (T)v.y);
  }
  float2 v = reinterpret_cast<const float2*>(p)[i];
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ inline void store_c(void* p, int64_t i, int f64, cplx<T> v) {
  if (f64) reinterpret_cast<double2*>(p)[i] = make_double2((double)v.x, (double)v.y);
  else reinterpret_cast<float2*>(p)[i] = make_float2((float)v.x, (float)v.y);
}

template <class T>
__global__ void __launch_bounds__(256) k_fft_pass(const void* __restrict__ in, int in_f64,
                                                  void* __restrict__ out, int out_f64, int64_t N,
                                                  int logR, int64_t Ns, int J, int sign,
                                                  const cplx<T>* __restrict__ tw, int lo_bits) {
  extern __shared__ unsigned char smraw[];
  cplx<T>* sm = reinterpret_cast<cplx<T>*>(smraw);     // [R][J]
  const int R = 1 << logR;
  cplx<T>* twR = sm + R * J;                           // [R/2] e^{sign 2 pi i m / R}
  const int64_t NR = N >> logR;
  const int64_t j0 = (int64_t)blockIdx.x * J;
  const int nth = blockDim.x;
  // signal blockIdx.y of a batch: vectors at stride N elements
  in = (const char*)in + (size_t)blockIdx.y * N * (in_f64 ? 16 : 8);
  out = (char*)out + (size_t)blockIdx.y * N * (out_f64 ? 16 : 8);

  for (int m = threadIdx.x; m < R / 2; m += nth)
    twR[m] = twiddle_t<T>(tw, (int64_t)m * (N >> logR), lo_bits, sign);

  // load with pass twiddle into bit-reversed position
  const int64_t tstep = N / (Ns << logR);
  for (int e = threadIdx.x; e < R * J; e += nth) {
    int r = e / J, jj = e - r * J;
    int64_t j = j0 + jj;
    cplx<T> v = load_c<T>(in, j + (int64_t)r * NR, in_f64);
    int64_t jm = j & (Ns - 1);
    if (jm != 0 && r != 0) {
      // w^{r jm / (Ns R)} = e^{2 pi i m / N} with m = r jm (N / (Ns R))
      int64_t m = ((int64_t)r * jm) * tstep;
      v = cmul(v, twiddle_t<T>(tw, m & (N - 1), lo_bits, sign));
    }
    int rb = logR ? (int)(__brev((unsigned)r) >> (32 - logR)) : 0;
    sm[rb * J + jj] = v;
  }
  __syncthreads();
  // radix-2 decimation-in-time butterflies
  for (int h = 1; h < R; h <<= 1) {
    int stride = R / (2 * h);
    for (int e = threadIdx.x; e < (R / 2) * J; e += nth) {
      int bf = e / J, jj = e - bf * J;
      int grp = bf / h, pos = bf - grp * h;
      int i0 = grp * 2 * h + pos, i1 = i0 + h;
      cplx<T> w = twR[pos * stride];
      cplx<T> a = sm[i0 * J + jj], b = cmul(sm[i1 * J + jj], w);
      sm[i0 * J + jj] = cadd(a, b);
      sm[i1 * J + jj] = csub(a, b);
    }
    __syncthreads();
  }
  // store: out[(j/Ns) Ns R + j%Ns + r Ns]
  for (int e = threadIdx.x; e < R * J; e += nth) {
    int r, jj;
    if (Ns >= J) { r = e / J; jj = e - r * J; }   // J contiguous per r
    else { jj = e / R; r = e - jj * R; }          // small Ns: R contiguous per j
    int64_t j = j0 + jj;
    int64_t jm = j & (Ns - 1);
    int64_t dst = (j / Ns) * Ns * R + jm + (int64_t)r * Ns;
    store_c<T>(out, dst, out_f64, sm[r * J + jj]);
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
  for (int i = 0; i < np; ++i) {
    bool last = (i == np - 1);
    void* dst = last ? out : (void*)((i & 1) ? buf2 : buf);
    int dst_f64 = last ? out_f64 : tf64;
    int R = 1 << logR[i];
    int J = kFftSmemElems / R;
    if (J > (int)(N >> logR[i])) J = (int)(N >> logR[i]);
    if (J < 1) J = 1;
    size_t smem = (size_t)(R * J + R / 2) * sizeof(cplx<T>);
    unsigned grid = (unsigned)((N >> logR[i]) / J);
    k_fft_pass<T><<<dim3(grid, (unsigned)batch), 256, smem, st>>>(src, src_f64, dst, dst_f64, N,
                                                                  logR[i], Ns, J, sign, tw, b);
    src = dst;
    src_f64 = dst_f64;
    Ns <<= logR[i];
  }
  return cudaGetLastError() == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int fft_configure() {
  size_t big = (size_t)(kFftSmemElems + 512) * sizeof(double2);
  if (cudaFuncSetAttribute(k_fft_pass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)big) != cudaSuccess)
    return NUFFT_ECUDA;
  if (cudaFuncSetAttribute(k_fft_pass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)big) != cudaSuccess)
    return NUFFT_ECUDA;
  return NUFFT_OK;
}

template int fft_run<double>(const void*, int, void*, int, double2*, double2*, int64_t, int, int,
                             const double2*, cudaStream_t);
template int fft_run<float>(const void*, int, void*, int, float2*, float2*, int64_t, int, int,
                            const float2*, cudaStream_t);
