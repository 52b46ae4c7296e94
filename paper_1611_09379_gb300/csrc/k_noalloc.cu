// Forward NUFFT that allocates no memory: nufft_fwd_noalloc.
//
// Some callers cannot allocate device memory at the point where they want a
// transform: applications whose device memory is owned by a pool allocator or
// a fixed budget (a raw cudaMalloc would bypass or exceed it), and
// latency-critical loops in which cudaMalloc / cudaFree, which may synchronise
// the device, are not acceptable.  For them this entry point runs the same
// binning, FFT, FMM and target kernels as nufft_fwd, but every workspace
// buffer is carved from one file-scope device array of fixed size,
// g_noalloc_scratch (16 MiB), which every GPU that loads the library holds
// until the process exits.
//
// The array's name is only a host-side stand-in in host code, so the first
// call on each device (with that device current) looks up its device address
// with cudaGetSymbolAddress and keeps it; that first call should come before
// any stream capture.  All calls share the array: a call overwrites the
// previous call's contents (what must start at zero is cleared each time),
// and calls whose GPU work overlaps race on it.  Host-side calls are
// serialised by a mutex; the operator tables are staged in static host
// arrays, so no host allocation happens either.
#include <cmath>
#include <mutex>

#include "common.cuh"

using namespace nufft;

int plan_configure();
void make_operator_tables(const nufft_plan_s* pl, long double* m2m, long double* m2l,
                          long double* l2l, long double* rp, double* reg);
size_t setup_tmp_bytes(int64_t M, int64_t B);
int setup_points(nufft_plan_s* pl, const double* y, void* tmp);
int fmm_pack_positions(nufft_plan_s* pl);
int fft_init_tables(double2* tw, float2* twf, int64_t N, cudaStream_t st);
size_t fft_table_elems(int64_t N);
int fft_num_passes(int64_t N);

namespace {
constexpr size_t kNoAllocBytes = size_t(16) << 20;  // fixed scratch per device
constexpr int64_t kNoAllocMaxN = int64_t(1) << 16;  // largest N and M accepted
constexpr int64_t kNoAllocMaxM = int64_t(1) << 16;
constexpr int kMaxDevices = 256;
constexpr int kMaxP = 64, kMaxPm = 65, kMaxQ2 = 64, kMaxS = 64;
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_dev[kMaxDevices] = {};

// operator tables staged on the host (largest sizes the limits allow)
long double h_m2m[2 * kMaxPm * kMaxPm], h_m2l[4 * kMaxP * kMaxP], h_l2l[2 * kMaxP * kMaxP],
    h_rp[kMaxS * kMaxPm];
double h_reg[4 * kMaxQ2 * kMaxQ2];
double h_cast[4 * kMaxP * kMaxP + 2 * kMaxPm * kMaxPm];

// Device address of the scratch array on the current device (looked up once).
int scratch_base(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NUFFT_ECUDA;
  if (!g_noalloc_dev[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return NUFFT_ECUDA;
    g_noalloc_dev[dev] = ptr;
  }
  *out = g_noalloc_dev[dev];
  return NUFFT_OK;
}

struct Carver {
  char* base;
  size_t off, cap;
  bool ok = true;
  template <class X>
  X* take(size_t bytes) {
    size_t a = (off + 255) & ~size_t(255);
    if (a + bytes > cap) { ok = false; return nullptr; }
    off = a + bytes;
    return reinterpret_cast<X*>(base + a);
  }
};

// Upload n long-double table entries as the plan's arithmetic type.
int upload_table(nufft_plan_s* pl, void* dst, const long double* src, size_t n) {
  if (pl->prec == NUFFT_FP64) {
    for (size_t i = 0; i < n; ++i) h_cast[i] = (double)src[i];
    return cudaMemcpyAsync(dst, h_cast, n * 8, cudaMemcpyHostToDevice, pl->stream) == cudaSuccess
               ? NUFFT_OK : NUFFT_ECUDA;
  }
  float* f = reinterpret_cast<float*>(h_cast);
  for (size_t i = 0; i < n; ++i) f[i] = (float)src[i];
  return cudaMemcpyAsync(dst, f, n * 4, cudaMemcpyHostToDevice, pl->stream) == cudaSuccess
             ? NUFFT_OK : NUFFT_ECUDA;
}

}  // namespace

extern "C" int nufft_fwd_noalloc(const void* c, int64_t N, const double* y, int64_t M, double eps,
                                 int prec, unsigned flags, void* g, void* stream) {
  if (!c || !y || !g) return NUFFT_EINVAL;
  if (N > kNoAllocMaxN || M > kNoAllocMaxM) return NUFFT_EINVAL;  // beyond the fixed scratch
  if (N & (N - 1)) return NUFFT_EINVAL;  // grids of a power of two only
  if (flags & ~NUFFT_IO_C64) return NUFFT_EINVAL;
  // Tree depth: Eq. 25 (l* = 5), but at least log2 N - 6, so that a leaf
  // holds at most kMaxS grid points (few points against a large grid would
  // otherwise give shallow trees with wide leaves, beyond the staged P2M
  // table's size)
  int LN = 0;
  while ((int64_t(1) << LN) < N) ++LN;
  int L = (int)std::lround(0.5 * std::log2((double)N * (double)M) - 5.0);
  if (L < LN - 6) L = LN - 6;
  if (L > LN) L = LN;
  if (L < 2) L = 2;
  nufft_params prm{L, 0, 0, 1, -1, -1};
  int rc = nufft_choose_params(N, M, eps, prec, &prm);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if ((rc = plan_configure())) return rc;
  void* base = nullptr;
  if ((rc = scratch_base(&base))) return rc;

  nufft_plan_s pl;  // on the stack; its buffers all point into the scratch
  pl.N = N; pl.Nc = N; pl.M = M; pl.L = prm.lmax; pl.B = 1 << prm.lmax; pl.s = (int)(N >> prm.lmax);
  pl.p = prm.p; pl.q = prm.q; pl.pm = prm.p > 2 * prm.q + 1 ? prm.p : 2 * prm.q + 1;
  pl.prec = prec; pl.flags = flags | NUFFT_NO_GRAPH; pl.eps = eps;  // a graph would allocate
  pl.side_ok = 0;  // so would a side stream
  pl.stream = (cudaStream_t)stream;
  if (pl.p > kMaxP || pl.pm > kMaxPm || 2 * pl.q > kMaxQ2 || pl.s > kMaxS) return NUFFT_EINVAL;
  const int64_t B = pl.B;
  const size_t csz = prec == NUFFT_FP64 ? sizeof(double2) : sizeof(float2);
  const size_t tsz = prec == NUFFT_FP64 ? sizeof(double) : sizeof(float);
  const int64_t nm = (int64_t(2) << pl.L) - 4, nl = (int64_t(2) << pl.L) - 8;
  Carver cv{(char*)base, 0, kNoAllocBytes};
  pl.status = cv.take<int>(16);
  pl.perm = cv.take<int32_t>(M * 4);
  pl.leaf_start = cv.take<int32_t>((B + 1) * 4);
  pl.k0 = cv.take<int32_t>(M * 4);
  pl.delta = cv.take<double>(M * 8);
  pl.F = cv.take<double2>(M * 16);
  pl.E = cv.take<double2>(M * 16);
  pl.mexp = cv.take<void>(nm * pl.pm * csz);
  pl.lexp = cv.take<void>((nl > 0 ? nl : 1) * pl.p * csz);
  pl.grid = cv.take<double2>(N * 16);
  pl.grid2 = cv.take<double2>(N * 16);
  if (fft_num_passes(N) >= 3) pl.grid3 = cv.take<double2>(N * 16);
  pl.lvl2 = cv.take<double2>((8 * pl.q + 1) * 16);
  pl.fft_tw = cv.take<double2>(fft_table_elems(N) * 16);
  pl.op_m2m = cv.take<void>((size_t)2 * pl.pm * pl.pm * tsz);
  pl.op_m2l = cv.take<void>((size_t)4 * pl.p * pl.p * tsz);
  pl.op_l2l = cv.take<void>((size_t)2 * pl.p * pl.p * tsz);
  pl.op_p2m = cv.take<void>((size_t)pl.s * pl.pm * tsz);
  pl.op_reg = cv.take<double>((size_t)4 * 4 * pl.q * pl.q * 8);
  if (prec == NUFFT_MIXED) {
    pl.delta_f = cv.take<float>(M * 4);
    pl.Ff = cv.take<float2>(M * 8);
    pl.Ef = cv.take<float2>(M * 8);
    pl.lvl2f = cv.take<float2>((8 * pl.q + 1) * 8);
    pl.fft_tw_f = cv.take<float2>(fft_table_elems(N) * 8);
  }
  pl.srcpos = cv.take<void>(M * csz);
  void* tmp = cv.take<void>(setup_tmp_bytes(M, B));
  if (!cv.ok) return NUFFT_EINVAL;  // does not fit the fixed scratch

  cudaStream_t st = pl.stream;
  if (cudaMemsetAsync(pl.status, 0, 16, st) != cudaSuccess) return NUFFT_ECUDA;
  if ((rc = fft_init_tables(pl.fft_tw, pl.fft_tw_f, N, st))) return rc;
  make_operator_tables(&pl, h_m2m, h_m2l, h_l2l, h_rp, h_reg);
  // pageable host sources: each copy has read its source when the call returns
  if ((rc = upload_table(&pl, pl.op_m2m, h_m2m, (size_t)2 * pl.pm * pl.pm)) ||
      (rc = upload_table(&pl, pl.op_m2l, h_m2l, (size_t)4 * pl.p * pl.p)) ||
      (rc = upload_table(&pl, pl.op_l2l, h_l2l, (size_t)2 * pl.p * pl.p)) ||
      (rc = upload_table(&pl, pl.op_p2m, h_rp, (size_t)pl.s * pl.pm)))
    return rc;
  if (cudaMemcpyAsync(pl.op_reg, h_reg, (size_t)4 * 4 * pl.q * pl.q * 8, cudaMemcpyHostToDevice,
                      st) != cudaSuccess)
    return NUFFT_ECUDA;
  if ((rc = setup_points(&pl, y, tmp))) return rc;
  if ((rc = fmm_pack_positions(&pl))) return rc;
  int hstat = 0;
  if (cudaMemcpyAsync(&hstat, pl.status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (hstat) return (hstat & kDevIllCond) ? NUFFT_EILLCOND : NUFFT_EINVAL;
  if ((rc = nufft_plan_exec_fwd(&pl, c, g))) return rc;
  return cudaStreamSynchronize(st) == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}
