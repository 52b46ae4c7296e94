// Host implementation of the C ABI declared in include/nufft.h: parameter
// choice (Eq. 18, 18.2, 25), construction of the FMM operators, plan
// lifecycle and the exec entry points.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

namespace nufft {
bool pdl_enabled() {
  static const bool on = std::getenv("NUFFT_NO_PDL") == nullptr;
  return on;
}
bool fused_up_enabled() {
  static const bool on = std::getenv("NUFFT_NO_FUSED_UP") == nullptr;
  return on;
}
namespace {
thread_local int g_low_depth = 0;
int high_priority() {
  static const int v = [] {
    if (std::getenv("NUFFT_NO_PRIORITY")) return 0;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return 0;
    return greatest < least ? greatest : 0;  // numerically lower is higher
  }();
  return v;
}
}  // namespace
int launch_priority() { return g_low_depth > 0 ? 0 : high_priority(); }
LowPriority::LowPriority() { ++g_low_depth; }
LowPriority::~LowPriority() { --g_low_depth; }
}  // namespace nufft

using namespace nufft;

// kernels and drivers from the other translation units
size_t setup_tmp_bytes(int64_t M, int64_t B);
int setup_points(nufft_plan_s* pl, const double* y, void* tmp);
int fft_init_tables(double2* tw, float2* twf, int64_t N, cudaStream_t st);
size_t fft_table_elems(int64_t N);
int fft_configure();
int setup_configure();
int near_tc_configure();
int fft_num_passes(int64_t N);
template <class T>
int fft_run(const void* in, int in_f64, void* out, int out_f64, cplx<T>* buf, cplx<T>* buf2,
            int64_t N, int batch, int sign, const cplx<T>* tw, cudaStream_t st, int64_t n_in,
            int64_t n_out);
template <class T> int fmm_configure();
bool m2l_tc_supported(int p, int pm);
size_t m2l_tc_table_floats(int p);
void m2l_tc_table(int p, const long double* m2l, const long double* l2l, float* out);
int m2l_tc_configure();
template <class T> int fmm_forward(nufft_plan_s* pl, void* g);
template <class T> int fmm_to_grid(nufft_plan_s* pl, const void* g, int inverse);
int inverse_precompute(nufft_plan_s* pl, void* tmp, size_t tmp_bytes);
int fmm_pack_positions(nufft_plan_s* pl);
int adaptive_setup(nufft_plan_s* pl);
int fmm_up_counters(int prec, int pm, int L);
size_t inverse_tmp_bytes(const nufft_plan_s* pl);

namespace {

int ilog2(int64_t n) {
  int L = 0;
  while ((int64_t(1) << L) < n) ++L;
  return L;
}

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

// zeta(s) for even s >= 2 by Euler-Maclaurin summation (K = 64, three
// correction terms; the remainder is below 1e-30).
long double zeta_even(int s) {
  const int K = 64;
  long double sum = 0;
  for (int k = 1; k < K; ++k) sum += powl((long double)k, -(long double)s);
  long double Kl = K;
  sum += powl(Kl, 1.0L - s) / (s - 1) + 0.5L * powl(Kl, -(long double)s);
  // + B2/2! s K^{-s-1} + B4/4! s(s+1)(s+2) K^{-s-3} + B6/6! s..(s+4) K^{-s-5}
  long double t1 = (1.0L / 6.0L) / 2.0L * s * powl(Kl, -(long double)s - 1);
  long double t2 = (-1.0L / 30.0L) / 24.0L * s * (s + 1.0L) * (s + 2.0L) * powl(Kl, -(long double)s - 3);
  long double t3 = (1.0L / 42.0L) / 720.0L * s * (s + 1.0L) * (s + 2.0L) * (s + 3.0L) * (s + 4.0L) *
                   powl(Kl, -(long double)s - 5);
  return sum + t1 + t2 + t3;
}

// binomial coefficients C(i, k), 0 <= k <= i <= kBinomMax, in a fixed table
constexpr int kBinomMax = 2 * 64 + 2;
struct Binom {
  long double c[(kBinomMax + 1) * (kBinomMax + 1)];
  Binom() {
    const int n = kBinomMax;
    for (int i = 0; i <= n; ++i) {
      c[i * (n + 1)] = 1;
      for (int k = 1; k <= n; ++k)
        c[i * (n + 1) + k] = (k > i) ? 0 : c[(i - 1) * (n + 1) + k - 1] + c[(i - 1) * (n + 1) + k];
    }
  }
  long double operator()(int i, int k) const {
    return (k < 0 || k > i) ? 0 : c[i * (kBinomMax + 1) + k];
  }
};

thread_local int g_configured = 0;

int configure_once() {
  if (g_configured) return NUFFT_OK;
  int rc = fft_configure();
  if (!rc) rc = fmm_configure<double>();
  if (!rc) rc = fmm_configure<float>();
  if (!rc) rc = m2l_tc_configure();
  if (!rc) rc = setup_configure();
  if (!rc) rc = near_tc_configure();
  if (!rc) g_configured = 1;
  return rc;
}

template <class T>
std::vector<T> cast_vec(const std::vector<long double>& v) {
  std::vector<T> r(v.size());
  for (size_t i = 0; i < v.size(); ++i) r[i] = (T)v[i];
  return r;
}

int upload(void** dst, const void* src, size_t bytes) {
  if (cudaMalloc(dst, bytes) != cudaSuccess) return NUFFT_ENOMEM;
  if (cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return NUFFT_ECUDA;
  return NUFFT_OK;
}

}  // namespace

int plan_configure() { return configure_once(); }

// The translation operators (level independent, scaled form) and the
// level-2 weights of a plan, written into caller arrays of sizes
// m2m 2 pm^2, m2l 4 p^2, l2l 2 p^2, rp s pm, reg 4 (2q)^2 (every entry set).
void make_operator_tables(const nufft_plan_s* pl, long double* m2m, long double* m2l,
                          long double* l2l, long double* rp, double* reg) {
  const int p = pl->p, pm = pl->pm, q = pl->q, Q2 = 2 * q, s = pl->s;
  static const Binom C;
  // M2M [sigma][k][m]
  for (size_t i = 0; i < (size_t)2 * pm * pm; ++i) m2m[i] = 0.0L;
  for (int sg = 0; sg < 2; ++sg) {
    long double sig = sg ? 0.25L : -0.25L;
    for (int m = 0; m < pm; ++m)
      for (int k = 0; k <= m; ++k)
        m2m[(size_t)sg * pm * pm + (size_t)k * pm + m] =
            C(m, k) * powl(0.5L, k) * powl(sig, m - k);
  }
  // M2L [d][m][n], d = -3, -2, 2, 3
  const int dval[4] = {-3, -2, 2, 3};
  for (int t = 0; t < 4; ++t)
    for (int m = 0; m < p; ++m)
      for (int n = 0; n < p; ++n) {
        long double v = C(m + n, n) * powl((long double)dval[t], -(long double)(m + n + 1));
        if ((m + 1) & 1) v = -v;  // (-1)^(m+1)
        m2l[(size_t)t * p * p + (size_t)m * p + n] = v;
      }
  // L2L [sigma][n'][n]
  for (size_t i = 0; i < (size_t)2 * p * p; ++i) l2l[i] = 0.0L;
  for (int sg = 0; sg < 2; ++sg) {
    long double sig = sg ? 0.25L : -0.25L;
    for (int n = 0; n < p; ++n)
      for (int k = n; k < p; ++k)
        l2l[(size_t)sg * p * p + (size_t)k * p + n] =
            0.5L * C(k, n) * powl(0.5L, n) * powl(sig, k - n);
  }
  // P2M table for the uniform grid: rho_o = o/s - 1/2
  for (int o = 0; o < s; ++o) {
    long double rho = (long double)o / s - 0.5L, pw = 1;
    for (int m = 0; m < pm; ++m) { rp[(size_t)o * pm + m] = pw; pw *= rho; }
  }
  // level-2 weights W1, W2 [l][i], shifts S-, S+ [i][r]
  for (size_t i = 0; i < (size_t)4 * Q2 * Q2; ++i) reg[i] = 0.0;
  for (int l = 0; l < Q2; ++l)
    for (int i = 0; i < Q2; ++i) {
      if (((i + l) & 1) == 0) continue;
      int m = (i + l + 1) / 2;
      if (m < 1 || m > q) continue;
      long double z = zeta_even(2 * m);
      long double am = 2.0L * z * powl(0.25L, m);
      long double bm = 2.0L * z * (1.0L - powl(0.25L, m));
      reg[(size_t)l * Q2 + i] = (double)(C(2 * m - 1, l) * am);
      reg[(size_t)Q2 * Q2 + (size_t)l * Q2 + i] = (double)(C(2 * m - 1, l) * bm);
    }
  for (int i = 0; i < Q2; ++i)
    for (int r = 0; r <= i; ++r) {
      long double c = C(i, r) * powl(0.5L, i - r);
      reg[(size_t)2 * Q2 * Q2 + (size_t)i * Q2 + r] = (double)(((i - r) & 1) ? -c : c);
      reg[(size_t)3 * Q2 * Q2 + (size_t)i * Q2 + r] = (double)c;
    }
}

namespace {

// Build the operators of a plan and upload them in the plan's arithmetic type.
int build_operators(nufft_plan_s* pl) {
  const int p = pl->p, pm = pl->pm, q = pl->q, Q2 = 2 * q, s = pl->s;
  std::vector<long double> m2m((size_t)2 * pm * pm), m2l((size_t)4 * p * p),
      l2l((size_t)2 * p * p), rp((size_t)s * pm);
  std::vector<double> reg((size_t)4 * Q2 * Q2);
  make_operator_tables(pl, m2m.data(), m2l.data(), l2l.data(), rp.data(), reg.data());
  int rc;
  if (pl->prec == NUFFT_FP64) {
    auto a = cast_vec<double>(m2m), b = cast_vec<double>(m2l), c = cast_vec<double>(l2l),
         d = cast_vec<double>(rp);
    if ((rc = upload(&pl->op_m2m, a.data(), a.size() * 8))) return rc;
    if ((rc = upload(&pl->op_m2l, b.data(), b.size() * 8))) return rc;
    if ((rc = upload(&pl->op_l2l, c.data(), c.size() * 8))) return rc;
    if ((rc = upload(&pl->op_p2m, d.data(), d.size() * 8))) return rc;
  } else {
    auto a = cast_vec<float>(m2m), b = cast_vec<float>(m2l), c = cast_vec<float>(l2l),
         d = cast_vec<float>(rp);
    if ((rc = upload(&pl->op_m2m, a.data(), a.size() * 4))) return rc;
    if ((rc = upload(&pl->op_m2l, b.data(), b.size() * 4))) return rc;
    if ((rc = upload(&pl->op_l2l, c.data(), c.size() * 4))) return rc;
    if ((rc = upload(&pl->op_p2m, d.data(), d.size() * 4))) return rc;
  }
  if (pl->tc_level >= 4) {
    std::vector<float> tc(m2l_tc_table_floats(p));
    m2l_tc_table(p, m2l.data(), l2l.data(), tc.data());
    if ((rc = upload((void**)&pl->op_tc, tc.data(), tc.size() * 4))) return rc;
  }
  return upload((void**)&pl->op_reg, reg.data(), reg.size() * 8);
}

void free_plan(nufft_plan_s* pl) {
  void* ptrs[] = {pl->perm, pl->leaf_start, pl->k0, pl->delta, pl->F, pl->E, pl->delta_f,
                  pl->Ff, pl->Ef, pl->lvl2f, pl->Dt, pl->Dtf, pl->Ct, pl->Ctf, pl->Sinv, pl->Sinvf, pl->selft, pl->srcpos, pl->Lambda, pl->mexp, pl->lexp,
                  pl->charge, pl->grid, pl->grid2, pl->grid3, pl->lvl2, pl->op_m2m, pl->op_m2l,
                  pl->op_l2l, pl->op_p2m, pl->op_reg, pl->fft_tw, pl->fft_tw_f, pl->status,
                  pl->seg_overflow, pl->lsq_work, pl->op_tc, pl->upcnt, pl->hnear,
                  pl->ad_box, pl->ad_perm, pl->ad_pos, pl->ad_F, pl->ad_E, pl->ad_Ff, pl->ad_Ef,
                  pl->ad_p2m, pl->ad_lexp, pl->ad_start, pl->ad_tiles, pl->ad_srange,
                  pl->ad_gbox, pl->ad_gil, pl->ad_mexp, pl->ad_Dt, pl->ad_S, pl->ad_Dtf,
                  pl->ad_Sf, pl->ad_charge, pl->ad_st, pl->ad_rleaf, pl->p2m_chunk,
                  pl->p2m_cfirst, pl->p2m_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (auto& gr : pl->graphs)
    if (gr.exec) cudaGraphExecDestroy(gr.exec);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  if (pl->aux) cudaStreamDestroy(pl->aux);
  if (pl->aux2) cudaStreamDestroy(pl->aux2);
  for (int i = 0; i < 3; ++i) {
    if (pl->ev_fork[i]) cudaEventDestroy(pl->ev_fork[i]);
    if (pl->ev_join[i]) cudaEventDestroy(pl->ev_join[i]);
  }
  if (pl->prof) {
    for (cudaEvent_t e : pl->prof->ev)
      if (e) cudaEventDestroy(e);
    delete pl->prof;
  }
  delete pl;
}

template <class X>
int dalloc(X** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  return cudaMalloc((void**)p, bytes) == cudaSuccess ? NUFFT_OK : NUFFT_ENOMEM;
}

// Chunks of the P2M of clustered sources: each leaf's sorted sources cut into
// runs of at most 256 (the chunked kernel's unit), leaf by leaf.
int build_p2m_chunks(nufft_plan_s* pl, const std::vector<int32_t>& start) {
  const int64_t B = pl->B;
  std::vector<int32_t> chunk, cfirst((size_t)B + 1);
  for (int64_t b = 0; b < B; ++b) {
    cfirst[(size_t)b] = (int32_t)(chunk.size() / 3);
    for (int32_t a = start[(size_t)b]; a < start[(size_t)b + 1]; a += 256) {
      const int32_t e = a + 256 < start[(size_t)b + 1] ? a + 256 : start[(size_t)b + 1];
      chunk.push_back((int32_t)b);
      chunk.push_back(a);
      chunk.push_back(e);
    }
  }
  cfirst[(size_t)B] = (int32_t)(chunk.size() / 3);
  pl->p2m_nchunk = (int64_t)chunk.size() / 3;
  const size_t csz = pl->prec == NUFFT_FP64 ? sizeof(double2) : sizeof(float2);
  int rc;
  if ((rc = upload((void**)&pl->p2m_chunk, chunk.data(), chunk.size() * 4)) ||
      (rc = upload((void**)&pl->p2m_cfirst, cfirst.data(), cfirst.size() * 4)) ||
      (rc = dalloc(&pl->p2m_part, (size_t)pl->batch * pl->p2m_nchunk * pl->pm * csz)))
    return rc;
  return NUFFT_OK;
}

}  // namespace

cudaStream_t side_begin(nufft_plan_s* pl, int slot) {
  if (!pl->side_ok || (pl->prof && pl->prof->enabled)) return pl->stream;
  cudaStream_t& as = slot == 2 ? pl->aux2 : pl->aux;
  if (!as) {
    if (cudaStreamCreateWithFlags(&as, cudaStreamNonBlocking) != cudaSuccess) {
      as = nullptr;
      pl->side_ok = 0;
      return pl->stream;
    }
  }
  if (!pl->ev_fork[slot]) {
    if (cudaEventCreateWithFlags(&pl->ev_fork[slot], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&pl->ev_join[slot], cudaEventDisableTiming) != cudaSuccess) {
      pl->side_ok = 0;
      return pl->stream;
    }
  }
  if (cudaEventRecord(pl->ev_fork[slot], pl->stream) != cudaSuccess ||
      cudaStreamWaitEvent(as, pl->ev_fork[slot], 0) != cudaSuccess)
    return pl->stream;
  return as;
}

void side_end(nufft_plan_s* pl, int slot, cudaStream_t s) {
  if (s != pl->stream) cudaEventRecord(pl->ev_join[slot], s);
}

void side_join(nufft_plan_s* pl, int slot) {
  // a no-op unless the branch ran on its side stream (its join event was recorded)
  cudaStream_t as = slot == 2 ? pl->aux2 : pl->aux;
  if (as && pl->side_ok && pl->ev_join[slot] && !(pl->prof && pl->prof->enabled))
    cudaStreamWaitEvent(pl->stream, pl->ev_join[slot], 0);
}

void prof_begin(nufft_plan_s* pl, int stage) {
  StageProf* pf = pl->prof;
  if (!pf) return;
  pf->open_stage = stage;
  if (!pf->enabled || pf->npairs >= StageProf::kMaxPairs) return;
  cudaEvent_t& e = pf->ev[2 * pf->npairs];
  if (!e && cudaEventCreate(&e) != cudaSuccess) { e = nullptr; return; }
  cudaEventRecord(e, pl->stream);
}

void prof_end(nufft_plan_s* pl, int launches) {
  StageProf* pf = pl->prof;
  if (!pf || pf->open_stage < 0) return;
  pf->launches[pf->open_stage] += launches;
  if (pf->enabled && pf->npairs < StageProf::kMaxPairs && pf->ev[2 * pf->npairs]) {
    cudaEvent_t& e = pf->ev[2 * pf->npairs + 1];
    if (e || cudaEventCreate(&e) == cudaSuccess) {
      cudaEventRecord(e, pl->stream);
      pf->stage[pf->npairs++] = pf->open_stage;
    }
  }
  pf->open_stage = -1;
}

extern "C" {

int nufft_plan_profile(nufft_plan pl, int enable) {
  if (!pl || !pl->prof) return NUFFT_EINVAL;
  StageProf* pf = pl->prof;
  pf->enabled = enable ? 1 : 0;
  pf->npairs = 0;
  for (int i = 0; i < NUFFT_NSTAGES; ++i) { pf->ms[i] = 0; pf->launches[i] = 0; }
  return NUFFT_OK;
}

int nufft_plan_stats(nufft_plan pl, double* stage_ms, int64_t* launches) {
  if (!pl || !pl->prof) return NUFFT_EINVAL;
  StageProf* pf = pl->prof;
  if (cudaStreamSynchronize(pl->stream) != cudaSuccess) return NUFFT_ECUDA;
  for (int i = 0; i < pf->npairs; ++i) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, pf->ev[2 * i], pf->ev[2 * i + 1]) != cudaSuccess)
      return NUFFT_ECUDA;
    pf->ms[pf->stage[i]] += ms;
  }
  pf->npairs = 0;
  for (int i = 0; i < NUFFT_NSTAGES; ++i) {
    if (stage_ms) stage_ms[i] = pf->ms[i];
    if (launches) launches[i] = pf->launches[i];
  }
  return NUFFT_OK;
}


const char* nufft_strerror(int status) {
  switch (status) {
    case NUFFT_OK: return "success";
    case NUFFT_EINVAL: return "invalid argument";
    case NUFFT_ENOMEM: return "out of memory";
    case NUFFT_ECUDA: return "CUDA error";
    case NUFFT_EILLCOND: return "inverse is ill-conditioned (duplicate points or exponent range)";
    case NUFFT_ENOTCONV: return "iteration did not converge";
    case NUFFT_ETIMEOUT: return "device wait timed out";
    case NUFFT_ENOTSUP: return "unsupported option combination";
    default: return "unknown status";
  }
}

int nufft_version(void) { return 100; }

// FMM grid of N coefficients: the next power of two
static int64_t grid_of(int64_t N) {
  int64_t g = 1;
  while (g < N) g <<= 1;
  return g;
}

// Threshold ("machine precision") error of the FP64 path on a grid of N
// points (Sec. 3.1-3.2): the error of the paper's f = 1 test, max_j |g_j - 1|,
// stops falling as eps is lowered at about log2(N) 2^-53 (measured on GB300
// for N = 2^8 .. 2^22, uniform points: 0.8e-15 .. 2.2e-15, each within 20 %
// below this line), at least 1e-15, the smallest eps accepted.
static double eps_threshold_fp64(int64_t N) {
  int L = 0;
  while ((int64_t(1) << L) < N) ++L;
  const double e = (double)L * 0x1p-53;
  return e > 1e-15 ? e : 1e-15;
}

extern "C" double nufft_eps_threshold(int64_t N) {
  if (N < 8 || N > (int64_t(1) << 26)) return -1.0;
  return eps_threshold_fp64(grid_of(N));
}

int nufft_choose_params(int64_t Nc, int64_t M, double eps, int prec, nufft_params* prm) {
  if (!prm) return NUFFT_EINVAL;
  if (Nc < 8 || Nc > (int64_t(1) << 26)) return NUFFT_EINVAL;
  const int64_t N = grid_of(Nc);  // the tree and the FFT live on this grid
  if (M < 1 || M > (int64_t(1) << 27)) return NUFFT_EINVAL;
  // eps = 0: machine precision (Sec. 3.2's second setting): the threshold
  // error eps_th(N) as the prescribed accuracy, p and q from Eq. 18.2 at it
  if (eps == 0.0 && prec == NUFFT_FP64) eps = eps_threshold_fp64(N);
  if (!(eps >= 1e-15 && eps <= 1e-1)) return NUFFT_EINVAL;
  if (prec != NUFFT_FP64 && prec != NUFFT_MIXED) return NUFFT_EINVAL;
  if (prec == NUFFT_MIXED && eps < 1e-7) return NUFFT_EINVAL;
  int LN = ilog2(N);
  int L = prm->lmax;
  if (L <= 0) {
    // Eq. 25 with the empirical l* = 5 of Sec. 3.2: log2 sqrt(N M) - 5
    double lopt = 0.5 * std::log2((double)N * (double)M) - 5.0;
    L = (int)std::lround(lopt);
    if (L < 2) L = 2;
    if (L > LN) L = LN;
  }
  if (L < 2 || L > LN || L > 24) return NUFFT_EINVAL;
  // Eq. 18.2 with the fraction of Eq. 18 solved for eps: 10 / (3 pi eps)
  double r = 10.0 / (3.0 * M_PI * eps);
  int q = prm->q, p = prm->p;
  if (q <= 0) {
    q = (int)std::ceil(0.5 * std::log2(r));
    if (q < 2) q = 2;
  }
  if (p <= 0) {
    p = (int)std::ceil(1.0 + std::log(r) / std::log(3.0) + L / std::log2(3.0));
    if (p < 4) p = 4;
  }
  if (q < 2 || q > 32 || p < 4 || p > 64) return NUFFT_EINVAL;
  int batch = prm->batch <= 0 ? 1 : prm->batch;
  if (batch > 4096) return NUFFT_EINVAL;
  int tc = prm->tc_level;
  if (tc != -1 && tc != 0 && (tc < 4 || tc > 30)) return NUFFT_EINVAL;
  if (prec != NUFFT_MIXED || !m2l_tc_supported(p, p > 2 * q + 1 ? p : 2 * q + 1)) tc = -1;
  if (tc == 0) {
    // finest levels with at least 2048 parents over all signals (32 tiles)
    tc = -1;
    for (int l = 6; l <= L; ++l)
      if ((int64_t(1) << (l - 1)) * batch >= 2048) { tc = l; break; }
  }
  if (tc > L) tc = -1;
  // near field of batched forwards on the tensor cores: groups of 64 signals
  int tn = prm->tc_near;
  if (tn != -1 && tn != 0 && tn != 1) return NUFFT_EINVAL;
  const bool tn_ok = prec == NUFFT_MIXED && batch % 64 == 0;
  if (tn == 0) tn = tn_ok ? 1 : -1;
  if (tn == 1 && !tn_ok) tn = -1;
  prm->lmax = L;
  prm->p = p;
  prm->q = q;
  prm->batch = batch;
  prm->tc_level = tc;
  prm->tc_near = tn;
  return NUFFT_OK;
}

int nufft_plan_create(nufft_plan* out, int64_t N, int64_t M, const double* y, double eps,
                      int prec, const nufft_params* params, unsigned flags, void* stream) {
  if (!out || !y) return NUFFT_EINVAL;
  *out = nullptr;
  nufft_params prm{0, 0, 0, 0, 0, 0};
  if (params) prm = *params;
  int rc = nufft_choose_params(N, M, eps, prec, &prm);
  if (rc) return rc;
  if (flags & ~(NUFFT_IO_C64 | NUFFT_WANT_INVERSE | NUFFT_NO_GRAPH | NUFFT_ADAPTIVE))
    return NUFFT_EINVAL;
  if ((flags & NUFFT_ADAPTIVE) && prm.batch != 1) return NUFFT_ENOTSUP;
  if ((flags & NUFFT_WANT_INVERSE) && M != N) return NUFFT_EINVAL;
  const int64_t Nc = N;
  N = grid_of(Nc);
  const int64_t nb = prm.batch;
  if ((rc = configure_once())) return rc;
  nufft_plan_s* pl = new (std::nothrow) nufft_plan_s();
  if (!pl) return NUFFT_ENOMEM;
  pl->prof = new (std::nothrow) StageProf();
  if (!pl->prof) { delete pl; return NUFFT_ENOMEM; }
  pl->N = N; pl->Nc = Nc; pl->M = M; pl->L = prm.lmax; pl->B = 1 << prm.lmax;
  // square inverse for Nc < N: C carries the phase e^{i pi k Nc / N}
  pl->inv_nc = ((flags & NUFFT_WANT_INVERSE) && Nc != N) ? Nc : 0;
  pl->s = (int)(N >> prm.lmax);
  pl->p = prm.p; pl->q = prm.q; pl->pm = prm.p > 2 * prm.q + 1 ? prm.p : 2 * prm.q + 1;
  pl->prec = prec; pl->flags = flags; pl->eps = eps; pl->batch = (int)nb;
  pl->tc_level = prm.tc_level;
  pl->tc_near = prm.tc_near;
  pl->stream = (cudaStream_t)stream;
  const int64_t B = pl->B;
  const size_t csz = prec == NUFFT_FP64 ? sizeof(double2) : sizeof(float2);
  const int64_t nm = (int64_t(2) << pl->L) - 4, nl = (int64_t(2) << pl->L) - 8;
  int64_t big = N > M ? N : M;
  if ((rc = dalloc(&pl->perm, M * 4)) || (rc = dalloc(&pl->leaf_start, (B + 1) * 4)) ||
      (rc = dalloc(&pl->k0, M * 4)) || (rc = dalloc(&pl->delta, M * 8)) ||
      (rc = dalloc(&pl->F, M * 16)) || (rc = dalloc(&pl->E, M * 16)) ||
      (rc = dalloc(&pl->mexp, nb * nm * pl->pm * csz)) ||
      (rc = dalloc(&pl->lexp, nb * (nl > 0 ? nl : 1) * pl->p * csz)) ||
      (rc = dalloc(&pl->charge, nb * big * csz)) || (rc = dalloc(&pl->selft, nb * M * csz)) ||
      (rc = dalloc(&pl->srcpos, M * csz)) ||
      (rc = dalloc(&pl->grid, nb * N * 16)) ||
      (rc = dalloc(&pl->grid2, nb * N * 16)) || (rc = dalloc(&pl->lvl2, nb * (8 * pl->q + 1) * 16)) ||
      (rc = dalloc(&pl->fft_tw, fft_table_elems(N) * 16)) || (rc = dalloc(&pl->status, 16))) {
    free_plan(pl);
    return rc;
  }
  if (fft_num_passes(N) >= 3 && (rc = dalloc(&pl->grid3, nb * N * 16))) { free_plan(pl); return rc; }
  // near-field sums of the split target evaluation (one signal)
  if (nb == 1 && (rc = dalloc(&pl->hnear, 2 * big * 16))) { free_plan(pl); return rc; }
  if (prec == NUFFT_MIXED &&
      ((rc = dalloc(&pl->delta_f, M * 4)) || (rc = dalloc(&pl->Ff, M * 8)) ||
       (rc = dalloc(&pl->Ef, M * 8)) || (rc = dalloc(&pl->lvl2f, nb * (8 * pl->q + 1) * 8)) ||
       (rc = dalloc(&pl->fft_tw_f, fft_table_elems(N) * 8)))) {
    free_plan(pl);
    return rc;
  }
  if ((rc = build_operators(pl))) { free_plan(pl); return rc; }
  cudaStream_t st = pl->stream;
  if (cudaMemsetAsync(pl->status, 0, 16, st) != cudaSuccess) { free_plan(pl); return NUFFT_ECUDA; }
  // group counters of the one-launch upward pass (start at zero, left at zero)
  const int ncnt = fmm_up_counters(prec, pl->pm, pl->L);
  if (ncnt >= 0) {
    const size_t cb = (size_t)nb * (ncnt > 0 ? ncnt : 1) * 4;
    if ((rc = dalloc(&pl->upcnt, cb))) { free_plan(pl); return rc; }
    if (cudaMemsetAsync(pl->upcnt, 0, cb, st) != cudaSuccess) { free_plan(pl); return NUFFT_ECUDA; }
    pl->upcnt_n = ncnt;
  }
  if ((rc = fft_init_tables(pl->fft_tw, pl->fft_tw_f, N, st))) { free_plan(pl); return rc; }
  size_t tb = setup_tmp_bytes(M, B);
  if (flags & NUFFT_WANT_INVERSE) {
    size_t ib = inverse_tmp_bytes(pl);
    if (ib > tb) tb = ib;
  }
  void* tmp = nullptr;
  if (cudaMalloc(&tmp, tb) != cudaSuccess) { free_plan(pl); return NUFFT_ENOMEM; }
  rc = setup_points(pl, y, tmp);
  if (!rc) rc = fmm_pack_positions(pl);
  std::vector<int32_t> ls((size_t)B + 1);
  if (!rc) {  // the fullest leaf (the adjoint's near-field kernel choice)
    if (cudaMemcpyAsync(ls.data(), pl->leaf_start, (B + 1) * 4, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = NUFFT_ECUDA;
    for (int64_t b = 0; !rc && b < B; ++b)
      if (ls[b + 1] - ls[b] > pl->max_leaf) pl->max_leaf = ls[b + 1] - ls[b];
  }
  if (!rc && (flags & NUFFT_WANT_INVERSE)) rc = inverse_precompute(pl, tmp, tb);
  // clustered sources (a leaf with at least 4x the mean count): the chunks of
  // the adjoint / inverse P2M, at most 256 sources of one leaf each
  if (!rc && M > 0 && (int64_t)pl->max_leaf * B >= 4 * M) rc = build_p2m_chunks(pl, ls);
  if (!rc && (flags & NUFFT_ADAPTIVE)) rc = adaptive_setup(pl);
  int hstat = 0;
  if (!rc) {
    if (cudaMemcpyAsync(&hstat, pl->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = NUFFT_ECUDA;
  }
  cudaFree(tmp);
  if (!rc && (hstat & kDevBadPoint)) rc = NUFFT_EINVAL;
  if (!rc && (hstat & kDevSegTooLarge)) rc = NUFFT_EINVAL;
  if (!rc && (hstat & kDevIllCond)) rc = NUFFT_EILLCOND;
  if (rc) { free_plan(pl); return rc; }
  *out = pl;
  return NUFFT_OK;
}

int nufft_plan_destroy(nufft_plan pl) {
  if (!pl) return NUFFT_EINVAL;
  cudaStreamSynchronize(pl->stream);
  free_plan(pl);
  return NUFFT_OK;
}

int nufft_plan_info(nufft_plan pl, int* lmax, int* p, int* q) {
  if (!pl) return NUFFT_EINVAL;
  if (lmax) *lmax = pl->L;
  if (p) *p = pl->p;
  if (q) *q = pl->q;
  return NUFFT_OK;
}

int nufft_plan_params(nufft_plan pl, nufft_params* out) {
  if (!pl || !out) return NUFFT_EINVAL;
  out->lmax = pl->L;
  out->p = pl->p;
  out->q = pl->q;
  out->batch = pl->batch;
  out->tc_level = pl->tc_level;
  out->tc_near = pl->tc_near;
  return NUFFT_OK;
}

int nufft_plan_sync(nufft_plan pl) {
  if (!pl) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  int h = 0;
  if (cudaMemcpyAsync(&h, pl->status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (h & kDevTimeout) {
    const int keep = h & ~kDevTimeout;
    if (cudaMemcpyAsync(pl->status, &keep, 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NUFFT_ECUDA;
    return NUFFT_ETIMEOUT;
  }
  return NUFFT_OK;
}

int nufft_plan_points(nufft_plan pl, int32_t* perm, int32_t* leaf_start, int32_t* k0,
                      double* delta) {
  if (!pl) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return !dst || cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess;
  };
  if (!cp(perm, pl->perm, pl->M * 4) || !cp(leaf_start, pl->leaf_start, (pl->B + 1) * 4) ||
      !cp(k0, pl->k0, pl->M * 4) || !cp(delta, pl->delta, pl->M * 8))
    return NUFFT_ECUDA;
  return NUFFT_OK;
}

int nufft_plan_inverse_coeffs(nufft_plan pl, double* Ct, double* Dt, double* Lambda) {
  if (!pl || !pl->Ct) return NUFFT_EINVAL;
  cudaStream_t st = pl->stream;
  if (Ct && cudaMemcpyAsync(Ct, pl->Ct, pl->N * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (Dt && cudaMemcpyAsync(Dt, pl->Dt, pl->M * 16, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return NUFFT_ECUDA;
  if (Lambda) {
    if (cudaMemcpyAsync(Lambda, pl->Lambda, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NUFFT_ECUDA;
  }
  return NUFFT_OK;
}

int nufft_plan_set_stream(nufft_plan pl, void* stream) {
  if (!pl) return NUFFT_EINVAL;
  pl->stream = (cudaStream_t)stream;
  return NUFFT_OK;
}

// c_n <-> grid with the FFT of the plan's arithmetic (FP64, or FP32 for the
// mixed path); caller data complex128 or complex64.
// (n_in / n_out: caller-side lengths, Nc for the coefficients, 0 = the grid)
static int fft_plan(nufft_plan_s* pl, const void* in, int in_f64, void* out, int out_f64,
                    int sign, int64_t n_in, int64_t n_out) {
  prof_begin(pl, NUFFT_STAGE_FFT);
  int rc;
  if (pl->prec == NUFFT_FP64)
    rc = fft_run<double>(in, in_f64, out, out_f64, pl->grid2, pl->grid3, pl->N, pl->batch, sign,
                         pl->fft_tw, pl->stream, n_in, n_out);
  else
    rc = fft_run<float>(in, in_f64, out, out_f64, (float2*)pl->grid2, (float2*)pl->grid3, pl->N,
                        pl->batch, sign, pl->fft_tw_f, pl->stream, n_in, n_out);
  prof_end(pl, fft_num_passes(pl->N));
  return rc;
}

static int exec_fwd_direct(nufft_plan_s* pl, const void* c, void* g) {
  const int io64 = (pl->flags & NUFFT_IO_C64) ? 0 : 1;
  const int t64 = pl->prec == NUFFT_FP64;
  // f_k = sum_n c_n e^{+2 pi i n k/N}  (Eq. p1, unscaled inverse DFT; c_n = 0
  // for Nc <= n < N)
  int rc = fft_plan(pl, c, io64, pl->grid, t64, +1, pl->Nc, 0);
  if (rc) return rc;
  return pl->prec == NUFFT_FP64 ? fmm_forward<double>(pl, g) : fmm_forward<float>(pl, g);
}

static int grid_to_coeffs(nufft_plan_s* pl, void* c) {
  // c'_n = sum_k u_k e^{-2 pi i n k/N}
  const int io64 = (pl->flags & NUFFT_IO_C64) ? 0 : 1;
  return fft_plan(pl, pl->grid, pl->prec == NUFFT_FP64, c, io64, -1, 0, pl->Nc);
}

static int exec_adj_direct(nufft_plan_s* pl, const void* g, void* c) {
  int rc = pl->prec == NUFFT_FP64 ? fmm_to_grid<double>(pl, g, 0) : fmm_to_grid<float>(pl, g, 0);
  if (rc) return rc;
  return grid_to_coeffs(pl, c);
}

static int exec_inv_direct(nufft_plan_s* pl, const void* g, void* c) {
  int rc = pl->prec == NUFFT_FP64 ? fmm_to_grid<double>(pl, g, 1) : fmm_to_grid<float>(pl, g, 1);
  if (rc) return rc;
  return grid_to_coeffs(pl, c);  // the 1/N of Eq. p1 is folded into C_k
}

// Run exec sequence `op` (0 fwd, 1 adj, 2 inv) on the plan's stream: replay
// the graph captured for (op, in, out) if there is one, else capture it on
// the private stream, instantiate and launch it; direct launches while
// profiling, while the plan's stream is itself capturing, or with
// NUFFT_NO_GRAPH.
static int exec_op(nufft_plan_s* pl, int op, const void* in, void* out) {
  auto direct = [&](nufft_plan_s* q) {
    return op == 0 ? exec_fwd_direct(q, in, out)
                   : (op == 1 ? exec_adj_direct(q, in, out) : exec_inv_direct(q, in, out));
  };
  bool graph = !(pl->flags & NUFFT_NO_GRAPH) && !(pl->prof && pl->prof->enabled);
  if (graph) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(pl->stream, &cs) != cudaSuccess) return NUFFT_ECUDA;
    graph = cs == cudaStreamCaptureStatusNone;
  }
  if (!graph) return direct(pl);
  for (auto& gr : pl->graphs)
    if (gr.exec && gr.op == op && gr.in == in && gr.out == out)
      return cudaGraphLaunch(gr.exec, pl->stream) == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
  if (!pl->cap && cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking) != cudaSuccess) {
    pl->cap = nullptr;
    return NUFFT_ECUDA;
  }
  cudaStream_t user = pl->stream;
  if (cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return NUFFT_ECUDA;
  pl->stream = pl->cap;
  int rc = direct(pl);
  pl->stream = user;
  cudaGraph_t g = nullptr;
  cudaError_t ec = cudaStreamEndCapture(pl->cap, &g);
  if (rc || ec != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc ? rc : NUFFT_ECUDA;
  }
  cudaGraphExec_t ex = nullptr;
  // per-node priorities (critical path high, the near-field branch default)
  ec = cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(g);
  if (ec != cudaSuccess) return NUFFT_ECUDA;
  auto& slot = pl->graphs[pl->graph_next];
  pl->graph_next = (pl->graph_next + 1) % nufft_plan_s::kGraphSlots;
  if (slot.exec) cudaGraphExecDestroy(slot.exec);
  slot.op = op;
  slot.in = in;
  slot.out = out;
  slot.exec = ex;
  return cudaGraphLaunch(ex, pl->stream) == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

int nufft_plan_exec_fwd(nufft_plan pl, const void* c, void* g) {
  if (!pl || !c || !g) return NUFFT_EINVAL;
  return exec_op(pl, 0, c, g);
}

int nufft_plan_exec_adj(nufft_plan pl, const void* g, void* c) {
  if (!pl || !c || !g) return NUFFT_EINVAL;
  return exec_op(pl, 1, g, c);
}

int nufft_plan_exec_inv(nufft_plan pl, const void* g, void* c) {
  if (!pl || !c || !g) return NUFFT_EINVAL;
  if (!(pl->flags & NUFFT_WANT_INVERSE) || !pl->Ct) return NUFFT_EINVAL;
  return exec_op(pl, 2, g, c);
}

static int one_shot(int which, const void* in, int64_t N, const double* y, int64_t M, double eps,
                    int prec, unsigned flags, void* out, void* stream) {
  nufft_plan pl = nullptr;
  if (which == 2) flags |= NUFFT_WANT_INVERSE;
  flags |= NUFFT_NO_GRAPH;  // one exec: capturing a graph would not pay
  int rc = nufft_plan_create(&pl, N, M, y, eps, prec, nullptr, flags, stream);
  if (rc) return rc;
  if (which == 0) rc = nufft_plan_exec_fwd(pl, in, out);
  else if (which == 1) rc = nufft_plan_exec_adj(pl, in, out);
  else rc = nufft_plan_exec_inv(pl, in, out);
  if (!rc && cudaStreamSynchronize(pl->stream) != cudaSuccess) rc = NUFFT_ECUDA;
  nufft_plan_destroy(pl);
  return rc;
}

int nufft_fwd(const void* c, int64_t N, const double* y, int64_t M, double eps, int prec,
              unsigned flags, void* g, void* stream) {
  return one_shot(0, c, N, y, M, eps, prec, flags, g, stream);
}

int nufft_adj(const void* g, const double* y, int64_t M, int64_t N, double eps, int prec,
              unsigned flags, void* c, void* stream) {
  return one_shot(1, g, N, y, M, eps, prec, flags, c, stream);
}

int inufft(const void* g, const double* y, int64_t M, int64_t N, double eps, int prec,
           unsigned flags, void* c, void* stream) {
  if (M == N) return one_shot(2, g, N, y, M, eps, prec, flags, c, stream);
  if (M < N || !g || !c) return NUFFT_EINVAL;  // fewer samples than coefficients
  if (flags & ~(NUFFT_IO_C64 | NUFFT_NO_GRAPH)) return NUFFT_EINVAL;
  if (flags & NUFFT_IO_C64) return NUFFT_ENOTSUP;
  // M > N: least squares by plain CG on the normal equations
  nufft_plan pl = nullptr;
  int rc = nufft_plan_create(&pl, N, M, y, eps, prec, nullptr, flags, stream);
  if (rc) return rc;
  const double tol = eps > 1e-14 ? eps : 1e-14;
  rc = nufft_plan_solve_lsq(pl, g, nullptr, 0u, tol, 100000, 0, c, nullptr);
  if (!rc && cudaStreamSynchronize(pl->stream) != cudaSuccess) rc = NUFFT_ECUDA;
  nufft_plan_destroy(pl);
  return rc;
}

}  // extern "C"
