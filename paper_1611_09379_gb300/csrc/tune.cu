// Empirical parameter choice (autotuner) for the FMM of Sec. 2.1 on a given
// point set.  The paper fixes l_max by balancing the near field against the
// translations (Eq. 23-25, empirical l* = 5 sources per box in log2 units,
// Sec. 3.2) and p, q by the error bounds of Eq. 18.2; both are worst-case
// estimates.  This measures instead: it times the requested exec sequence
// for candidate parameter sets on the caller's points with probe data, and
// keeps the fastest one whose result stays within the accuracy target of a
// reference computed by the FP64 FMM at eps = 1e-15.
//
// Search (coordinate descent, 10 to 40 candidates):
//   1. l_max in {l0 - 1, l0, l0 + 1}, l0 from Eq. 25, p and q from Eq. 18.2;
//   2. p lowered in steps of 2 while the result stays accurate;
//   3. q lowered in steps of 1 likewise;
//   4. mixed precision: the first tensor-core level (tc_level), every level
//      from max(4, l_max - 9) to l_max and "never";
//   5. l_max again, one level at a time away from the best depth while that
//      gains, at the lowered p (or p + 2) and q and the chosen tensor-core
//      level's distance from the leaves;
//   6. mixed batches of 64 signals: the near field on the tensor cores or not.
// A candidate is accurate when every output's relative L2 error is at most
// max(eps / 4, min(1.5 x that of the formula's parameters, eps / 2)): tuning
// keeps a plan within eps / 2, and within eps / 4 or the paper's choice.  Errors: the
// forward and adjoint against the reference FMM; the inverse, when timed
// with the forward, as the round trip inv(fwd(c)) against c itself (the
// pipeline's error, including the inverse's conditioning), else against the
// reference inverse.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "common.cuh"

using namespace nufft;

namespace {

constexpr int kErrBlocks = 512;

// probe values: components uniform in [-1, 1), exactly representable in
// FP32 (so complex64 and complex128 copies hold the same numbers), from a
// counter-based hash (SplitMix64 finaliser) of the element index
__device__ inline float probe_unit(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (float)((int64_t)(x >> 40) - (int64_t(1) << 23)) * (1.0f / (float)(1 << 23));
}

__global__ void k_probe(double2* __restrict__ d, float2* __restrict__ f, int64_t n, uint64_t seed) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float re = probe_unit(seed + 2 * (uint64_t)i), im = probe_unit(seed + 2 * (uint64_t)i + 1);
  d[i] = make_double2(re, im);
  f[i] = make_float2(re, im);
}

// partial sums of |a - ref|^2 and |ref|^2 (a complex64 or complex128)
__global__ void __launch_bounds__(256) k_err_partial(const void* __restrict__ a, int a64,
                                                     const double2* __restrict__ ref, int64_t n,
                                                     double2* __restrict__ partial) {
  __shared__ double2 sh[256];
  double e = 0, r = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double2 v = a64 ? static_cast<const double2*>(a)[i]
                    : to_d2(static_cast<const float2*>(a)[i]);
    double2 w = ref[i];
    double dx = v.x - w.x, dy = v.y - w.y;
    e += dx * dx + dy * dy;
    r += w.x * w.x + w.y * w.y;
  }
  sh[threadIdx.x] = make_double2(e, r);
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < (unsigned)h) sh[threadIdx.x] = cadd(sh[threadIdx.x], sh[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// round complex128 samples to complex64 and back, so both element types
// hold the same numbers
__global__ void k_round_to(double2* __restrict__ d, float2* __restrict__ f, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float2 v = make_float2((float)d[i].x, (float)d[i].y);
  f[i] = v;
  d[i] = make_double2(v.x, v.y);
}

struct Buffers {
  // probe inputs (both element types), reference and candidate outputs
  double2 *c_d = nullptr, *g_d = nullptr, *gi_d = nullptr;
  float2 *c_f = nullptr, *g_f = nullptr, *gi_f = nullptr;
  double2 *ref_g = nullptr, *ref_a = nullptr, *ref_i = nullptr;
  void *out_g = nullptr, *out_a = nullptr, *out_i = nullptr;
  double2* partial = nullptr;
  ~Buffers() {
    void* ps[] = {c_d, g_d, gi_d, c_f, g_f, gi_f, ref_g, ref_a, ref_i, out_g, out_a, out_i, partial};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
};

struct Tuner {
  int64_t N, M;
  const double* y;
  double eps;
  int prec;
  unsigned flags;
  int batch;
  unsigned ops;
  int reps;
  cudaStream_t st;
  Buffers buf;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double def_err[3] = {0, 0, 0};   // errors of the formula parameters (fwd, adj, inv)
  double last_err[3] = {0, 0, 0};  // errors of the last candidate evaluated
  std::vector<nufft_tune_trial> log;

  ~Tuner() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }

  bool io64() const { return !(flags & NUFFT_IO_C64); }

  // The exec sequence.  A candidate's inverse, timed together with its
  // forward, takes that forward's output (the round trip of the pipeline);
  // otherwise it takes the reference forward's samples of the probe series.
  int run(nufft_plan pl, bool reference, void* og, void* oa, void* oi) {
    const bool d = reference || io64();
    int rc = NUFFT_OK;
    if (ops & NUFFT_OP_FWD)
      rc = nufft_plan_exec_fwd(pl, d ? (void*)buf.c_d : (void*)buf.c_f, og);
    if (!rc && (ops & NUFFT_OP_ADJ))
      rc = nufft_plan_exec_adj(pl, d ? (void*)buf.g_d : (void*)buf.g_f, oa);
    if (!rc && (ops & NUFFT_OP_INV)) {
      const void* gin = (!reference && (ops & NUFFT_OP_FWD)) ? og
                        : (d ? (void*)buf.gi_d : (void*)buf.gi_f);
      rc = nufft_plan_exec_inv(pl, gin, oi);
    }
    return rc;
  }

  // relative L2 difference of a (complex64 or complex128) to ref
  int rel_err(const void* a, int a64, const double2* ref, int64_t n, double* err) {
    k_err_partial<<<kErrBlocks, 256, 0, st>>>(a, a64, ref, n, buf.partial);
    std::vector<double2> h(kErrBlocks);
    if (cudaMemcpyAsync(h.data(), buf.partial, kErrBlocks * sizeof(double2), cudaMemcpyDeviceToHost,
                        st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return NUFFT_ECUDA;
    double e2 = 0, r2 = 0;
    for (const double2& v : h) { e2 += v.x; r2 += v.y; }
    *err = r2 > 0 ? std::sqrt(e2 / r2) : std::sqrt(e2);
    return NUFFT_OK;
  }

  unsigned plan_flags() const { return flags | ((ops & NUFFT_OP_INV) ? NUFFT_WANT_INVERSE : 0u); }

  int setup() {
    const int64_t nc = (int64_t)batch * N, ng = (int64_t)batch * M;
    const size_t csz = io64() ? 16 : 8;
    if (cudaMalloc(&buf.c_d, nc * 16) != cudaSuccess || cudaMalloc(&buf.c_f, nc * 8) != cudaSuccess ||
        cudaMalloc(&buf.g_d, ng * 16) != cudaSuccess || cudaMalloc(&buf.g_f, ng * 8) != cudaSuccess ||
        cudaMalloc(&buf.gi_d, ng * 16) != cudaSuccess || cudaMalloc(&buf.gi_f, ng * 8) != cudaSuccess ||
        cudaMalloc(&buf.ref_g, ng * 16) != cudaSuccess || cudaMalloc(&buf.ref_a, nc * 16) != cudaSuccess ||
        cudaMalloc(&buf.ref_i, nc * 16) != cudaSuccess || cudaMalloc(&buf.out_g, ng * csz) != cudaSuccess ||
        cudaMalloc(&buf.out_a, nc * csz) != cudaSuccess || cudaMalloc(&buf.out_i, nc * csz) != cudaSuccess ||
        cudaMalloc(&buf.partial, kErrBlocks * sizeof(double2)) != cudaSuccess)
      return NUFFT_ENOMEM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return NUFFT_ECUDA;
    k_probe<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(buf.c_d, buf.c_f, nc, 1000);
    k_probe<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(buf.g_d, buf.g_f, ng, 1ull << 40);
    // reference: the FP64 FMM at eps = 1e-15 (complex128 in and out)
    nufft_params rp{0, 0, 0, batch, -1, -1};
    nufft_plan ref = nullptr;
    int rc = nufft_plan_create(&ref, N, M, y, 1e-15, NUFFT_FP64, &rp,
                               (ops & NUFFT_OP_INV) ? NUFFT_WANT_INVERSE : 0u, st);
    if (rc) return rc;
    if ((ops & NUFFT_OP_INV)) {
      // the inverse acts on samples of a band-limited series: g = A c
      rc = nufft_plan_exec_fwd(ref, buf.c_d, buf.gi_d);
      if (!rc) {
        k_round_to<<<(unsigned)((ng + 255) / 256), 256, 0, st>>>(buf.gi_d, buf.gi_f, ng);
      }
    }
    if (!rc) rc = run(ref, true, buf.ref_g, buf.ref_a, buf.ref_i);
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = NUFFT_ECUDA;
    nufft_plan_destroy(ref);
    return rc;
  }

  // one candidate: plan, warm-up, `reps` timed runs (median), error
  int eval(nufft_params prm, nufft_tune_trial* out, bool* valid) {
    *valid = false;
    nufft_plan pl = nullptr;
    int rc = nufft_plan_create(&pl, N, M, y, eps, prec, &prm, plan_flags(), st);
    if (rc == NUFFT_EINVAL || rc == NUFFT_ENOTSUP) return NUFFT_OK;  // not a valid combination
    if (rc) return rc;
    nufft_plan_params(pl, &out->params);
    rc = run(pl, false, buf.out_g, buf.out_a, buf.out_i);
    std::vector<float> ms;
    for (int r = 0; !rc && r < reps; ++r) {
      cudaEventRecord(e0, st);
      rc = run(pl, false, buf.out_g, buf.out_a, buf.out_i);
      cudaEventRecord(e1, st);
      float t = 0;
      if (!rc && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        rc = NUFFT_ECUDA;
      ms.push_back(t);
    }
    if (!rc) rc = nufft_plan_sync(pl);
    // per output: forward vs the reference forward, adjoint vs the reference
    // adjoint, inverse vs the probe coefficients themselves (round trip, when
    // timed with the forward) or vs the reference inverse
    const int a64 = io64();
    const int64_t nc = (int64_t)batch * N, ng = (int64_t)batch * M;
    double e[3] = {0, 0, 0};
    if (!rc && (ops & NUFFT_OP_FWD)) rc = rel_err(buf.out_g, a64, buf.ref_g, ng, &e[0]);
    if (!rc && (ops & NUFFT_OP_ADJ)) rc = rel_err(buf.out_a, a64, buf.ref_a, nc, &e[1]);
    if (!rc && (ops & NUFFT_OP_INV))
      rc = rel_err(buf.out_i, a64, (ops & NUFFT_OP_FWD) ? buf.c_d : buf.ref_i, nc, &e[2]);
    nufft_plan_destroy(pl);
    if (rc) return rc;
    std::sort(ms.begin(), ms.end());
    out->ms = ms[ms.size() / 2];
    out->err = std::max(e[0], std::max(e[1], e[2]));
    for (int i = 0; i < 3; ++i) last_err[i] = e[i];
    out->accepted = 0;
    *valid = true;
    return NUFFT_OK;
  }

  // every output within max(eps / 4, min(1.5 x the formula parameters'
  // error, eps / 2))
  bool accurate() const {
    for (int i = 0; i < 3; ++i)
      if (last_err[i] > std::max(0.25 * eps, std::min(1.5 * def_err[i], 0.5 * eps))) return false;
    return true;
  }

  // evaluate, log, and keep if accurate and faster than *best
  int try_params(nufft_params prm, nufft_tune_trial* best, bool* took, bool* acc = nullptr) {
    nufft_tune_trial t{};
    bool valid = false;
    *took = false;
    if (acc) *acc = false;
    int rc = eval(prm, &t, &valid);
    if (rc || !valid) return rc;
    const bool ok = accurate();
    if (acc) *acc = ok;
    if (ok && (best->ms <= 0 || t.ms < best->ms)) {
      *best = t;
      *took = true;
    }
    log.push_back(t);
    return NUFFT_OK;
  }
};

}  // namespace

extern "C" int nufft_autotune(int64_t N, int64_t M, const double* y, double eps, int prec,
                              unsigned flags, int batch, unsigned ops, int reps, nufft_params* best,
                              nufft_tune_trial* trials, int max_trials, int* n_trials,
                              void* stream) {
  if (!y || !best || ops == 0 || (ops & ~(NUFFT_OP_FWD | NUFFT_OP_ADJ | NUFFT_OP_INV)) ||
      (flags & ~NUFFT_IO_C64) || reps < 1 || batch < 1 || (max_trials > 0 && !trials))
    return NUFFT_EINVAL;
  if ((ops & NUFFT_OP_INV) && M != N) return NUFFT_EINVAL;
  // machine precision (eps = 0, FP64): tune against the threshold error
  if (eps == 0.0 && prec == NUFFT_FP64) eps = nufft_eps_threshold(N);
  nufft_params d0{0, 0, 0, batch, 0, 0};
  int rc = nufft_choose_params(N, M, eps, prec, &d0);
  if (rc) return rc;
  Tuner tu;
  tu.N = N; tu.M = M; tu.y = y; tu.eps = eps; tu.prec = prec; tu.flags = flags;
  tu.batch = batch; tu.ops = ops; tu.reps = reps; tu.st = (cudaStream_t)stream;
  if ((rc = tu.setup())) return rc;

  // the formula's parameters first: their error sets the accuracy floor
  nufft_tune_trial cur{};
  bool valid = false, took = false, acc = false;
  if ((rc = tu.eval(d0, &cur, &valid))) return rc;
  if (!valid) return NUFFT_EINVAL;
  for (int i = 0; i < 3; ++i) tu.def_err[i] = tu.last_err[i];
  cur.accepted = 1;
  tu.log.push_back(cur);
  nufft_tune_trial bestt = cur;

  int LN = 0;
  while ((int64_t(1) << LN) < N) ++LN;
  // 1. tree depth (p, q from Eq. 18.2 for that depth; tc_level automatic)
  const int L0 = d0.lmax;
  for (int L : {L0 - 1, L0 + 1}) {
    if (L < 2 || L > LN) continue;
    nufft_params prm{L, 0, 0, batch, 0, 0};
    if ((rc = tu.try_params(prm, &bestt, &took))) return rc;
  }
  // 2. expansion order p, 3. regular-series order q
  {
    const nufft_params base = bestt.params;
    for (int dp = 2; dp <= 40; dp += 2) {
      nufft_params prm = base;
      prm.p = base.p - dp;
      prm.tc_level = 0;
      if (prm.p < 4) break;
      if ((rc = tu.try_params(prm, &bestt, &took, &acc))) return rc;
      if (!acc) break;
    }
  }
  {
    const nufft_params base = bestt.params;
    for (int dq = 1; dq <= 20; ++dq) {
      nufft_params prm = base;
      prm.q = base.q - dq;
      prm.tc_level = 0;
      if (prm.q < 2) break;
      if ((rc = tu.try_params(prm, &bestt, &took, &acc))) return rc;
      if (!acc) break;
    }
  }
  // 4. first tensor-core level (mixed precision)
  if (prec == NUFFT_MIXED) {
    const nufft_params base = bestt.params;
    const int Lb = base.lmax;
    std::vector<int> levels{-1};
    for (int l = std::max(4, Lb - 9); l <= Lb; ++l)
      if (l != base.tc_level) levels.push_back(l);
    for (int l : levels) {
      nufft_params prm = base;
      prm.tc_level = l;
      if ((rc = tu.try_params(prm, &bestt, &took))) return rc;
    }
  }
  // 5. tree depth again at the lowered orders (the formula's p grows with
  // the depth, so step 1 compared depths at orders that steps 2-3 then
  // lowered): one level at a time away from the best depth while that
  // gains, with the chosen tensor-core level kept at the same distance from
  // the leaves (or none), and p + 2 when p alone is not accurate there
  {
    const nufft_params b0 = bestt.params;
    for (int dir : {+1, -1}) {
      bool gained = false;
      for (int L = b0.lmax + dir; L >= 2 && L <= LN; L += dir) {
        bool any = false;
        for (int dp = 0; dp <= 2 && !any; dp += 2) {
          nufft_params prm = bestt.params;
          prm.lmax = L;
          prm.p = bestt.params.p + dp;
          if (prm.tc_level > 0) prm.tc_level += L - bestt.params.lmax;
          if ((rc = tu.try_params(prm, &bestt, &took, &acc))) return rc;
          any = took;
          if (acc) break;  // accurate but slower: a larger p will not be faster
        }
        if (!any) break;
        gained = true;
      }
      if (gained) break;
    }
  }
  if (prec == NUFFT_MIXED) {
    // 6. near field of batched forwards on the tensor cores, or not
    if (batch % 64 == 0 && (ops & NUFFT_OP_FWD)) {
      nufft_params prm = bestt.params;
      prm.tc_near = bestt.params.tc_near > 0 ? -1 : 1;
      if ((rc = tu.try_params(prm, &bestt, &took))) return rc;
    }
  }
  *best = bestt.params;
  for (nufft_tune_trial& t : tu.log)
    t.accepted = (t.params.lmax == bestt.params.lmax && t.params.p == bestt.params.p &&
                  t.params.q == bestt.params.q && t.params.tc_level == bestt.params.tc_level &&
                  t.params.tc_near == bestt.params.tc_near)
                     ? 1 : 0;
  if (n_trials) *n_trials = (int)tu.log.size();
  for (int i = 0; i < max_trials && i < (int)tu.log.size(); ++i) trials[i] = tu.log[i];
  return NUFFT_OK;
}
