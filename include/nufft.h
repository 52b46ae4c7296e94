/*
 * nufft.h - C ABI of the GB300 (sm_103a) FMM-based NUFFT / INUFFT library.
 *
 * Method: Gumerov & Duraiswami, "Fast Multipole Method based filtering of
 * non-uniformly sampled data".  A 2 pi-periodic band-limited function
 *     f(x) = sum_{n=0}^{N-1} c_n e^{i n x}                        (Eq. p1)
 * is sampled on the uniform grid x_k = 2 pi k / N (f_k) and at M non-uniform
 * points y_j in [0, 2 pi) (g_j).  The library computes
 *   forward  (problem (i), Sec. 2):   c_n -> g_j = f(y_j)
 *            via f = IDFT(c) and g_j = F_j sum_k G(y_j - x_k) f_k   (Eq. p4, p5)
 *   adjoint:                          g_j -> c'_n = sum_j e^{-i n y_j} g_j
 *   inverse  (problem (ii), M = N):   g_j -> c_n with f(y_j) = g_j
 *            via f_k = C_k sum_j G(x_k - y_j) D_j g_j             (Eq. p6, p8)
 * where G(t) = 1/(e^{it} - 1) = -(1 + i cot(t/2))/2, and every matrix-vector
 * product with G runs through a multilevel FMM on the circle (Sec. 2.1-2.3).
 *
 * Conventions for every call below
 *   - Data pointers marked [device] are CUDA device pointers owned by the
 *     caller; [host] pointers are ordinary host memory.  The library never
 *     frees or retains caller pointers beyond the call.
 *   - Complex data are interleaved (re, im).  Element type: complex128
 *     (2 x double) unless the plan was created with NUFFT_IO_C64, then
 *     complex64 (2 x float).
 *   - Frequencies are one-sided, n = 0..N-1 (Eq. p1).
 *   - N (the number of coefficients) is any integer 8 <= N <= 2^26;
 *     1 <= M <= 2^27.  The FMM and its FFT run on the grid of
 *     N' = 2^ceil(log2 N) points: the series of Eq. p1 with N terms is the
 *     series with N' terms whose top N' - N coefficients are zero, so the
 *     forward, adjoint and least-squares results are the same sums (inputs
 *     are zero padded and outputs truncated inside the FFT passes).  The
 *     square inverse evaluates its interpolant (Eq. p6 / p8 with N points)
 *     at the N' grid points, whose N'-point DFT gives the N coefficients.
 *     Grid quantities of a plan (leaves, k0, delta, C_k) are on the N' grid.
 *   - y_j must be finite and in [0, 2 pi) (binary64 2 pi excluded).
 *   - All work is enqueued on the plan's CUDA stream and is asynchronous;
 *     a return of NUFFT_OK means the work was enqueued without error.
 *     Calls that must inspect device results (plan creation validates y)
 *     synchronise the stream and say so.
 *   - Every function returns a nufft_status; it never aborts the process.
 */
#ifndef NUFFT_GB300_H
#define NUFFT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NUFFT_OK = 0,
  NUFFT_EINVAL = 1,     /* bad argument: N not a power of two, y out of range, ... */
  NUFFT_ENOMEM = 2,     /* device or host allocation failed */
  NUFFT_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  NUFFT_EILLCOND = 4,   /* inverse coefficients out of range / duplicate points */
  NUFFT_ENOTCONV = 5,   /* iterative solve did not reach the tolerance */
  NUFFT_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  NUFFT_ENOTSUP = 7     /* combination of options not supported */
} nufft_status;

/* Arithmetic of the FMM (the far field: P2M, M2M, M2L, L2L, L2P and the
 * level-2 regular part).  F_j, C_k, D_j and the near-field singular pair are
 * always formed in FP64. */
typedef enum {
  NUFFT_FP64 = 0,   /* everything in binary64; target rel. L2 error ~ eps (1e-12) */
  NUFFT_MIXED = 1   /* far field and near field in binary32 (FP64 F_j and
                       singular pair); target rel. L2 error ~ eps (1e-6) */
} nufft_prec;

/* plan flags */
#define NUFFT_IO_C64 0x1u        /* caller data are complex64 instead of complex128 */
#define NUFFT_WANT_INVERSE 0x2u  /* precompute C_k, D_j (Eq. p8) for exec_inv (M == N) */
#define NUFFT_NO_GRAPH 0x4u      /* launch exec kernels one by one (no CUDA graph replay) */
#define NUFFT_ADAPTIVE 0x8u      /* leaves holding more points than the mean are
                                    refined (non-uniform tree depth, see
                                    nufft_adaptive_depths); one signal (batch 1) */

/* Opaque plan: the "data structure" of the paper (Sec. 3.3): the binned point
 * set, F_j, optionally C_k / D_j, the expansion workspace and the FMM
 * operators.  Owns its device memory. */
typedef struct nufft_plan_s *nufft_plan;

/* FMM parameters.  Any field <= 0 is chosen automatically:
 *   lmax: tree depth, default max(2, round(log2 sqrt(N M)) - 5) (Eq. 25 with
 *         the empirical l* = 5 of Sec. 3.2)
 *   p:    1/t MLFMM truncation number, q: regular-series truncation number,
 *         both from Eq. 18.2 with the fraction read as 10/(3 pi eps)
 *   batch: number of signals sharing the point set (default 1); exec calls
 *         then take [batch][N] coefficients and [batch][M] samples
 *   tc_level: first tree level whose M2L + L2L (Sec. 2.1) runs as a dense
 *         GEMM on the tensor cores (three TF32 passes, FP32 accumulation;
 *         NUFFT_MIXED with p <= 24 only); coarser levels use the FP32 SIMT
 *         kernels.  0 = automatic (the finest levels holding at least 2048
 *         parent boxes over all signals), -1 = never.  Reported back as -1
 *         when no level qualifies.
 *   tc_near: near field of batched forward transforms as a dense GEMM on
 *         the tensor cores (kernel values x window samples of 64 signals per
 *         tile, three TF32 passes; NUFFT_MIXED with batch a multiple of 64
 *         only).  0 = automatic (on where allowed), -1 = never, 1 = where
 *         allowed.  Reported back as 1 or -1.
 * Constraints: 2 <= lmax <= log2 N, 4 <= p <= 64, 2 <= q <= 32,
 * batch <= 4096, tc_level -1, 0 or in [4, 30], tc_near -1, 0 or 1. */
typedef struct {
  int lmax;
  int p;
  int q;
  int batch;
  int tc_level;
  int tc_near;
} nufft_params;

/* ---------------------------------------------------------------- host only */

/* Human-readable text for a status code (static storage). */
const char *nufft_strerror(int status);

/* Library version as 10000*major + 100*minor + patch. */
int nufft_version(void);

/* Parameter choice of a plan without creating it (no GPU needed); the tree
 * depth refers to the grid N' = 2^ceil(log2 N).
 * in/out: *params (fields <= 0 are filled in).  Returns NUFFT_EINVAL for an
 * invalid N, M, eps or prec.  eps must lie in [1e-15, 1e-1], or be 0 with
 * NUFFT_FP64: machine precision, the threshold error nufft_eps_threshold(N)
 * taken as the prescribed accuracy (the second setting of Sec. 3.2); every
 * call that takes eps accepts the same values. */
int nufft_choose_params(int64_t N, int64_t M, double eps, int prec,
                        nufft_params *params);

/* Threshold ("machine precision") error eps_th(N) of the FP64 path (Sec.
 * 3.1): the value at which the error of the paper's f = 1 test, max_j
 * |g_j - 1|, stops falling as eps is lowered, modelled as log2(N') 2^-53
 * (measured on GB300 for N = 2^8 .. 2^22 with uniform points: 0.8e-15 ..
 * 2.2e-15, each within 20 % below the model), at least 1e-15.  The
 * straightforward method of Sec. 3.1 (Eq. p4 in plain binary64) has a far
 * larger threshold; this one comes from the exact grid coordinates.  Returns
 * -1 for N outside [8, 2^26].  Host only. */
double nufft_eps_threshold(int64_t N);

/* Adaptive tree depth (plan flag NUFFT_ADAPTIVE).  The tree of Sec. 2.1 is
 * uniform: every target meets the 3 s grid points of its leaf and the two
 * adjacent ones (s = N' >> lmax), so the near field (Sec. 2.4, 3 N M / 2^lmax
 * pairs) costs the same per target however the points cluster, while a
 * leaf in a cluster holds many more targets than grid points.  A refined
 * leaf b takes d_b more levels: its targets' local expansions come from the
 * downward pass continued to level lmax + d_b (L2L of the parent plus the
 * M2L of the interaction list, whose multipoles are formed from the grid
 * samples: the sources are the uniform grid at every level) and their near
 * field from the 3 boxes of that level (3 s / 2^d_b grid points).  The
 * adjoint and the inverse take the same leaves' points as sources: near
 * field from the 3 boxes of level lmax + d_b, and the grid boxes of the
 * interaction lists of their boxes at levels lmax + 1 .. lmax + d_b through
 * those boxes' multipoles (M2L into the grid boxes, evaluated at the grid
 * points).
 * The depth of leaf b from its target count n_b and the mean nbar = M / B:
 *   d_b = the largest d <= dmax with n_b >= 2^d nbar,
 *   dmax = min(3, log2(s) - 3) (a refined box keeps at least 8 grid points).
 * in: leaf_start[B + 1] (host; n_b = leaf_start[b + 1] - leaf_start[b]), B a
 * power of two, M = leaf_start[B], s a power of two.  out: depth[B] (host).
 * Returns max_b d_b, or -1 for invalid arguments.  Host only. */
int nufft_adaptive_depths(const int32_t *leaf_start, int64_t B, int64_t M, int s, int *depth);

/* Refinement of a plan created with NUFFT_ADAPTIVE: *levels = max_b d_b (0:
 * the uniform tree, e.g. for uniform points, or a plan without the flag);
 * count[d] = the points whose leaf has d_b = d, d = 0..3.  Host only. */
int nufft_plan_adaptive(nufft_plan pl, int *levels, int64_t count[4]);

/* ---------------------------------------------------------------- autotuner */

/* Exec calls an autotuning run times together (bit mask). */
#define NUFFT_OP_FWD 0x1u  /* nufft_plan_exec_fwd */
#define NUFFT_OP_ADJ 0x2u  /* nufft_plan_exec_adj */
#define NUFFT_OP_INV 0x4u  /* nufft_plan_exec_inv (needs M == N) */

/* One candidate of an autotuning run. */
typedef struct {
  nufft_params params;  /* resolved parameters of the candidate */
  double ms;            /* median time of one pass of the exec sequence */
  double err;           /* largest relative L2 error over the outputs */
  int accepted;         /* 1 for the returned choice */
} nufft_tune_trial;

/* Empirical choice of lmax, p, q and tc_level for one point set (no
 * counterpart in the paper, which fixes lmax by the cost balance of Eq.
 * 23-25 with l* = 5 and p, q by the error bound of Eq. 18.2).  Times the
 * exec sequence `ops` (NUFFT_OP_* mask) on probe data for 10 to 40 candidate
 * parameter sets, each through a plan of its own, and returns the fastest
 * whose every output has a relative L2 error of at most max(eps / 4,
 * min(1.5 x the formula parameters' error, eps / 2)): forward and adjoint
 * against the FP64 FMM
 * at eps = 1e-15, the inverse (when timed with the forward) as the round
 * trip inv(fwd(c)) against the probe coefficients c.  Search:
 * lmax in {l0 - 1, l0, l0 + 1}; p lowered in steps of 2 and q in steps of 1
 * while accurate; for NUFFT_MIXED every tc_level from max(4, lmax - 9) to
 * lmax and -1; lmax again, one level at a time while that gains, at the
 * lowered p (or p + 2) and q; for batches of 64 signals tc_near on and off.
 *   N, M, y [device], eps, prec, flags (0 or NUFFT_IO_C64), batch: as for
 *          nufft_plan_create (y is read during the call only)
 *   ops    NUFFT_OP_FWD | NUFFT_OP_ADJ | NUFFT_OP_INV (INV needs M == N)
 *   reps   timed repetitions per candidate (>= 1; one untimed run first)
 *   best   [host] receives the chosen parameters (pass them to
 *          nufft_plan_create)
 *   trials [host] optional log of up to max_trials candidates in the order
 *          tried; n_trials [host, optional] receives the number tried
 * Synchronous on `stream`; allocates probe and reference buffers of
 * (batch x max(N, M)) complex values for the duration of the call.  Errors:
 * as nufft_plan_create (EILLCOND for an inverse on duplicate points), EINVAL
 * for a bad ops mask / reps / batch. */
int nufft_autotune(int64_t N, int64_t M, const double *y, double eps, int prec,
                   unsigned flags, int batch, unsigned ops, int reps,
                   nufft_params *best, nufft_tune_trial *trials, int max_trials,
                   int *n_trials, void *stream);

/* ---------------------------------------------------------------- plans */

/* Build a plan: validate y, bin it into the 2^lmax leaves of the binary tree
 * on the circle by a stable counting sort (Sec. 2.1, "setting the data
 * structure", Sec. 3.3), precompute F_j (Eq. p5) and, with
 * NUFFT_WANT_INVERSE, the log-sums behind C_k and D_j (Eq. p8).
 *   out     [host]   receives the plan
 *   N, M             number of coefficients (the grid is N' = 2^ceil(log2 N)) and
 *                    number of points
 *   y       [device] M binary64 points in [0, 2 pi); read during the call only
 *   eps              requested accuracy in [1e-15, 1e-1]
 *   prec             nufft_prec
 *   params  [host]   optional overrides (NULL = automatic)
 *   flags            NUFFT_IO_C64 | NUFFT_WANT_INVERSE | NUFFT_NO_GRAPH |
 *                    NUFFT_ADAPTIVE (one-signal plans: forward, adjoint
 *                    and inverse on the adaptive tree)
 * Exec calls replay a CUDA graph of their kernel sequence, captured on the
 * first call with the same operation and buffer pointers (up to 8 kept per
 * plan); they launch kernels one by one instead while profiling is enabled,
 * while the stream is being captured by the caller, or with NUFFT_NO_GRAPH.
 *   stream           cudaStream_t to run on (NULL = legacy default stream)
 * Synchronises the stream (it reads back validation flags).  Errors:
 * EINVAL (bad sizes / eps / y), EILLCOND (inverse requested with duplicate
 * points or coefficients outside the exponent range), ENOTSUP
 * (NUFFT_ADAPTIVE with batch > 1), ENOMEM, ECUDA. */
int nufft_plan_create(nufft_plan *out, int64_t N, int64_t M, const double *y,
                      double eps, int prec, const nufft_params *params,
                      unsigned flags, void *stream);

/* Release the plan and its device memory (synchronises its stream). */
int nufft_plan_destroy(nufft_plan plan);

/* Report the parameters in use (any output pointer may be NULL). */
int nufft_plan_info(nufft_plan plan, int *lmax, int *p, int *q);

/* All parameters of the plan (the resolved nufft_params).  out [host]. */
int nufft_plan_params(nufft_plan plan, nufft_params *out);

/* Wait for the plan's stream and read its device status word: returns
 * NUFFT_ETIMEOUT if a kernel's bounded wait on the tensor cores gave up since
 * the last call (its outputs are then invalid; the word is cleared), else
 * NUFFT_OK.  Exec calls never block, so they cannot report this themselves. */
int nufft_plan_sync(nufft_plan plan);

/* Copy the plan's binned point set (the stable counting sort of Sec. 2.1)
 * into caller buffers, for inspection and tests.  Any pointer may be NULL.
 *   perm       [device] int32[M]   original index of the i-th sorted point
 *   leaf_start [device] int32[B+1] first sorted index of each leaf, B = 2^lmax
 *   k0         [device] int32[M]   nearest grid index round(y N' / 2 pi) mod N'
 *   delta      [device] double[M]  y N' / (2 pi) - round(y N' / 2 pi)
 * Asynchronous on the plan's stream. */
int nufft_plan_points(nufft_plan plan, int32_t *perm, int32_t *leaf_start,
                      int32_t *k0, double *delta);

/* Copy the inverse coefficients of a plan made with NUFFT_WANT_INVERSE.
 * With lamC_k = sum_l log|2 sin((x_k - y_l)/2)|, lamD_j = -sum_{l!=j}
 * log|2 sin((y_j - y_l)/2)|, nC_k = #{l: y_l > x_k}, nD_j = #{l: y_l > y_j}:
 *   Ct     [device] double[N']  (-1)^(k + nC_k) e^{lamC_k + Lambda} / N'
 *                               (0 where a point sits exactly on x_k); for
 *                               N < N' the sign is (-1)^(nC_k) and C_k has
 *                               the further phase e^{i pi k N / N'}
 *   Dt     [device] double2[M]  (-1)^nD_j e^{lamD_j - Lambda} i e^{-i N y_j/2}
 *                               (sorted point order, see nufft_plan_points)
 *   Lambda [host]   the common scale, the midpoint of the range of lamD
 * so that N Ct_k Dt_j = C_k D_j of Eq. p8.  Any pointer may be NULL.
 * Synchronises the stream when Lambda is requested. */
int nufft_plan_inverse_coeffs(nufft_plan plan, double *Ct, double *Dt, double *Lambda);

/* Change the stream later calls are enqueued on. */
int nufft_plan_set_stream(nufft_plan plan, void *stream);

/* Forward NUFFT (problem (i)): g_j = sum_n c_n e^{i n y_j}.
 *   c [device] batch x N coefficients, g [device] batch x M outputs (original
 *   point order), signal-major.
 * c and g must not overlap.  Asynchronous. */
int nufft_plan_exec_fwd(nufft_plan plan, const void *c, void *g);

/* Adjoint NUFFT: c_n = sum_j e^{-i n y_j} g_j (conjugate transpose of the
 * forward map; the FMM runs with sources and targets exchanged, Sec. 2.1).
 *   g [device] batch x M inputs, c [device] batch x N outputs.  Asynchronous. */
int nufft_plan_exec_adj(nufft_plan plan, const void *g, void *c);

/* Square inverse NUFFT (problem (ii), M == N): the unique band-limited c
 * with sum_n c_n e^{i n y_j} = g_j, by the Lagrange form Eq. p6 / p8
 * followed by the DFT of Eq. p1.  Needs NUFFT_WANT_INVERSE.
 *   g [device] batch x M inputs, c [device] batch x N outputs.  Asynchronous. */
int nufft_plan_exec_inv(nufft_plan plan, const void *g, void *c);

/* Least-squares INUFFT for M > N (problem (ii) of Sec. 2 with more samples
 * than coefficients; the paper states the problem, the CG solver is this
 * library's): c = argmin sum_j |sum_n c_n e^{i n y_j} - g_j|^2 by conjugate
 * gradients on the normal equations A^H A c = A^H g, A_jn = e^{i n y_j}, each
 * product being one forward and one adjoint FMM of the plan.
 * Weights w (density compensation, e.g. nufft_plan_dcf_weights):
 *   mode 0 (default): w preconditions the same equations (the solution does
 *     not change).  A^H A acts on coefficients like a product with the
 *     sample density in x (its Toeplitz symbol), so P = F diag(wt) F^H with
 *     wt_k the weights carried to the grid points (mean of w_j over the
 *     points whose nearest grid point is k; empty grid points take the
 *     nearest occupied one's) is close to its inverse; CG runs on P A^H A.
 *   NUFFT_LSQ_WEIGHTED: CG on the weighted equations A^H W A c = A^H W g
 *     instead (the minimiser of sum_j w_j |(A c)_j - g_j|^2, which is the
 *     same c only for consistent data).
 * Stopping test, the same in every mode: the residual of the UNWEIGHTED
 * normal equations, ||A^H (g - A c)|| / ||A^H g|| <= tol, recomputed from
 * the iterate c (one forward and one adjoint FMM) every `check_every`
 * iterations (0 = 16) and after the last one.
 *   g      [device] M samples (complex128, original point order)
 *   w      [device] float[M] positive weights (original order), NULL = plain CG
 *   mode   0 or NUFFT_LSQ_WEIGHTED
 *   tol    tolerance of the stopping test above
 *   maxit  iteration cap
 *   c      [device] N coefficients out (complex128)
 *   info   [host, optional] what the solve did:
 *            iters       CG iterations run
 *            checks      evaluations of the stopping test
 *            resid       the stopping test's value at the end
 *            resid_w     the residual of the system CG iterates on, from
 *                        its recurrence, relative to its right-hand side,
 *                        at the last test (unweighted equations in mode 0)
 *            data_resid  ||g - A c|| / ||g||, recomputed at the last test
 *            hist, hist_cap  (read on entry) optional host array of hist_cap
 *                        doubles: hist[i] receives the stopping test's value
 *                        at the i-th test (i < hist_cap)
 * Needs a complex128 plan with batch 1; use NUFFT_FP64 for tolerances below
 * ~1e-6.  Work vectors (6N + M complex and a few real arrays) are allocated
 * by the plan on first use.  Synchronises at every test.  Returns
 * NUFFT_ENOTCONV when maxit is reached first (c then holds the last
 * iterate); g with A^H g = 0 gives c = 0 and NUFFT_OK. */
#define NUFFT_LSQ_WEIGHTED 0x1u
typedef struct {
  int iters;
  int checks;
  double resid;
  double resid_w;
  double data_resid;
  double *hist;
  int hist_cap;
} nufft_lsq_info;
int nufft_plan_solve_lsq(nufft_plan plan, const void *g, const float *w, unsigned mode,
                         double tol, int maxit, int check_every, void *c, nufft_lsq_info *info);

/* ---------------------------------------------------------------- learned weights */

/* Density-compensation features of a plan's points, for the learned weights
 * of nufft_plan_solve_lsq: in periodic position order, the 8 gaps around
 * each point (ranks r-4..r+4), as log(gap M / N) with the gap in grid units
 * (scale free).  feat [device] float[M][8], original point order.
 * Synchronises the stream. */
int nufft_plan_dcf_features(nufft_plan plan, float *feat);

/* Training data for the network below.  y [device] double[S][M]: S point sets,
 * each sorted ascending in [0, 2 pi).
 * nufft_dcf_features_sorted: feat [device] float[S*M][8], the features above.
 * nufft_dcf_targets: logw [device] float[S*M] = log(w / mean w) (floored at
 *   log 1e-4) for the weights of the equations sum_j |D_N(y_i - y_j)|^2 w_j = N
 *   (D_N(t) = sum_{n<N} e^{int}), which make A^H W A closest to the identity in
 *   Frobenius norm, found by `iters` multiplicative fixed-point steps
 *   w_i <- w_i N / sum_j |D_N(y_i - y_j)|^2 w_j (they keep w positive; a direct
 *   solve is ill-conditioned and gives signed weights).  M <= 1024.
 * Both asynchronous. */
int nufft_dcf_features_sorted(const double *y, int64_t S, int64_t M, float *feat, void *stream);
int nufft_dcf_targets(const double *y, int64_t S, int64_t M, int64_t N, int iters,
                      float *logw, void *stream);

/* A density-compensation network w = softplus(MLP(feat)), MLP 8 -> 64 -> 64 -> 1
 * with GELU hidden layers; 4801 parameters laid out W1[64][8] b1[64]
 * W2[64][64] b2[64] W3[64] b3.  FP32 master weights for training; inference
 * uses the weights rounded to BF16 with FP32 accumulation.  The paper has no
 * learned component; it serves the least-squares solve above. */
typedef struct nufft_mlp_s *nufft_mlp;
int nufft_mlp_create(nufft_mlp *out);   /* all parameters zero */
int nufft_mlp_destroy(nufft_mlp mlp);
int nufft_mlp_num_params(void);
/* host float[4801]; reset_optimizer != 0 clears the Adam state */
int nufft_mlp_set_params(nufft_mlp mlp, const float *params, int reset_optimizer);
int nufft_mlp_get_params(nufft_mlp mlp, float *params);
/* w [device] float[n] = softplus(MLP(feat [device] float[n][8])); asynchronous */
int nufft_mlp_infer(nufft_mlp mlp, const float *feat, int64_t n, float *w, void *stream);
/* gradient of mean_i (log w_i - target_i)^2 w.r.t. the FP32 parameters:
 * grad [host] float[4801] and loss [host] (either may be NULL; synchronises
 * when one is given).  target [device] float[n] = log of the desired weights. */
int nufft_mlp_grad(nufft_mlp mlp, const float *feat, const float *target, int64_t n,
                   float *grad, float *loss, void *stream);
/* one Adam step (lr) on that loss; loss [host] optional (synchronises) */
int nufft_mlp_train_step(nufft_mlp mlp, const float *feat, const float *target, int64_t n,
                         float lr, float *loss, void *stream);

/* Learned weights of a plan's points for nufft_plan_solve_lsq: the features
 * of nufft_plan_dcf_features through the network's BF16 inference, scaled to
 * mean 1 on the device (the weights are scale free).  w [device] float[M],
 * original point order.  Asynchronous on the plan's stream except for the
 * feature step, which synchronises it. */
int nufft_plan_dcf_weights(nufft_plan plan, nufft_mlp mlp, float *w);

/* ---------------------------------------------------------------- profiling */

/* Stages of an evaluation, for nufft_plan_stats. */
enum {
  NUFFT_STAGE_FFT = 0,      /* c_n <-> f_k (Eq. p1) */
  NUFFT_STAGE_P2M = 1,      /* charges + leaf multipoles */
  NUFFT_STAGE_M2M = 2,      /* upward pass */
  NUFFT_STAGE_LEVEL2 = 3,   /* regular-part coefficients (Eq. p20) */
  NUFFT_STAGE_M2L = 4,      /* M2L + L2L, levels 3..lmax */
  NUFFT_STAGE_TARGETS = 5,  /* L2P + near field + regular part + F_j / C_k */
  NUFFT_STAGE_OTHER = 6,    /* self terms of the adjoint / inverse, packing, conversions */
  NUFFT_NSTAGES = 7
};

/* Enable (1) or disable (0) per-stage timing: when enabled, every exec call
 * records CUDA events around each stage on the plan's stream.  Enabling
 * resets the accumulated times and launch counts. */
int nufft_plan_profile(nufft_plan plan, int enable);

/* Accumulated device time (ms, from the CUDA events) and kernel launches per
 * stage since profiling was last enabled.  stage_ms [host] double[NUFFT_NSTAGES],
 * launches [host] int64[NUFFT_NSTAGES]; either may be NULL.  Synchronises the
 * stream.  Launch counts are kept even when timing is disabled. */
int nufft_plan_stats(nufft_plan plan, double *stage_ms, int64_t *launches);

/* ---------------------------------------------------------------- uneven batches */

/* Many independent forward transforms of uneven sizes, each with its own grid
 * size N[i], point count M[i] and points y[i] ([device] double[M[i]]), run as
 * one CUDA graph launch: every transform's kernel chain is captured on one of
 * several forked streams (independent transforms overlap) and the
 * instantiated graph is replayed while the caller's buffers stay the same.
 * The paper treats one transform at a time; this groups many.
 * nufft_multi_create builds one plan per transform (same eps, prec, flags;
 * NUFFT_WANT_INVERSE not supported) and synchronises the stream; params
 * [host] (NULL, or count entries) gives each plan's parameters as
 * nufft_plan_create's params (zero fields: the formulas), for instance the
 * autotuner's choice per size class.
 * nufft_multi_exec_fwd: c[i] [device] N[i] coefficients, g[i] [device] M[i]
 * outputs; captures a new graph when the pointers differ from the previous
 * call's, then launches it on the stream (asynchronous). */
typedef struct nufft_multi_s *nufft_multi;
int nufft_multi_create(nufft_multi *out, int count, const int64_t *N, const int64_t *M,
                       const double *const *y, double eps, int prec,
                       const nufft_params *params, unsigned flags, void *stream);
int nufft_multi_exec_fwd(nufft_multi multi, const void *const *c, void *const *g);
int nufft_multi_destroy(nufft_multi multi);

/* ---------------------------------------------------------------- one-shot */

/* Plan + exec + destroy in one call, with the paper's argument order
 * (nufft_fwd(c_n, N, y_j, M, eps) -> g_j).  All data pointers [device].
 * Synchronises the stream.
 * inufft (problem (ii) of Sec. 2): M == N uses the square Lagrange form of
 * Eq. p6 / p8 (as nufft_plan_exec_inv); M > N returns the least-squares
 * solution by plain CG (nufft_plan_solve_lsq with unit weights, tolerance
 * max(eps, 1e-14) on the unweighted normal-equation residual, at most 100000
 * iterations, NUFFT_ENOTCONV if it is not reached; complex128 only, else
 * NUFFT_ENOTSUP); M < N is underdetermined and returns NUFFT_EINVAL. */
int nufft_fwd(const void *c, int64_t N, const double *y, int64_t M, double eps,
              int prec, unsigned flags, void *g, void *stream);
int nufft_adj(const void *g, const double *y, int64_t M, int64_t N, double eps,
              int prec, unsigned flags, void *c, void *stream);
int inufft(const void *g, const double *y, int64_t M, int64_t N, double eps,
           int prec, unsigned flags, void *c, void *stream);

/* ---------------------------------------------------------------- no allocation */

/* nufft_fwd without any memory allocation.  The paper has no counterpart:
 * this serves callers that cannot allocate device memory when they need a
 * transform -- applications whose device memory belongs to a pool allocator
 * or a fixed budget, and latency-critical loops where cudaMalloc / cudaFree
 * (which may synchronise the device) are not acceptable.
 * Same arguments, result and accuracy as nufft_fwd (automatic parameters;
 * flags: 0 or NUFFT_IO_C64), but every work buffer lives in one fixed
 * 16 MiB device array compiled into the library, held by every GPU that loads
 * it until the process exits.  Limits: N a power of two, N <= 2^16 and
 * M <= 2^16; other sizes return NUFFT_EINVAL and do nothing.  The tree depth
 * is that of Eq. 25 but at least log2 N - 6 (leaves of at most 64 grid
 * points), so the result can differ from nufft_fwd's in the last digits when
 * M is much smaller than N.
 * The first call on a device looks up the array's device address and must run
 * with that device current; make it before any stream capture.  Calls share
 * the array and overwrite its contents; calls whose GPU work overlaps (other
 * streams, other threads) race on it.  Synchronises the stream. */
int nufft_fwd_noalloc(const void *c, int64_t N, const double *y, int64_t M,
                      double eps, int prec, unsigned flags, void *g, void *stream);

/* ---------------------------------------------------------------- diagnostics */

/* The near-field pair reciprocal 1/t (the singular part 2/t of Eq. p20, t in
 * grid units, |t| >= 1/2 for every pair the target kernels evaluate) as the
 * kernels compute it, on caller values: r64[i] = the FP64 path's reciprocal
 * of t[i] (hardware estimate + two Newton-Raphson steps), r32[i] = the mixed
 * path's reciprocal of (float)t[i] (rcp.approx.ftz.f32).  t [device]
 * double[n]; r64 [device] double[n], r32 [device] float[n], either may be
 * NULL.  Asynchronous. */
int nufft_diag_rcp(const double *t, int64_t n, double *r64, float *r32, void *stream);

/* Throughput of the two pipes that bound the near-field pair loop (one FP32
 * reciprocal and two FP32 FMAs per pair, Sec. 2.4's 3NM/2^lmax term): FP32
 * reciprocals (rcp.approx.ftz.f32) and FP32 FMAs completed per SM per SM
 * clock, measured by a kernel of independent chains on every SM (1024
 * threads per SM), timed with each SM's own clock counter; the median over
 * the SMs.  rcp_per_clk, ffma_per_clk [host] (either may be NULL).  Allocates
 * a few KB of device memory for the call; synchronises the stream. */
int nufft_diag_pipe_rates(double *rcp_per_clk, double *ffma_per_clk, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* NUFFT_GB300_H */
