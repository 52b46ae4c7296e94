// Internal definitions shared by the CUDA translation units of the library.
//
// Coordinates.  Every point lives in "grid units" Y = y N / (2 pi), so the
// uniform grid x_k = 2 pi k / N sits at the integers.  A non-uniform point is
// stored as its nearest grid index k0 (int) plus an offset delta in
// [-1/2, 1/2] (binary64, relative precision of delta itself), formed from
// y with a double-double product.  Distances between a point and grid
// points, t = (k0 - k) + delta, then keep full relative precision down to
// the exact hit, which the kernel G(t) of Eq. p5 needs near its pole.
//
// Tree.  Level l has 2^l arcs (boxes) of W_l = N / 2^l grid units
// (Sec. 2.1); leaves are level L = lmax with s = N / 2^L grid points each.
// Box i at level l has centre (i + 1/2) W_l.  Expansions are scaled by the
// box width so the translation operators do not depend on the level.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/nufft.h"

namespace nufft {

constexpr double kTwoPiHi = 6.283185307179586;          // fl(2 pi)
constexpr double kTwoPiLo = 2.4492935982947064e-16;     // 2 pi - fl(2 pi)
constexpr double kInvTwoPiHi = 0.15915494309189535;     // fl(1/(2 pi))
constexpr double kInvTwoPiLo = -9.839338337591243e-18;  // 1/(2 pi) - fl(1/(2 pi))
constexpr double kInvPi = 0.3183098861837907;           // fl(1/pi)
constexpr double kPi = 3.141592653589793;

// box offset of level l (>= 2) in the per-level concatenated arrays
__host__ __device__ inline int64_t level_off(int l) { return (int64_t(1) << l) - 4; }

template <class T> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <class T> using cplx = typename cplx_t<T>::type;

template <class T> __host__ __device__ inline cplx<T> mk(T a, T b) { cplx<T> r; r.x = a; r.y = b; return r; }
template <class V> __host__ __device__ inline V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <class V> __host__ __device__ inline V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <class V> __host__ __device__ inline V cmul(V a, V b) {
  V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <class V, class S> __host__ __device__ inline V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }
template <class V> __host__ __device__ inline V cconj(V a) { a.y = -a.y; return a; }

__device__ inline double2 to_d2(float2 a) { return make_double2(a.x, a.y); }
__device__ inline double2 to_d2(double2 a) { return a; }
template <class T> __device__ inline cplx<T> from_d2(double2 a);
template <> __device__ inline double2 from_d2<double>(double2 a) { return a; }
template <> __device__ inline float2 from_d2<float>(double2 a) { return make_float2((float)a.x, (float)a.y); }

// complex128 <-> the arithmetic type (hardware conversions: measured faster
// here than integer-operation versions of the IEEE-754 conversion)
template <class T> __device__ inline cplx<T> c128_to(double2 a);
template <> __device__ inline double2 c128_to<double>(double2 a) { return a; }
template <> __device__ inline float2 c128_to<float>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}
__device__ inline double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
__device__ inline double2 to_c128(double2 a) { return a; }

// delta < 0 for a binary64 delta (-0.0 counts as zero), tested on its bits
__device__ inline bool neg_bits(double d) {
  const long long b = __double_as_longlong(d);
  return b < 0 && b != (long long)0x8000000000000000ull;
}

// 1/t of a near-field pair (the singular part 2/t of Eq. p20; |t| >= 1/2 in
// grid units for every pair that is not a point's nearest grid point, so t
// is never subnormal).  FP32: the special-function unit's reciprocal
// (rcp.approx, at most 1 ulp).
// FP64: the unit's FP64 reciprocal estimate (rcp.approx.ftz.f64, about 20
// correct bits) refined by two Newton-Raphson steps r <- r + r (1 - t r),
// each of which squares the relative error, so r is within a few ulp of
// 1/t (t is never subnormal here).  (An FP32 estimate refined in FP64 was
// measured slower than a division: its two precision conversions run at the
// FP64 rate.)  t = 0 gives a NaN; callers that meet t = 0 replace r by 0.
__device__ inline float rcp_t(float t) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(t));
  return r;
}
__device__ inline double rcp_t(double t) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(t));
  double e = fma(-t, r, 1.0);
  r = fma(r, e, r);
  e = fma(-t, r, 1.0);
  return fma(r, e, r);
}

// Leaf index and offset of a point from its grid coordinates (int32: N <= 2^26):
// leaf = floor((k0 + delta)/s) mod 2^L, o = k0 - leaf s in [0, s].
__device__ inline void point_local(int k0, double delta, int N, int s, int* leaf, int* o) {
  int fl = neg_bits(delta) ? k0 - 1 : k0;
  fl &= (N - 1);
  int b = fl >> (__ffs(s) - 1);  // s is a power of two
  *leaf = b;
  *o = (k0 - b * s) & (N - 1);
}

// Sizes and pointers of one FMM evaluation, passed by value to kernels.
struct TreeDims {
  int64_t N;   // grid size (power of two)
  int L;       // leaf level
  int s;       // grid points per leaf = N >> L
  int p;       // 1/t expansion length
  int q;       // regular-series truncation number
  int pm;      // multipole length kept (max(p, 2q + 1))
  int64_t mstride = 0;  // per-signal strides (batched plans; blockIdx.y = signal)
  int64_t lstride = 0;  //   multipoles, locals (complex elements)
  int64_t M_ = 0;       //   and points (charges per signal)
  // per-plan constants formed on the host (kernels need no FP64 division):
  // 2/N, 1/s, N/pi in both precisions
  double two_n = 0, inv_s = 0, n_pi = 0;
  float two_n_f = 0, inv_s_f = 0, n_pi_f = 0;
  // square inverse with Nc = nc coefficients on this grid (nc < N): C at the
  // grid point k carries the phase e^{i pi k nc / N} (0: the phase is the
  // sign (-1)^k, already in C)
  int64_t nc = 0;
};

// e^{i pi (k nc mod 2N) / N}, the phase of C(x_k) of the square inverse on a
// grid of N > nc points (the argument reduced exactly in integers)
__device__ inline double2 inv_phase(const TreeDims& d, int64_t k) {
  const int64_t a = (k * d.nc) % (2 * d.N);
  double s, c;
  sincospi((double)a / (double)d.N, &s, &c);
  return make_double2(c, s);
}

template <class T> struct KConst;
template <> struct KConst<double> {
  __device__ static double two_n(const TreeDims& d) { return d.two_n; }
  __device__ static double inv_s(const TreeDims& d) { return d.inv_s; }
  __device__ static double n_pi(const TreeDims& d) { return d.n_pi; }
};
template <> struct KConst<float> {
  __device__ static float two_n(const TreeDims& d) { return d.two_n_f; }
  __device__ static float inv_s(const TreeDims& d) { return d.inv_s_f; }
  __device__ static float n_pi(const TreeDims& d) { return d.n_pi_f; }
};

// Device-side error word (set by kernels, read back by the host).
enum DevStatus : int {
  kDevOk = 0,
  kDevBadPoint = 1,     // y not finite or outside [0, 2 pi)
  kDevSegTooLarge = 2,  // a leaf held more points than the segment sort supports
  kDevIllCond = 4,      // duplicate points / exponent range in the inverse
  kDevTimeout = 8,      // a bounded wait (tensor-core barrier) gave up
};

// Programmatic dependent launch.  Kernels of a transform are launched with
// programmatic stream serialization (launch_pdl), so a kernel's CTAs may
// start while its predecessor in the stream is still finishing.  Every such
// kernel calls pdl_wait() before it reads or writes any global data that an
// earlier kernel of the stream touches (only constant plan tables may be read
// before it); griddepcontrol.wait returns once the predecessor grid has
// completed and its writes are visible, and is a no-op for a kernel launched
// without the attribute.  pdl_trigger() lets the successor's launch begin
// once every CTA of this grid has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool pdl_enabled();  // false when the environment sets NUFFT_NO_PDL
// false when the environment sets NUFFT_NO_FUSED_UP: the upward pass then
// runs as one launch per subtree level band (same arithmetic, same results)
bool fused_up_enabled();

// Launch priority: kernels on the critical path of an exec sequence run at
// the device's highest priority, so the CTAs of a side-branch kernel that
// fills the GPU (the near field beside the tree passes) do not hold them
// back; a LowPriority scope (the side branch) launches at the default.
// 0 = no attribute (NUFFT_NO_PRIORITY, or no priority range on the device).
int launch_priority();
struct LowPriority {
  LowPriority();
  ~LowPriority();
};

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (pdl_enabled()) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  const int prio = launch_priority();
  if (prio != 0) {
    at[na].id = cudaLaunchAttributePriority;
    at[na].val.priority = prio;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace nufft

// One kernel's FMM operator set (device pointers): the cot kernel's 1/t
// operators or the log kernel's (inverse coefficients).
struct FmmOps {
  const void* m2l = nullptr;   // [4][p][p]
  const void* l2l = nullptr;   // [2][p][p]
  const double* reg = nullptr; // [4][nq][nq] level-2 weights and shifts
  int nq = 0;                  // number of level-2 polynomial coefficients
  double c1 = 0, c2 = 0;       // constants per unit charge in Omega_1 / Omega_2
  int log_kernel = 0;          // adds M_0 log W_l in M2L
  const double* leaf_shift = nullptr;  // moments subtracted from every leaf
};

// Per-stage event timing of a plan (see nufft_plan_profile).
struct StageProf {
  static constexpr int kMaxPairs = 4096;
  int enabled = 0;
  int npairs = 0;
  cudaEvent_t ev[2 * kMaxPairs] = {};
  int stage[kMaxPairs] = {};
  double ms[NUFFT_NSTAGES] = {};
  int64_t launches[NUFFT_NSTAGES] = {};
  int open_stage = -1;
};

// The plan object behind the opaque handle of nufft.h.
struct nufft_plan_s {
  // N: the FMM grid (a power of two); Nc: the caller's number of coefficients
  // (N itself, or any Nc <= N with N = 2^ceil(log2 Nc): the band-limited
  // series with Nc terms is also one with N terms, its top N - Nc zero)
  int64_t N = 0, M = 0, Nc = 0;
  int L = 0, B = 0, s = 0, p = 0, q = 0, pm = 0;
  int prec = 0;
  int batch = 1;        // signals sharing the point set
  unsigned flags = 0;
  double eps = 0;
  cudaStream_t stream = nullptr;
  // non-uniform point set, sorted by leaf (stable by original index)
  int32_t *perm = nullptr;        // [M] original index of sorted point
  int32_t *leaf_start = nullptr;  // [B+1]
  int32_t *k0 = nullptr;          // [M] nearest grid index (sorted order)
  double *delta = nullptr;        // [M] offset in grid units (sorted order)
  double2 *F = nullptr;           // [M] F_j = (e^{i N y_j} - 1)/N, Eq. p5
  double2 *E = nullptr;           // [M] e^{i pi delta} sin(pi delta)/(pi delta)
  // FP32 copies for the mixed path (rounded from the FP64 values)
  float *delta_f = nullptr;       // [M]
  float2 *Ff = nullptr, *Ef = nullptr;  // [M]
  float2 *lvl2f = nullptr;        // level-2 coefficients
  // inverse coefficients (Eq. p8), scaled by a common factor
  double2 *Dt = nullptr;          // [M] D_j e^{-Lambda}
  float2 *Dtf = nullptr;          // [M] FP32 copy (mixed path)
  double *Ct = nullptr;           // [N] real C_k e^{+Lambda} / N
  float *Ctf = nullptr;           // [N] FP32 copy (mixed path)
  double2 *Sinv = nullptr;        // [M] sorted: the inverse's self term st_j = q_j S_j
  float2 *Sinvf = nullptr;        // [M] FP32 copy (mixed path)
  double *Lambda = nullptr;       // [1] common scale of C and D
  int64_t inv_nc = 0;             // Nc when C carries the phase e^{i pi k Nc / N} (Nc < N)
  // FMM workspace
  void *mexp = nullptr;    // [levels 2..L][box][pm] complex (T)
  void *lexp = nullptr;    // [levels 3..L][box][p] complex (T)
  void *charge = nullptr;  // [max(N, M)] complex (T): charges in sorted order
  void *selft = nullptr;   // [M] complex (T): nearest-pair terms of the adjoint / inverse
  void *srcpos = nullptr;  // [M] packed (k0, delta) source positions: 8 B (FP32) / 16 B (FP64)
  double2 *grid = nullptr; // [N] work vector on the grid (complex128 storage; used
                           //     as complex64 by the mixed path)
  double2 *grid2 = nullptr;// [N] FFT scratch
  double2 *grid3 = nullptr;// [N] second FFT scratch (three or more passes)
  double2 *lvl2 = nullptr; // [4*2q + 1] level-2 polynomial coefficients D_l, then Q
  // operators (device copies, in T)
  void *op_m2m = nullptr;  // [2][pm][pm]  transposed: [sigma][k][m]
  void *op_m2l = nullptr;  // [4][p][p]    transposed: [d][m][n], d = -3,-2,2,3
  void *op_l2l = nullptr;  // [2][p][p]    transposed: [sigma][n'][n]
  void *op_p2m = nullptr;  // [s][pm] powers rho_o^m of the uniform grid in a leaf
  double *op_reg = nullptr;// [2][2q][2q] level-2 weights W1, W2 (FP64)
  float *op_tc = nullptr;  // tensor-core M2L + L2L operator (hi, lo), kernel layout
  int tc_level = -1;       // first level on the tensor cores (-1: none)
  int tc_near = -1;        // 1: batched forward near field on the tensor cores
  double2 *fft_tw = nullptr; // FFT twiddle tables
  float2 *fft_tw_f = nullptr;
  int fft_tw_lo_bits = 0;
  int *status = nullptr;   // device error word
  int *seg_overflow = nullptr;
  int *upcnt = nullptr;    // [batch][upcnt_n] group counters of the one-launch upward pass
  int upcnt_n = 0;         //     (zero between launches); null: upward pass in several launches
  StageProf *prof = nullptr;
  void *lsq_work = nullptr;  // CG work vectors (created on first least-squares solve)
  // exec sequences captured as CUDA graphs, keyed by operation and buffers
  struct GraphEntry {
    int op = -1;
    const void* in = nullptr;
    void* out = nullptr;
    cudaGraphExec_t exec = nullptr;
  };
  static constexpr int kGraphSlots = 8;
  GraphEntry graphs[kGraphSlots];
  int graph_next = 0;            // slot replaced next (round robin)
  cudaStream_t cap = nullptr;    // private capture origin
  // side branch: work the main chain does not wait for at once (level-2
  // coefficients, self terms) runs on `aux`, forked and joined by events
  cudaStream_t aux = nullptr;
  cudaStream_t aux2 = nullptr;   // slot 2: the near field, beside the tree passes
  cudaEvent_t ev_fork[3] = {}, ev_join[3] = {};
  int side_ok = 1;               // 0: keep everything on `stream`
  int max_leaf = 0;              // most points in one leaf (host copy, set at plan creation)
  // chunked P2M of clustered sources (a leaf with >= 4x the mean count):
  // chunk i = (leaf, first, end) of at most 256 sources; leaf b's chunks are
  // p2m_cfirst[b] .. p2m_cfirst[b + 1] - 1; their moments in p2m_part
  int32_t *p2m_chunk = nullptr;  // [p2m_nchunk][3]
  int32_t *p2m_cfirst = nullptr; // [B + 1]
  int64_t p2m_nchunk = 0;
  void *p2m_part = nullptr;      // [batch][p2m_nchunk][pm] complex (T)
  void *hnear = nullptr;         // near-field sums of one signal (2 max(N, M) complex):
                                 //     forward [M], adjoint / inverse [N][2] (sum, self terms)
  // adaptive tree (NUFFT_ADAPTIVE, forward): leaf b refined by d_b levels;
  // class d = the targets of leaves with d_b = d, stored class after class
  static constexpr int kAdMax = 3;
  int ad_D = 0;                    // max d_b (0: uniform tree)
  int64_t ad_off[kAdMax + 2] = {}; // class d: [ad_off[d], ad_off[d + 1]) of the ad_ arrays
  int64_t ad_boff[kAdMax + 1] = {};// boxes of level L + d (d >= 1): ad_box[ad_boff[d-1], ad_boff[d])
  int64_t ad_toff[kAdMax + 1] = {};// P2M table of level L + d: ad_p2m + ad_toff[d - 1] (s_d x p)
  int32_t *ad_box = nullptr;       // box indices at their level
  int32_t *ad_rleaf = nullptr;     // [ad_nrleaf][2] the refined leaves and their depths d_b
  int64_t ad_nrleaf = 0;
  int32_t *ad_perm = nullptr;      // [M] original index, class-major order
  void *ad_pos = nullptr;          // [M] packed positions (as srcpos)
  double2 *ad_F = nullptr, *ad_E = nullptr;   // [M]
  float2 *ad_Ff = nullptr, *ad_Ef = nullptr;  // [M] (mixed)
  void *ad_p2m = nullptr;          // rho_o^m of the grid points of a box, per deep level (T)
  void *ad_lexp = nullptr;         // locals in the lexp layout of levels 3..L + ad_D
                                   //     (levels L + 1 .. L + ad_D written)
  // adjoint / inverse on the same classes (sources): class d as the uniform
  // tree of depth L + d (its points sorted by leaf of that level)
  int32_t *ad_start = nullptr;     // class d: leaf starts of level L + d (within the class) at ad_soff[d]
  int64_t ad_soff[kAdMax + 1] = {};
  int32_t *ad_tiles = nullptr;     // class d >= 1: the grid tiles (2 kTgtThreads points) its sources reach
  int64_t ad_tioff[kAdMax + 1] = {};
  int32_t *ad_srange = nullptr;    // [ad_boff[D]][2] source range of each deep box (class-major indices)
  int32_t *ad_gbox = nullptr;      // grid boxes of level L + d with a deep box in their interaction list
  int32_t *ad_gil = nullptr;       //     [][3]: that list's slots as deep-box indices of the level (-1: none)
  int64_t ad_goff[kAdMax + 1] = {};
  void *ad_mexp = nullptr;         // [ad_boff[D]][p] multipoles of the deep boxes (T)
  void *ad_charge = nullptr, *ad_st = nullptr; // [M] charges / self terms of the deeper classes (T, class order)
  double2 *ad_Dt = nullptr, *ad_S = nullptr;   // [M] inverse coefficients / self-term factors (class order)
  float2 *ad_Dtf = nullptr, *ad_Sf = nullptr;  // [M] (mixed)
};

// Begin a side branch (slot 0, 1 or 2; slot 2 has a stream of its own): returns the stream to launch it on --
// `aux` after it waits for the work issued so far on the plan's stream, or
// the plan's stream itself while profiling (per-stage events need one
// stream order) or when the side stream cannot be made.  side_end marks the
// branch's end; side_join makes the plan's stream wait for it.
cudaStream_t side_begin(nufft_plan_s* pl, int slot);
void side_end(nufft_plan_s* pl, int slot, cudaStream_t s);
void side_join(nufft_plan_s* pl, int slot);

// Bracket the launches of one stage (no-ops unless profiling is enabled).
void prof_begin(nufft_plan_s* pl, int stage);
void prof_end(nufft_plan_s* pl, int launches);
