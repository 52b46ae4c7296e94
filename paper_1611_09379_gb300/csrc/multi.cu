// Many independent forward transforms of uneven sizes (own N_i, M_i and point
// set y_i each) executed as one CUDA graph launch.  Each transform keeps its
// own plan (the data structure of Sec. 3.3); an execution captures every
// plan's kernel chain on one of 64 forked streams, so independent
// transforms overlap on the GPU, and replays the instantiated graph with a
// single cudaGraphLaunch while the caller's buffers stay the same.  The
// per-transform kernels are the ones of nufft_plan_exec_fwd.
#include <new>
#include <vector>

#include "common.cuh"

namespace {
// streams the transforms are spread over (measured for 256 transforms of
// 2^10..2^16: 16 streams 1.10 ms, 32 0.98, 64 0.96); each plan then runs on
// its stream alone, without its own side branches (0.93 ms)
constexpr int kMultiStreams = 64;
}

struct nufft_multi_s {
  std::vector<nufft_plan> plans;
  cudaStream_t user = nullptr;
  cudaStream_t cap = nullptr;  // private capture origin (the legacy stream cannot be captured)
  cudaStream_t side[kMultiStreams] = {};
  cudaEvent_t fork = nullptr, join[kMultiStreams] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> last_c;
  std::vector<void*> last_g;
};

static void multi_free(nufft_multi_s* m) {
  if (m->exec) cudaGraphExecDestroy(m->exec);
  if (m->graph) cudaGraphDestroy(m->graph);
  for (nufft_plan p : m->plans)
    if (p) nufft_plan_destroy(p);
  for (int i = 0; i < kMultiStreams; ++i) {
    if (m->side[i]) cudaStreamDestroy(m->side[i]);
    if (m->join[i]) cudaEventDestroy(m->join[i]);
  }
  if (m->fork) cudaEventDestroy(m->fork);
  if (m->cap) cudaStreamDestroy(m->cap);
  delete m;
}

extern "C" {

int nufft_multi_create(nufft_multi* out, int count, const int64_t* N, const int64_t* M,
                       const double* const* y, double eps, int prec,
                       const nufft_params* params, unsigned flags, void* stream) {
  if (!out || count < 1 || !N || !M || !y) return NUFFT_EINVAL;
  if (flags & NUFFT_WANT_INVERSE) return NUFFT_ENOTSUP;
  *out = nullptr;
  nufft_multi_s* m = new (std::nothrow) nufft_multi_s();
  if (!m) return NUFFT_ENOMEM;
  m->user = (cudaStream_t)stream;
  m->plans.assign(count, nullptr);
  for (int i = 0; i < count; ++i) {
    int rc = nufft_plan_create(&m->plans[i], N[i], M[i], y[i], eps, prec,
                               params ? &params[i] : nullptr, flags, stream);
    if (rc) { multi_free(m); return rc; }
    m->plans[i]->side_ok = 0;
  }
  if (cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&m->cap, cudaStreamNonBlocking) != cudaSuccess) {
    multi_free(m);
    return NUFFT_ECUDA;
  }
  for (int i = 0; i < kMultiStreams; ++i)
    if (cudaStreamCreateWithFlags(&m->side[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->join[i], cudaEventDisableTiming) != cudaSuccess) {
      multi_free(m);
      return NUFFT_ECUDA;
    }
  *out = m;
  return NUFFT_OK;
}

int nufft_multi_destroy(nufft_multi m) {
  if (!m) return NUFFT_EINVAL;
  cudaStreamSynchronize(m->user);
  multi_free(m);
  return NUFFT_OK;
}

int nufft_multi_exec_fwd(nufft_multi m, const void* const* c, void* const* g) {
  if (!m || !c || !g) return NUFFT_EINVAL;
  const int n = (int)m->plans.size();
  bool same = m->exec && (int)m->last_c.size() == n;
  for (int i = 0; same && i < n; ++i) same = (m->last_c[i] == c[i] && m->last_g[i] == g[i]);
  if (!same) {
    // (re)capture on the private stream: fork into the side streams, one
    // transform per side stream in turn, join back; the graph is launched on
    // the caller's stream, after its earlier work
    if (m->exec) { cudaGraphExecDestroy(m->exec); m->exec = nullptr; }
    if (m->graph) { cudaGraphDestroy(m->graph); m->graph = nullptr; }
    if (cudaStreamBeginCapture(m->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return NUFFT_ECUDA;
    int rc = NUFFT_OK;
    if (cudaEventRecord(m->fork, m->cap) != cudaSuccess) rc = NUFFT_ECUDA;
    for (int s = 0; !rc && s < kMultiStreams; ++s)
      if (cudaStreamWaitEvent(m->side[s], m->fork, 0) != cudaSuccess) rc = NUFFT_ECUDA;
    for (int i = 0; !rc && i < n; ++i) {
      nufft_plan_set_stream(m->plans[i], m->side[i % kMultiStreams]);
      rc = nufft_plan_exec_fwd(m->plans[i], c[i], g[i]);
    }
    for (int s = 0; !rc && s < kMultiStreams; ++s)
      if (cudaEventRecord(m->join[s], m->side[s]) != cudaSuccess ||
          cudaStreamWaitEvent(m->cap, m->join[s], 0) != cudaSuccess)
        rc = NUFFT_ECUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t ec = cudaStreamEndCapture(m->cap, &graph);
    for (int i = 0; i < n; ++i) nufft_plan_set_stream(m->plans[i], m->user);
    if (rc || ec != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return rc ? rc : NUFFT_ECUDA;
    }
    m->graph = graph;
    if (cudaGraphInstantiate(&m->exec, m->graph, 0) != cudaSuccess) {
      m->exec = nullptr;
      return NUFFT_ECUDA;
    }
    m->last_c.assign(c, c + n);
    m->last_g.assign(g, g + n);
  }
  return cudaGraphLaunch(m->exec, m->user) == cudaSuccess ? NUFFT_OK : NUFFT_ECUDA;
}

}  // extern "C"
