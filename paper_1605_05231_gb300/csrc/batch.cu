// Batches of independent projector problems of mixed sizes.  A batch owns one
// plan per item.  Its forward + adjoint over all items is captured once into a
// CUDA graph: items are dealt, largest first, to the least loaded of up to 12
// worker streams forked from the caller's stream, so small problems run
// concurrently, and every later call
// replays the whole sequence with one cudaGraphLaunch.  The graph is captured
// again only when the caller passes different buffers.
#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"

struct nufft3d_batch_s {
  std::vector<nufft3d_plan> plans;
  int device = 0;
  cudaStream_t cap = nullptr;  // capture origin (the legacy stream cannot be captured)
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> join;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> key;  // buffers the graph was captured with
};

namespace {

constexpr int kMaxWorkerStreams = 12;

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

void free_batch(nufft3d_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  for (nufft3d_plan p : b->plans) nufft3d_plan_destroy(p);
  delete b;
}

int capture(nufft3d_batch b, const void* const* vols, void* const* lines, void* const* vols_out,
            cudaStream_t launch_st) {
  const int n = (int)b->plans.size();
  cudaStream_t st = b->cap;
  const int ns = (int)b->streams.size();
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_rc(e);
  int rc = NUFFT3D_OK;
  e = cudaEventRecord(b->fork, st);
  for (int s = 0; s < ns && e == cudaSuccess; ++s) e = cudaStreamWaitEvent(b->streams[s], b->fork, 0);
  // items dealt largest first to the least loaded worker stream (work taken as
  // the evaluated points plus the grid cells), so the streams finish together
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto work = [&](int i) {
    const nufft3d_plan p = b->plans[i];
    return (double)p->P_eval + (double)p->K * p->K * p->K;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return work(a) > work(c); });
  std::vector<double> load(ns, 0.0);
  for (int q = 0; q < n && e == cudaSuccess && rc == NUFFT3D_OK; ++q) {
    const int i = order[q];
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += work(i);
    cudaStream_t ws = b->streams[w];
    rc = nufft::plan_forward_enqueue(b->plans[i], vols[i], lines[i], ws);
    if (rc == NUFFT3D_OK) rc = nufft::plan_adjoint_enqueue(b->plans[i], lines[i], vols_out[i], ws);
  }
  for (int s = 0; s < ns && e == cudaSuccess; ++s) {
    e = cudaEventRecord(b->join[s], b->streams[s]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->join[s], 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = e2;
  if (rc != NUFFT3D_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return rc != NUFFT3D_OK ? rc : cuda_rc(e);
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph = g;
  e = cudaGraphInstantiate(&b->exec, g, 0);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return cuda_rc(e);
  }
  for (nufft3d_plan p : b->plans) p->last_stream = launch_st;
  return NUFFT3D_OK;
}

}  // namespace

extern "C" {

int nufft3d_batch_create(nufft3d_batch* out, const nufft3d_params* ps, int count, void* cuda_stream) {
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  if (!ps || count < 1) return NUFFT3D_ERR_ARG;
  nufft3d_batch b = new (std::nothrow) nufft3d_batch_s();
  if (!b) return NUFFT3D_ERR_NOMEM;
  int rc = NUFFT3D_OK;
  cudaError_t e = cudaGetDevice(&b->device);
  if (e != cudaSuccess) rc = cuda_rc(e);
  for (int i = 0; i < count && rc == NUFFT3D_OK; ++i) {
    nufft3d_plan p = nullptr;
    rc = nufft3d_plan_create(&p, ps + i, cuda_stream);
    if (rc == NUFFT3D_OK) b->plans.push_back(p);
  }
  const int ns = count < kMaxWorkerStreams ? count : kMaxWorkerStreams;
  for (int s = 0; s < ns && rc == NUFFT3D_OK; ++s) {
    cudaStream_t st;
    cudaEvent_t ev;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->join.push_back(ev);
    if (e != cudaSuccess) rc = cuda_rc(e);
  }
  if (rc == NUFFT3D_OK) {
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_rc(e);
  }
  if (rc != NUFFT3D_OK) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return NUFFT3D_OK;
}

int nufft3d_batch_size(nufft3d_batch b, int* count) {
  if (!b || !count) return NUFFT3D_ERR_ARG;
  *count = (int)b->plans.size();
  return NUFFT3D_OK;
}

int nufft3d_batch_item(nufft3d_batch b, int i, nufft3d_plan* out) {
  if (!b || !out || i < 0 || i >= (int)b->plans.size()) return NUFFT3D_ERR_ARG;
  *out = b->plans[i];
  return NUFFT3D_OK;
}

int nufft3d_batch_forward_adjoint(nufft3d_batch b, const void* const* vols, void* const* lines,
                                  void* const* vols_out, void* cuda_stream) {
  if (!b || !vols || !lines || !vols_out) return NUFFT3D_ERR_ARG;
  const int n = (int)b->plans.size();
  std::vector<const void*> key;
  key.reserve(3 * n);
  for (int i = 0; i < n; ++i) {
    if (!vols[i] || !lines[i] || !vols_out[i]) return NUFFT3D_ERR_ARG;
    key.push_back(vols[i]);
    key.push_back(lines[i]);
    key.push_back(vols_out[i]);
  }
  nufft::DeviceGuard guard(b->device);
  if (guard.status != cudaSuccess) return cuda_rc(guard.status);
  cudaError_t e = cudaSuccess;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!b->exec || key != b->key) {
    // plans' earlier work on other streams must not race the replay
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_rc(e);
    const int rc = capture(b, vols, lines, vols_out, st);
    if (rc != NUFFT3D_OK) return rc;
    b->key = key;
  }
  return cuda_rc(cudaGraphLaunch(b->exec, st));
}

int nufft3d_batch_invalidate(nufft3d_batch b) {
  if (!b) return NUFFT3D_ERR_ARG;
  b->key.clear();
  return NUFFT3D_OK;
}

int nufft3d_batch_destroy(nufft3d_batch b) {
  if (!b) return NUFFT3D_OK;
  nufft::DeviceGuard guard(b->device);
  cudaDeviceSynchronize();
  free_batch(b);
  return NUFFT3D_OK;
}

}  // extern "C"
