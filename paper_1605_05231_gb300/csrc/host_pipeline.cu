// Host-to-host forward + adjoint: the projector applied to volumes that live
// in host memory, with the host<->device copies on the library's own streams,
// overlapped with the kernels of the previous call.
//
// Per call, with b alternating between two sets of device buffers:
//   upload   stream: wait until set b is free; volume host -> device
//   compute  stream: wait for the upload; forward (volume -> lines);
//                    adjoint (lines -> volume out)
//   download stream: wait for the forward; lines device -> host; wait for the
//                    adjoint; volume out device -> host; set b is free again
// The plan's workspace is used by the compute stream only, so successive
// calls serialise their kernels there while copies of neighbouring calls run
// on the other two streams.
#include <new>

#include "internal.h"

struct nufft3d_host_pipeline_s {
  nufft3d_plan plan = nullptr;
  int device = 0;
  size_t vol_bytes = 0, lines_bytes = 0;
  cudaStream_t compute = nullptr, upload = nullptr, download = nullptr;
  void* vol[2] = {nullptr, nullptr};
  void* lines[2] = {nullptr, nullptr};
  void* vout[2] = {nullptr, nullptr};
  cudaEvent_t freed[2] = {nullptr, nullptr}, up[2] = {nullptr, nullptr}, fwd[2] = {nullptr, nullptr},
              adj[2] = {nullptr, nullptr};
  unsigned long long calls = 0;
};

namespace {

int rc_of(cudaError_t e) {
  if (e == cudaSuccess) return NUFFT3D_OK;
  return e == cudaErrorMemoryAllocation ? NUFFT3D_ERR_NOMEM : NUFFT3D_ERR_CUDA;
}

void release(nufft3d_host_pipeline hp) {
  for (int b = 0; b < 2; ++b) {
    for (void* q : {hp->vol[b], hp->lines[b], hp->vout[b]})
      if (q) cudaFree(q);
    for (cudaEvent_t e : {hp->freed[b], hp->up[b], hp->fwd[b], hp->adj[b]})
      if (e) cudaEventDestroy(e);
  }
  for (cudaStream_t s : {hp->compute, hp->upload, hp->download})
    if (s) cudaStreamDestroy(s);
  delete hp;
}

}  // namespace

extern "C" {

int nufft3d_host_pipeline_create(nufft3d_plan plan, nufft3d_host_pipeline* out) {
  if (!out) return NUFFT3D_ERR_ARG;
  *out = nullptr;
  if (!plan) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard guard(plan->device);
  if (guard.status != cudaSuccess) return NUFFT3D_ERR_CUDA;
  nufft3d_host_pipeline hp = new (std::nothrow) nufft3d_host_pipeline_s();
  if (!hp) return NUFFT3D_ERR_NOMEM;
  hp->plan = plan;
  hp->device = plan->device;
  hp->vol_bytes = (size_t)plan->N * plan->N * plan->N * (plan->complex_volume ? 8 : 4);
  hp->lines_bytes = (size_t)plan->P * 8;
  cudaError_t e = cudaSuccess;
  for (cudaStream_t* s : {&hp->compute, &hp->upload, &hp->download})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMalloc(&hp->vol[b], hp->vol_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&hp->lines[b], hp->lines_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&hp->vout[b], hp->vol_bytes);
    for (cudaEvent_t* ev : {&hp->freed[b], &hp->up[b], &hp->fwd[b], &hp->adj[b]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    release(hp);
    return rc_of(e);
  }
  *out = hp;
  return NUFFT3D_OK;
}

int nufft3d_host_forward_adjoint(nufft3d_host_pipeline hp, const void* vol_host, void* lines_host,
                                 void* vol_out_host) {
  if (!hp || !vol_host || !lines_host || !vol_out_host) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard guard(hp->device);
  if (guard.status != cudaSuccess) return NUFFT3D_ERR_CUDA;
  const int b = (int)(hp->calls & 1ull);
  cudaError_t e = cudaStreamWaitEvent(hp->upload, hp->freed[b], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hp->vol[b], vol_host, hp->vol_bytes, cudaMemcpyHostToDevice, hp->upload);
  if (e == cudaSuccess) e = cudaEventRecord(hp->up[b], hp->upload);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->compute, hp->up[b], 0);
  if (e != cudaSuccess) return rc_of(e);
  int rc = nufft::plan_forward_enqueue(hp->plan, hp->vol[b], hp->lines[b], hp->compute);
  if (rc != NUFFT3D_OK) return rc;
  e = cudaEventRecord(hp->fwd[b], hp->compute);
  if (e != cudaSuccess) return rc_of(e);
  rc = nufft::plan_adjoint_enqueue(hp->plan, hp->lines[b], hp->vout[b], hp->compute);
  if (rc != NUFFT3D_OK) return rc;
  e = cudaEventRecord(hp->adj[b], hp->compute);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->download, hp->fwd[b], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(lines_host, hp->lines[b], hp->lines_bytes, cudaMemcpyDeviceToHost, hp->download);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hp->download, hp->adj[b], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vol_out_host, hp->vout[b], hp->vol_bytes, cudaMemcpyDeviceToHost, hp->download);
  if (e == cudaSuccess) e = cudaEventRecord(hp->freed[b], hp->download);
  if (e != cudaSuccess) return rc_of(e);
  hp->calls++;
  return NUFFT3D_OK;
}

int nufft3d_host_pipeline_sync(nufft3d_host_pipeline hp) {
  if (!hp) return NUFFT3D_ERR_ARG;
  nufft::DeviceGuard guard(hp->device);
  if (guard.status != cudaSuccess) return NUFFT3D_ERR_CUDA;
  cudaError_t e = cudaStreamSynchronize(hp->upload);
  if (e == cudaSuccess) e = cudaStreamSynchronize(hp->compute);
  if (e == cudaSuccess) e = cudaStreamSynchronize(hp->download);
  return rc_of(e);
}

int nufft3d_host_pipeline_destroy(nufft3d_host_pipeline hp) {
  if (!hp) return NUFFT3D_OK;
  nufft::DeviceGuard guard(hp->device);
  cudaStreamSynchronize(hp->upload);
  cudaStreamSynchronize(hp->compute);
  cudaStreamSynchronize(hp->download);
  // the plan remembers the stream of its last call; that stream is about to go
  if (hp->plan->last_stream == hp->compute) hp->plan->last_stream = nullptr;
  release(hp);
  return NUFFT3D_OK;
}

}  // extern "C"
