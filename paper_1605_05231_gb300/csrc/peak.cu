// FP32 FMA throughput of the current device, measured: the denominator of the
// interpolation kernels' arithmetic roofline.  Not part of the projector.
//
// Every thread runs kChains independent multiply-add chains (enough to cover
// the FMA latency with 8 warps per scheduler) for `iters` rounds; the result
// is stored so that nothing is optimised away.
#include "internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 4;

__global__ void __launch_bounds__(kThreads) k_fma_chains(float* __restrict__ out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], b, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int nufft3d_fp32_fma_peak(double* tflops, int* sm_count, void* cuda_stream) {
  if (!tflops || !sm_count) return NUFFT3D_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) return NUFFT3D_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int blocks = sms * kBlocksPerSM, iters = 4096;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc((void**)&out, (size_t)blocks * kThreads * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  // one untimed launch, then the fastest of five
  for (int rep = 0; rep < 6 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_fma_chains<<<blocks, kThreads, 0, st>>>(out, iters, 0.9999f, 1e-4f);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess || best <= 0.f) return NUFFT3D_ERR_CUDA;
  const double flops = 2.0 * kChains * 16.0 * iters * (double)blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  *sm_count = sms;
  return NUFFT3D_OK;
}
