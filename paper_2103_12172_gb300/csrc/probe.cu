// FP64 FMA throughput probe (the roofline denominator of the FP64-bound kernels).
#include "mdp_probe.h"
#include <cuda_runtime.h>

namespace {
__global__ void __launch_bounds__(256) k_dfma_chains(double *out, int iters, double b, double c) {
  double a[8];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = g * 1e-9 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[g] = s;
}
}  // namespace

extern "C" mdp_status mdp_probe_dfma_gflops(int iters, double *gflops, void *cuda_stream) {
  if (!gflops || iters < 0) return MDP_ERR_ARG;
  if (iters == 0) iters = 4096;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDP_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return MDP_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mdp_status rc = MDP_OK;
  float ms = 0.f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MDP_ERR_CUDA;
  if (rc == MDP_OK) {
    k_dfma_chains<<<blocks, threads, 0, st>>>(buf, 64, 1.0000001, 1e-7);  // warm-up
    cudaEventRecord(e0, st);
    k_dfma_chains<<<blocks, threads, 0, st>>>(buf, iters, 1.0000001, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = MDP_ERR_CUDA;
  }
  if (rc == MDP_OK) *gflops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e6);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}
