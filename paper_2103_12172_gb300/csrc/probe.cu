// FP64 throughput probes: FMA on the FP64 pipe (the roofline denominator of the FP64-bound
// kernels) and the FP64 tensor-core path (mma.sync m8n8k4, DMMA), the alternative for a dense
// FP64 contraction.
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
// 8 independent m8n8k4 FP64 MMA chains per warp: D = A B + C with A 8x4 (one value per lane),
// B 4x8 (one per lane) and C, D 8x8 (two per lane); 512 flops per instruction.
__global__ void __launch_bounds__(256) k_dmma_chains(double *out, int iters, double b) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const double a = 1e-9 * (threadIdx.x + 1);
  double c[8][2];
#pragma unroll
  for (int i = 0; i < 8; ++i) { c[i][0] = g * 1e-9 + i; c[i][1] = i; }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[i][0]), "+d"(c[i][1]) : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += c[i][0] + c[i][1];
  out[g] = s;
}

// Times `kern` (one warm-up launch of 64 iterations, then one of `iters`) over sms x 8 blocks of
// 256 threads; returns the elapsed milliseconds in *ms.
template <class F>
mdp_status time_probe(F launch, int iters, void *cuda_stream, float *ms) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDP_ERR_CUDA;
  const int blocks = sms * 8, threads = 256;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double *buf = nullptr;
  if (cudaMalloc(&buf, (size_t)blocks * threads * sizeof(double)) != cudaSuccess) return MDP_ERR_CUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mdp_status rc = MDP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MDP_ERR_CUDA;
  if (rc == MDP_OK) {
    launch(blocks, threads, st, buf, 64);   // warm-up
    cudaEventRecord(e0, st);
    launch(blocks, threads, st, buf, iters);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      rc = MDP_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return rc;
}
}  // namespace

extern "C" mdp_status mdp_probe_dmma_gflops(int iters, double *gflops, void *cuda_stream) {
  if (!gflops || iters < 0) return MDP_ERR_ARG;
  if (iters == 0) iters = 2048;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDP_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MDP_ERR_CUDA;
  float ms = 0.f;
  const mdp_status rc = time_probe(
      [](int blocks, int threads, cudaStream_t st, double *buf, int it) {
        k_dmma_chains<<<blocks, threads, 0, st>>>(buf, it, 1.0000001);
      },
      iters, cuda_stream, &ms);
  if (rc == MDP_OK) *gflops = 512.0 * 8.0 * iters * ((double)sms * 8 * 256 / 32) / (ms * 1e6);
  return rc;
}

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
