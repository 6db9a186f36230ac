// probe.cu -- measured FP64 arithmetic rate of this GPU, the roof of the FP64
// plain pass (which is bound by FP64 operations, not by HBM): every thread of
// a full grid runs eight independent FMA chains, timed with CUDA events.
#include <cuda_runtime.h>

#include "cl.h"

namespace {

constexpr int kChains = 8;

__global__ void fp64_fma_kernel(double* out, int iters, double y, double z) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], y, z);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 1234.5) out[blockIdx.x] = s;  // keeps the chains live
}

}  // namespace

extern "C" cl_status cl_measure_fp64_rate(void* stream, double* flops_per_s) {
  if (!flops_per_s) return CL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CL_ECUDA;
  const int threads = 256, blocks = nsm * 8, iters = 4096;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cl_status s = CL_OK;
  if (cudaMalloc(&out, blocks * sizeof(double)) != cudaSuccess) return CL_ENOMEM;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) s = CL_ECUDA;
  float best = 0.f;
  for (int rep = 0; rep < 4 && s == CL_OK; ++rep) {  // the first launch is a warm-up
    cudaEventRecord(e0, st);
    fp64_fma_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      s = CL_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (s == CL_OK && best > 0.f)
    *flops_per_s = 2.0 * (double)threads * blocks * kChains * iters / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return s;
}
