// probe.cu -- measured FP64 arithmetic rate of this GPU, the roof of the FP64
// plain pass (which is bound by FP64 operations, not by HBM): every thread of
// a full grid runs eight independent FMA chains, timed with CUDA events.  Also
// the self-test of the bounded device waits that the persistent passes use.
#include <cuda_runtime.h>

#include "cl.h"
#include "common.cuh"

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

// One thread runs one of the passes' bounded waits: kind 0 waits for *counter
// to reach 1 (wait_counter), kind 1 for phase 0 of a fresh mbarrier that
// expects one arrival (mbar_wait_bounded), given (arrive = 1) or not.
__global__ void wait_selftest_kernel(const unsigned* counter, int kind, int arrive, unsigned long long limit_ns,
                                     int* status, unsigned long long* elapsed_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x | blockIdx.x) return;
  const unsigned long long t0 = clg::global_ns();
  bool ok;
  if (kind == 1) {
    clg::mbar_init(&bar, 1u);
    clg::fence_mbar_init();
    if (arrive) clg::mbar_arrive(&bar);
    ok = clg::mbar_wait_bounded(&bar, 0u, limit_ns);
  } else {
    ok = clg::wait_counter(counter, 1u, limit_ns);
  }
  *elapsed_ns = clg::global_ns() - t0;
  *status = ok ? (int)CL_OK : (int)CL_ETIMEOUT;
}

struct WaitProbe {
  unsigned counter;
  int status;
  unsigned long long elapsed_ns;
};

}  // namespace

extern "C" cl_status cl_selftest_wait(void* stream, int kind, int satisfied, uint64_t limit_ns,
                                      uint64_t* elapsed_ns) {
  if ((kind != 0 && kind != 1) || limit_ns == 0 || limit_ns > 10000000000ull) return CL_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  WaitProbe h{satisfied ? 1u : 0u, -1, 0ull};
  WaitProbe* d = nullptr;
  if (cudaMalloc(&d, sizeof(WaitProbe)) != cudaSuccess) return CL_ENOMEM;
  cl_status s = CL_OK;
  if (cudaMemcpyAsync(d, &h, sizeof(WaitProbe), cudaMemcpyHostToDevice, st) != cudaSuccess) s = CL_ECUDA;
  if (s == CL_OK) {
    wait_selftest_kernel<<<1, 32, 0, st>>>(&d->counter, kind, satisfied ? 1 : 0, (unsigned long long)limit_ns,
                                           &d->status, &d->elapsed_ns);
    if (cudaGetLastError() != cudaSuccess) s = CL_ECUDA;
  }
  if (s == CL_OK && (cudaMemcpyAsync(&h, d, sizeof(WaitProbe), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                     cudaStreamSynchronize(st) != cudaSuccess))
    s = CL_ECUDA;
  cudaFree(d);
  if (s != CL_OK) return s;
  if (elapsed_ns) *elapsed_ns = h.elapsed_ns;
  return h.status == (int)CL_OK ? CL_OK : h.status == (int)CL_ETIMEOUT ? CL_ETIMEOUT : CL_ECUDA;
}

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
