// noalloc.cu -- volume averages of a scalar-field state held in caller memory,
// computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: applications that hand the library all
// of their device memory up front (a fixed memory budget, or another
// framework's pool), and loops that must not synchronise the device, which
// cudaMalloc and cudaFree may do.  For them, cl_volume_averages_noalloc keeps
// its per-block partial sums in the file-scope array below instead of in
// context-owned scratch.  The array is 1024 rows x 16 doubles (128 KiB) and
// every GPU that loads this library holds it until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "cl.h"

namespace {

constexpr int kMaxBlocks = CL_NOALLOC_MAX_BLOCKS;
constexpr int kSlots = CL_NOALLOC_OUT;
constexpr int kThreads = 256;

// Shared by every call on a device; rows [0, nblk) are written by the first
// kernel of a call before the second kernel of the same call reads them.
static __device__ __align__(256) double g_avg_scratch[kMaxBlocks * kSlots];

// Device address of g_avg_scratch for each device, looked up with that device
// current (the host-side name is only a stand-in).  It is looked up again on
// every call whose stream is not being captured, so that an address made
// stale by a device reset (which reloads the module) is never used; a call
// during a stream capture takes the address the last uncaptured call found.
std::mutex g_mu;
double* g_scratch_ptr[64] = {nullptr};

template <typename T>
__global__ void avg_partial_kernel(const T* phi0, const T* pi0, const T* phi1, const T* pi1, int nf,
                                   int N, double q, int model, double* rows) {
  __shared__ double sh[kThreads / 32][kSlots];
  const long long V = (long long)N * N * N, NN = (long long)N * N;
  double s[kSlots];
  for (int k = 0; k < kSlots; ++k) s[k] = 0.0;
  const T* fl[2] = {phi0, phi1};
  const T* mo[2] = {pi0, pi1};
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / NN);
    const long long xp = x + 1 < N ? n + 1 : n + 1 - N;
    const long long yp = y + 1 < N ? n + N : n + N - NN;
    const long long zp = z + 1 < N ? n + NN : n + NN - V;
    double f[2] = {0.0, 0.0};
    for (int c = 0; c < nf; ++c) {
      const double p = (double)fl[c][n], m = (double)mo[c][n];
      f[c] = p;
      const double gx = (double)fl[c][xp] - p, gy = (double)fl[c][yp] - p, gz = (double)fl[c][zp] - p;
      s[0 + c] += m * m;                      // sum pi^2
      s[2 + c] += gx * gx + gy * gy + gz * gz;  // sum (grad^+ phi)^2
      s[6 + c] += p;
      s[8 + c] += p * p;
      s[10 + c] += m;
      if (!isfinite(m)) s[15] += 1.0;
    }
    // potential terms (eq. PotNat)
    s[4] += 0.25 * f[0] * f[0] * f[0] * f[0];
    if (model == CL_MODEL_LPHI4_CHI) s[5] += 0.5 * q * f[0] * f[0] * f[1] * f[1];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < kSlots; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[w][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < kSlots) {
    double v = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) v += sh[i][threadIdx.x];
    rows[(size_t)blockIdx.x * kSlots + threadIdx.x] = v;
  }
}

// Rows summed in a fixed order, then normalised (eqs. KandGprogramUnits, EK_EG_EV).
__global__ void avg_final_kernel(const double* rows, int nblk, int nf, int N, double dx, double a,
                                 double* out) {
  __shared__ double tot[kSlots];
  if (threadIdx.x < kSlots) {
    double v = 0.0;
    for (int i = 0; i < nblk; ++i) v += rows[(size_t)i * kSlots + threadIdx.x];
    tot[threadIdx.x] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double V = (double)N * N * N, a2 = a * a, a6 = a2 * a2 * a2;
  double rho = 0.0;
  for (int c = 0; c < 2; ++c) {
    const bool on = c < nf;
    out[0 + c] = on ? tot[0 + c] / (2.0 * a6 * V) : 0.0;                // E_K per field
    out[2 + c] = on ? tot[2 + c] / (2.0 * a2 * dx * dx * V) : 0.0;      // E_G per field
    out[6 + c] = on ? tot[6 + c] / V : 0.0;                              // <phi>
    out[8 + c] = on ? tot[8 + c] / V : 0.0;                              // <phi^2>
    out[10 + c] = on ? tot[10 + c] / V : 0.0;                            // <pi>
    out[12 + c] = on ? tot[0 + c] / V : 0.0;                             // <pi^2>
    rho += out[0 + c] + out[2 + c];
  }
  out[4] = tot[4] / V;  // E_V per potential term
  out[5] = tot[5] / V;
  out[14] = rho + out[4] + out[5];
  out[15] = tot[15];
}

cl_status scratch_for_current_device(cudaStream_t st, double** ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CL_ECUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return CL_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_avg_scratch) != cudaSuccess || !p) return CL_ECUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  } else if (!g_scratch_ptr[dev]) {
    return CL_ECUDA;  // no uncaptured call on this device yet
  }
  *ptr = g_scratch_ptr[dev];
  return CL_OK;
}

}  // namespace

extern "C" cl_status cl_volume_averages_noalloc(int model, int N, double kIR, double a, double q,
                                                int precision, const void* const* arrays,
                                                double* out, void* stream) {
  if (model != CL_MODEL_LPHI4 && model != CL_MODEL_LPHI4_CHI) return CL_EINVAL;
  if (N < 2 || N > CL_NOALLOC_MAX_N) return CL_EINVAL;  // beyond the no-allocation limit
  if (!(kIR > 0.0) || !(a > 0.0) || !arrays || !out) return CL_EINVAL;
  if (precision != CL_FP32 && precision != CL_FP64) return CL_EINVAL;
  const int nf = model == CL_MODEL_LPHI4 ? 1 : 2;
  for (int i = 0; i < 2 * nf; ++i)
    if (!arrays[i]) return CL_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* rows = nullptr;
  cl_status s = scratch_for_current_device(st, &rows);
  if (s != CL_OK) return s;
  const long long V = (long long)N * N * N;
  long long want = (V + kThreads - 1) / kThreads;
  const int nblk = (int)(want < kMaxBlocks ? want : kMaxBlocks);
  const void* p1 = nf > 1 ? arrays[2] : arrays[0];
  const void* m1 = nf > 1 ? arrays[3] : arrays[1];
  if (precision == CL_FP32)
    avg_partial_kernel<float><<<nblk, kThreads, 0, st>>>(
        (const float*)arrays[0], (const float*)arrays[1], (const float*)p1, (const float*)m1, nf, N, q,
        model, rows);
  else
    avg_partial_kernel<double><<<nblk, kThreads, 0, st>>>(
        (const double*)arrays[0], (const double*)arrays[1], (const double*)p1, (const double*)m1, nf, N,
        q, model, rows);
  if (cudaGetLastError() != cudaSuccess) return CL_ECUDA;
  const double dx = 2.0 * 3.14159265358979323846 / ((double)N * kIR);
  avg_final_kernel<<<1, 32, 0, st>>>(rows, nblk, nf, N, dx, a, out);
  if (cudaGetLastError() != cudaSuccess) return CL_ECUDA;
  return CL_OK;
}
