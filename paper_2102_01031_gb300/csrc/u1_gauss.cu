// u1_gauss.cu -- U(1) Gauss law: initial link momenta and the constraint monitor.
//
// Lattice Gauss law (CosmoLattice manual Sec. 4.2 eq. GaussU1-eom, in the
// Hamiltonian variables of Sec. 4.3):
//   sum_i grad^-_i pi_A,i = (f_s/omega_s)^2 2 gQ Im[phi^* pi_phi]
//                         = (f_s/omega_s)^2 gQ (phi_0 pi_1 - phi_1 pi_0).
// Initial link momenta (eq. GaugeCurrentFluc on the lattice): with the
// backward-difference symbol kappa_i = (1 - e^{-2 pi i n_i/N})/dx,
//   pi_A,i(n~) = conj(kappa_i) rho(n~) / |kappa|^2,  n~ != 0.
#include "common.cuh"

namespace clg {

template <typename T>
__device__ __forceinline__ double rho_at(const LatConst& L, int parity, long long n) {
  const T* f0 = reinterpret_cast<const T*>(L.buf[parity][0]);
  const T* p0 = reinterpret_cast<const T*>(L.buf[parity][1]);
  const T* f1 = reinterpret_cast<const T*>(L.buf[parity][2]);
  const T* p1 = reinterpret_cast<const T*>(L.buf[parity][3]);
  return L.fo2 * L.gQ * ((double)f0[n] * (double)p1[n] - (double)f1[n] * (double)p0[n]);
}

__global__ void u1_gauss_rho_kernel(const LatConst* Lc, int parity, double2* rho) {
  const LatConst& L = *Lc;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < L.V;
       n += (long long)gridDim.x * blockDim.x) {
    const double r = L.esz == 4 ? rho_at<float>(L, parity, n) : rho_at<double>(L, parity, n);
    rho[n] = make_double2(r, 0.0);
  }
}

__global__ void u1_gauss_modes_kernel(const double2* rho, double2* E, int N, int i, double dx) {
  const long long V = (long long)N * N * N;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= V) return;
  if (idx == 0) {
    E[0] = make_double2(0.0, 0.0);
    return;
  }
  const int n3[3] = {(int)(idx % N), (int)((idx / N) % N), (int)(idx / ((long long)N * N))};
  double kk = 0.0, kr = 0.0, ki = 0.0;
  for (int j = 0; j < 3; ++j) {
    double s, c;
    sincospi(2.0 * (double)n3[j] / (double)N, &s, &c);
    const double re = (1.0 - c) / dx, im = s / dx;  // 1 - e^{-i t} = (1 - cos t) + i sin t
    kk += re * re + im * im;
    if (j == i) {
      kr = re;
      ki = im;
    }
  }
  const double2 r = rho[idx];
  // conj(kappa_i) * rho / |kappa|^2
  E[idx] = make_double2((kr * r.x + ki * r.y) / kk, (kr * r.y - ki * r.x) / kk);
}

template <typename T>
__global__ void u1_take_real_kernel(const double2* E, T* out, long long V) {
  const double inv = 1.0 / (double)V;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = (T)(E[n].x * inv);
}
template __global__ void u1_take_real_kernel<float>(const double2*, float*, long long);
template __global__ void u1_take_real_kernel<double>(const double2*, double*, long long);

template <typename T>
__device__ void gauss_sums(const LatConst& L, int parity, double& sd, double& ss, double& mx) {
  const int N = L.N;
  const long long NN = (long long)N * N;
  const T* pA[3];
  for (int i = 0; i < 3; ++i) pA[i] = reinterpret_cast<const T*>(L.buf[parity][2 * (2 + i) + 1]);
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < L.V;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / NN);
    const long long nx = (x ? n - 1 : n + N - 1), ny = (y ? n - N : n + NN - N),
                    nz = (z ? n - NN : n + L.V - NN);
    const double lhs = (((double)pA[0][n] - (double)pA[0][nx]) + ((double)pA[1][n] - (double)pA[1][ny]) +
                        ((double)pA[2][n] - (double)pA[2][nz])) / L.dx;
    const double rhs = rho_at<T>(L, parity, n);
    const double d = fabs(lhs - rhs);
    sd += d;
    ss += fabs(lhs + rhs);
    mx = fmax(mx, d);
  }
}

// Per-block sums of |L - R|, |L + R| and max |L - R|.
__global__ void u1_gauss_monitor_kernel(const LatConst* Lc, int parity, double* part) {
  __shared__ double sh[3][32];
  double sd = 0.0, ss = 0.0, mx = 0.0;
  if (Lc->esz == 4) gauss_sums<float>(*Lc, parity, sd, ss, mx);
  else gauss_sums<double>(*Lc, parity, sd, ss, mx);
  for (int o = 16; o > 0; o >>= 1) {
    sd += __shfl_down_sync(0xffffffffu, sd, o);
    ss += __shfl_down_sync(0xffffffffu, ss, o);
    mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = sd;
    sh[1][w] = ss;
    sh[2][w] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      a += sh[0][i];
      b += sh[1][i];
      m = fmax(m, sh[2][i]);
    }
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = m;
  }
}

__global__ void u1_gauss_final_kernel(const double* part, int nblk, long long V, double* out) {
  if (threadIdx.x | blockIdx.x) return;
  double a = 0.0, b = 0.0, m = 0.0;
  for (int i = 0; i < nblk; ++i) {
    a += part[3 * i];
    b += part[3 * i + 1];
    m = fmax(m, part[3 * i + 2]);
  }
  out[0] = b > 0.0 ? a / b : 0.0;
  out[1] = a / (double)V;
  out[2] = b / (double)V;
  out[3] = m;
}

cudaError_t launch_u1_gauss_init(const LatConst* L, int parity, double2* rho, double2* E, int N,
                                 int i, double dx, int fp32, void* out, long long V, int stage,
                                 cudaStream_t st) {
  const int tb = 256;
  const int g = (int)((V + tb - 1) / tb < 65536 ? (V + tb - 1) / tb : 65536);
  if (stage == 0) {
    u1_gauss_rho_kernel<<<g, tb, 0, st>>>(L, parity, rho);
  } else if (stage == 1) {
    u1_gauss_modes_kernel<<<(unsigned)((V + tb - 1) / tb), tb, 0, st>>>(rho, E, N, i, dx);
  } else {
    if (fp32) u1_take_real_kernel<float><<<g, tb, 0, st>>>(E, (float*)out, V);
    else u1_take_real_kernel<double><<<g, tb, 0, st>>>(E, (double*)out, V);
  }
  return cudaGetLastError();
}

cudaError_t launch_u1_gauss_monitor(const LatConst* L, int parity, double* part, int nblk,
                                    long long V, cudaStream_t st) {
  u1_gauss_monitor_kernel<<<nblk, 256, 0, st>>>(L, parity, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  u1_gauss_final_kernel<<<1, 32, 0, st>>>(part, nblk, V, part + 3 * nblk);
  return cudaGetLastError();
}

}  // namespace clg
