// adjoint_kernels.cu -- seeds of the adjoint sweep: the gradient of the final
// observable with respect to the final state (outside the timed loop).
//
// Objective 0, the chi energy fraction J = (E_K^chi + E_G^chi)/rho of the
// two-field model, with (eq. EK_EG_EV, gradient term with forward differences)
//   dE_K^f/dpi_f = pi_f/(a^6 V),   dE_G^f/dphi_f = -Lap phi_f/(a^2 dx^2 V),
//   dE_V/dphi_f  = dV/dphi_f / V:
//   dJ/dpi_f  = (delta_{f,chi} - J) pi_f/(a^6 V rho)
//   dJ/dphi_f = [delta_{f,chi} dE_G^f/dphi_f - J (dE_G^f/dphi_f + dE_V/dphi_f)]/rho
//   dJ/dq (explicit) = -(J/rho) <phi^2 chi^2/2>,
//   dJ/da = [-(6 E_K^chi + 2 E_G^chi) + J (6 E_K + 2 E_G)]/(a rho)
// (E_K ~ a^-6, E_G ~ a^-2 at fixed phi, pi; the seed of lam_a with
// self-consistent expansion).
// Objective 1, one bin of the binned spectrum (eq. discretePS) of an array u:
//   J = C_b sum_{n in b} |F(n)|^2, F = sum_x u(x) e^{-ik.x},
//   C_b = k_b^3/(2 pi^2) (dx/N)^3/(4 pi nbar_b^2),
//   dJ/du(x) = 2 C_b Re[ sum_{n in b} F(n) e^{+ik.x} ].
#include <algorithm>

#include "common.cuh"

namespace clg {

template <typename T>
__global__ void seed_chi_fraction_kernel(const LatConst* Lc, const LatScalars* Sc, int parity, T* lphi0,
                                         T* lpi0, T* lphi1, T* lpi1, double* part) {
  __shared__ double red[256 / 32];
  const LatConst& L = *Lc;
  const LatScalars& S = *Sc;
  const int N = L.N;
  const long long V = L.V, NN = (long long)N * N;
  const double rho = S.obs.rho, J = (S.obs.EK[1] + S.obs.EG[1]) / rho;
  const double a = S.a, a2 = a * a, a6 = a2 * a2 * a2;
  const double kK = 1.0 / (a6 * (double)V * rho), kG = -L.inv_dx2 / (a2 * (double)V), q = L.q;
  const T* ph[2] = {reinterpret_cast<const T*>(L.buf[parity][0]), reinterpret_cast<const T*>(L.buf[parity][2])};
  const T* pm[2] = {reinterpret_cast<const T*>(L.buf[parity][1]), reinterpret_cast<const T*>(L.buf[parity][3])};
  T* lf[2] = {lphi0, lphi1};
  T* lp[2] = {lpi0, lpi1};
  double s = 0.0;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(n % N), y = (int)((n / N) % N), z = (int)(n / NN);
    const long long xp = x + 1 < N ? n + 1 : n + 1 - N, xm = x > 0 ? n - 1 : n + N - 1;
    const long long yp = y + 1 < N ? n + N : n + N - NN, ym = y > 0 ? n - N : n + NN - N;
    const long long zp = z + 1 < N ? n + NN : n + NN - V, zm = z > 0 ? n - NN : n + V - NN;
    const double f0 = (double)ph[0][n], f1 = (double)ph[1][n];
    const double d[2] = {f0 * f0 * f0 + q * f0 * f1 * f1, q * f0 * f0 * f1};
    for (int g = 0; g < 2; ++g) {
      const T* u = ph[g];
      const double c = (double)u[n];
      const double lap = ((double)u[xp] + (double)u[xm] - 2.0 * c) + ((double)u[yp] + (double)u[ym] - 2.0 * c) +
                         ((double)u[zp] + (double)u[zm] - 2.0 * c);
      const double dEG = kG * lap;
      const double chi = g == 1 ? 1.0 : 0.0;
      lp[g][n] = (T)((chi - J) * (double)pm[g][n] * kK);
      lf[g][n] = (T)((chi * dEG - J * (dEG + d[g] / (double)V)) / rho);
    }
    s += 0.5 * f0 * f0 * f1 * f1;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// J and the explicit dJ/dq of objective 0: out[0] = J, out[1] = -(J/rho) <phi^2 chi^2/2>;
// with self-consistent expansion also the seed of lam_a, Sc->adja = dJ/da.
__global__ void chi_fraction_final_kernel(const double* part, int nblk, const LatConst* Lc,
                                          LatScalars* Sc, double* out) {
  if (threadIdx.x | blockIdx.x) return;
  double s = 0.0;
  for (int i = 0; i < nblk; ++i) s += part[i];
  const cl_energies_t& o = Sc->obs;
  const double rho = o.rho, J = (o.EK[1] + o.EG[1]) / rho;
  out[0] = J;
  out[1] = -J / rho * s * Lc->inv_V;
  if (Lc->expansion == CL_EXP_SELF) {
    double ek = 0.0, eg = 0.0;
    for (int k = 0; k < 4; ++k) {
      ek += o.EK[k];
      eg += o.EG[k];
    }
    Sc->adja = (-(6.0 * o.EK[1] + 2.0 * o.EG[1]) + J * (6.0 * ek + 2.0 * eg)) / (Sc->a * rho);
  }
}

// Objective 1: keep bin b of F scaled by 2 C_b (zero elsewhere); bins[] holds
// (k_b, delta_b, mult_b) rows of length nb as written by the bin kernels.
// out[0] = J = delta_b.
__global__ void spectrum_seed_mask_kernel(double2* F, int N, double dk, int nb, int bin, const double* bins,
                                          double kIR, double dx, double* out) {
  const long long V = (long long)N * N * N;
  const double kb = bins[bin], nbar = kb / kIR;
  const double pi = 3.14159265358979323846;
  const double fac = dx / (double)N;
  const double Cb = kb * kb * kb / (2.0 * pi * pi) * fac * fac * fac / (4.0 * pi * nbar * nbar);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < V;
       idx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(idx % N), y = (int)((idx / N) % N), z = (int)(idx / ((long long)N * N));
    const int nx = x <= N / 2 ? x : x - N, ny = y <= N / 2 ? y : y - N, nz = z <= N / 2 ? z : z - N;
    const double nn = sqrt((double)(nx * nx + ny * ny + nz * nz));
    int b = (int)floor(nn / dk);
    if (b >= nb) b = nb - 1;
    const bool keep = idx != 0 && b == bin;
    const double2 v = F[idx];
    F[idx] = keep ? make_double2(2.0 * Cb * v.x, 2.0 * Cb * v.y) : make_double2(0.0, 0.0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = bins[nb + bin];
    out[1] = 0.0;
  }
}

template <typename T>
__global__ void real_part_kernel(const double2* F, T* out, long long V) {
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < V;
       n += (long long)gridDim.x * blockDim.x)
    out[n] = (T)F[n].x;
}

cudaError_t launch_seed_chi_fraction(int fp32, const LatConst* L, LatScalars* S, int parity,
                                     void* const* lam, double* part, int nblk, double* out,
                                     cudaStream_t st) {
  if (fp32)
    seed_chi_fraction_kernel<float><<<nblk, 256, 0, st>>>(L, S, parity, (float*)lam[0], (float*)lam[1],
                                                          (float*)lam[2], (float*)lam[3], part);
  else
    seed_chi_fraction_kernel<double><<<nblk, 256, 0, st>>>(L, S, parity, (double*)lam[0], (double*)lam[1],
                                                           (double*)lam[2], (double*)lam[3], part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  chi_fraction_final_kernel<<<1, 32, 0, st>>>(part, nblk, L, S, out);
  return cudaGetLastError();
}

cudaError_t launch_spectrum_seed(int fp32, double2* F, int N, double dk, int nb, int bin, const double* bins,
                                 double kIR, double dx, double* out, int stage, void* lam, cudaStream_t st) {
  const long long V = (long long)N * N * N;
  const int g = (int)std::min<long long>((V + 255) / 256, 4096);
  if (stage == 0) {
    spectrum_seed_mask_kernel<<<g, 256, 0, st>>>(F, N, dk, nb, bin, bins, kIR, dx, out);
  } else if (fp32) {
    real_part_kernel<float><<<g, 256, 0, st>>>(F, (float*)lam, V);
  } else {
    real_part_kernel<double><<<g, 256, 0, st>>>(F, (double*)lam, V);
  }
  return cudaGetLastError();
}

}  // namespace clg
