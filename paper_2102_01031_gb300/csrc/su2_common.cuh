// su2_common.cuh -- what the two doublet-model passes share: the layout of the
// state's arrays, the quaternion algebra of SU(2) links (U = u0 - i u.s, s the
// Pauli matrices, stored as (u0, u1, u2, u3)), the doublet's hops, and the end
// of a pass (the CTA's partial sums, the last CTA's lattice sums, the Friedmann
// and measurement update of the scalar state).
#pragma once

#include "common.cuh"
#include "tail.cuh"

namespace clg {

enum : int { SF = 0, SP = 4, SA = 8, SPA = 11, SU = 14, SPB = 26, SNARR = 35,
              // lphi4SU2U1: singlet, its momentum, vphi components, their momenta
              SS = 35, SPS = 36, SC = 37, SPC = 39, SNARR_FULL = 41 };

template <typename T> struct alignas(4 * sizeof(T)) Q4 {
  T w, x, y, z;
};

// Quaternion algebra of the link convention U = u0 - i u.s:
// (a0 - i a.s)(b0 - i b.s) = (a0 b0 - a.b) - i (a0 b + b0 a + a x b).s
template <typename T>
__device__ __forceinline__ Q4<T> qmul(const Q4<T>& a, const Q4<T>& b) {
  Q4<T> r;
  r.w = fmaT(-a.z, b.z, fmaT(-a.y, b.y, fmaT(-a.x, b.x, a.w * b.w)));
  r.x = fmaT(a.y, b.z, fmaT(-a.z, b.y, fmaT(b.w, a.x, a.w * b.x)));
  r.y = fmaT(a.z, b.x, fmaT(-a.x, b.z, fmaT(b.w, a.y, a.w * b.y)));
  r.z = fmaT(a.x, b.y, fmaT(-a.y, b.x, fmaT(b.w, a.z, a.w * b.z)));
  return r;
}
template <typename T>
__device__ __forceinline__ Q4<T> qconj(const Q4<T>& a) {
  Q4<T> r;
  r.w = a.w;
  r.x = -a.x;
  r.y = -a.y;
  r.z = -a.z;
  return r;
}
template <typename T>
__device__ __forceinline__ void qadd(Q4<T>& s, const Q4<T>& a) {
  s.w += a.w;
  s.x += a.x;
  s.y += a.y;
  s.z += a.z;
}

// cos x and sin(x)/x.  FP32: for x^2 <= (pi/4)^2 their Taylor series about 0
// in Horner form (first omitted terms below 3e-9 there), else the library;
// the drift angles are small in practice.  FP64: the library.
__device__ __forceinline__ void cos_sinc(float x2, float& c, float& sc) {
  if (x2 <= 0.61685028f) {
    c = cos_taylor(x2);
    sc = sin_taylor(x2);
  } else {
    const float x = sqrtf(x2);
    float s;
    sincos_slow(x, &s, &c);
    sc = s / x;
  }
}
__device__ __forceinline__ void cos_sinc(double x2, double& c, double& sc) {
  if (x2 == 0.0) {
    c = 1.0;
    sc = 1.0;
    return;
  }
  const double x = sqrt(x2);
  double s;
  sincos(x, &s, &c);
  sc = s / x;
}


// Renormalise a link to unit length (FP32 storage only: keeps the rounding
// of repeated drifts from walking off the group; FP64 follows the plain
// products).
__device__ __forceinline__ void renorm(Q4<float>& u) {
  const float r = rsqrtf(u.w * u.w + u.x * u.x + u.y * u.y + u.z * u.z);
  u.w *= r;
  u.x *= r;
  u.y *= r;
  u.z *= r;
}
__device__ __forceinline__ void renorm(Q4<double>&) {}

// U psi and U^dag psi for psi = (p, q) = (w + i x, y + i z) held in a quaternion slot
template <typename T>
__device__ __forceinline__ Q4<T> umul(const Q4<T>& u, const Q4<T>& f) {
  Q4<T> r;
  r.w = u.w * f.w + u.z * f.x - u.y * f.y + u.x * f.z;
  r.x = u.w * f.x - u.z * f.w - u.y * f.z - u.x * f.y;
  r.y = u.y * f.w + u.x * f.x + u.w * f.y - u.z * f.z;
  r.z = u.y * f.x - u.x * f.w + u.w * f.z + u.z * f.y;
  return r;
}
template <typename T>
__device__ __forceinline__ Q4<T> udmul(const Q4<T>& u, const Q4<T>& f) {
  Q4<T> r;
  r.w = u.w * f.w - u.z * f.x + u.y * f.y - u.x * f.z;
  r.x = u.w * f.x + u.z * f.w + u.y * f.z + u.x * f.y;
  r.y = -u.y * f.w - u.x * f.x + u.w * f.y + u.z * f.z;
  r.z = -u.y * f.x + u.x * f.w + u.w * f.z - u.z * f.y;
  return r;
}
// multiply both components by exp(-i t) given (c, s) = (cos t, sin t); (c, -s) gives exp(+i t)
template <typename T>
__device__ __forceinline__ void phase(Q4<T>& f, T c, T s) {
  const T w = f.w * c + f.x * s, x = f.x * c - f.w * s;
  const T y = f.y * c + f.z * s, z = f.z * c - f.y * s;
  f.w = w;
  f.x = x;
  f.y = y;
  f.z = z;
}

// 1 - w for a unit quaternion, without cancellation: |v|^2/(1 + w)
template <typename T>
__device__ __forceinline__ T one_minus_w(const Q4<T>& p) {
  return (p.x * p.x + p.y * p.y + p.z * p.z) / (T(1) + p.w);
}

constexpr int SU2_NQ = 30;  // partial sums per CTA (the measurement pass uses 23, 29 for lphi4SU2U1)

constexpr int SU2_TY = 8;  // tile height of the passes; the width TX (32 or 16) is a template parameter

// End of a doublet pass, all threads of the CTA: warp sums of the accumulators
// into red_s, the CTA's slot of P.partials, and in the last CTA to arrive the
// fixed-order lattice sums, the energies (RED 2), the scale-factor update and
// the drift coefficients of the next pass.  RED: 0 no sums, 1 the Friedmann
// kicks' sums, 2 a full measurement.
template <typename T, int RED, bool FULL, int NACC>
__device__ void su2_pass_end(const PassArgs& P, const LatConst& L, Acc<T> (&acc)[NACC], float nonfinite,
                             double (*red_s)[9], unsigned& last_s, int tid, int lane, int warp, int nth) {
  if constexpr (RED > 0) {
    const int nw = nth >> 5;
#pragma unroll
    for (int q = 0; q < NACC; ++q) {
      const double v = warp_sum(acc[q]);
      if (lane == 0) red_s[q][warp] = v;
    }
    if constexpr (RED == 2) {
      float nf = nonfinite;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nf += __shfl_down_sync(0xffffffffu, nf, o);
      if (lane == 0) red_s[NACC][warp] = (double)nf;
    }
    __syncthreads();
    constexpr int NOUT = RED == 2 ? NACC + 1 : NACC;
    if (tid < NOUT) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += red_s[tid][w];
      P.partials[(size_t)tid * gridDim.x + blockIdx.x] = s;
    }
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    last_s = atomicAdd(&P.counters[0], 1u) == gridDim.x - 1 ? 1u : 0u;
  }
  __syncthreads();
  if (!last_s) return;
  __threadfence();
  constexpr int NOUT = RED == 0 ? 0 : (RED == 2 ? NACC + 1 : NACC);
  for (int q = warp; q < NOUT; q += nth >> 5) {
    const double s = warp_slot_sum(P.partials, q * gridDim.x, (q + 1) * gridDim.x, lane);
    if (lane == 0) red_s[q][0] = s;
  }
  __syncthreads();
  if (tid != 0) return;
  ScalarState W;
  load_state_cg(W, P.sc);
  const double a = W.a, a2 = a * a, a4 = a2 * a2, a6 = a4 * a2;
  const double gdx2 = L.gQ * L.dx * L.dx, bdx2 = L.gQB * L.dx * L.dx;
  const double kphi = 0.5 * L.inv_V / a6;                                  // E_K per sum of pi_c^2
  const double gphi = 0.5 * L.inv_V * L.inv_dx2 / a2;                      // E_G per sum |W psi(n+i) - psi|^2
  const double kA = 0.5 * L.inv_V / (L.fo2 * a4);                          // E_K^A, E_K^B per sum of momenta^2
  const double mA = gdx2 != 0.0 ? L.inv_V / (L.fo2 * a4 * gdx2 * gdx2) : 0.0;  // E_G^A per sum (1 - cos)
  const double mB = 4.0 * L.inv_V / (L.fo2 * a4 * bdx2 * bdx2);           // E_G^B per sum (1 - Tr U_ij/2)
  PassSums E = {0, 0, 0, 0, 0, 0, 0};
  double EKA = 0, EKB = 0, EGA = 0, EGB = 0;
  if (RED > 0) {
    double spost, slinks;
    if (RED == 1) {
      spost = red_s[0][0];
      slinks = red_s[1][0];
      E.EG = red_s[2][0] * gphi;
      EGA = red_s[3][0] * mA;
      EGB = red_s[4][0] * mB;
      E.EV = red_s[5][0] * L.inv_V;
    } else {
      spost = red_s[0][0] + red_s[1][0] + red_s[2][0] + red_s[3][0];
      slinks = red_s[4][0] + red_s[5][0];
      EKA = red_s[4][0] * kA;
      EKB = red_s[5][0] * kA;
      E.EG = red_s[6][0] * gphi;
      EGA = red_s[7][0] * mA;
      EGB = red_s[8][0] * mB;
      E.EV = red_s[9][0] * L.inv_V;
      if (FULL) {  // the Friedmann kicks take the totals of the three scalar species
        spost += red_s[23][0] + red_s[24][0];
        E.EG += (red_s[25][0] + red_s[26][0]) * gphi;
        E.EV += (red_s[27][0] + red_s[28][0]) * L.inv_V;
      }
    }
    // the two link sectors enter the Friedmann kicks with one coefficient, (alpha - 1)
    E.EKpre = W.pi2 * kphi;
    E.EKpost = spost * kphi;
    E.EKApre = W.pi2A * kA;
    E.EKA = slinks * kA;
    E.EGA = EGA + EGB;
    W.pi2 = spost;
    W.pi2A = slinks;
  }
  advance_scalars(P, L, W, E, RED > 0);
  if (RED == 2) {
    cl_energies_t& ob = P.sc->obs;
    for (int k2 = 0; k2 < 4; ++k2) {
      ob.EK[k2] = ob.EG[k2] = ob.EV[k2] = 0.0;
      ob.mean_phi[k2] = red_s[10 + k2][0] * L.inv_V;
      ob.mean_phi2[k2] = red_s[14 + k2][0] * L.inv_V;
      ob.mean_pi[k2] = red_s[18 + k2][0] * L.inv_V;
      ob.mean_pi2[k2] = red_s[k2][0] * L.inv_V;
    }
    ob.EK[0] = E.EKpost;
    ob.EG[0] = E.EG;
    ob.EV[0] = E.EV;
    if (FULL) {  // per species: [0] doublet, [1] singlet, [2] vphi; EV per potential term
      ob.EK[1] = red_s[23][0] * kphi;
      ob.EK[2] = red_s[24][0] * kphi;
      ob.EK[0] = E.EKpost - ob.EK[1] - ob.EK[2];
      ob.EG[0] = red_s[6][0] * gphi;
      ob.EG[1] = red_s[25][0] * gphi;
      ob.EG[2] = red_s[26][0] * gphi;
      ob.EV[0] = red_s[9][0] * L.inv_V;
      ob.EV[1] = red_s[27][0] * L.inv_V;
      ob.EV[2] = red_s[28][0] * L.inv_V;
    }
    ob.EKA = EKA;
    ob.EGA = EGA;
    ob.EKB = EKB;
    ob.EGB = EGB;
    ob.nonfinite = (int64_t)red_s[NACC][0];
    finish_obs(P, L, W, ob);
  }
  advance_drift(P, L, W);
  store_state(P.sc, W);
  P.counters[0] = 0u;
  __threadfence();
}

}  // namespace clg
