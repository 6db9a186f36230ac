// tail.cuh -- per-lattice scalar update run by the last CTA of a DK pass:
// Friedmann kicks of b = a', the next drift coefficient, and the packaging of
// measured volume averages.  FP64 throughout.
#pragma once

#include <cstddef>

#include "common.cuh"

namespace clg {

constexpr int kStateWords = (int)(sizeof(ScalarState) / sizeof(double));
static_assert(kStateWords == 14 && offsetof(LatScalars, pi2A) == 13 * sizeof(double),
              "ScalarState mirrors the leading members of LatScalars");

// The evolving scalars of a lattice, read past L1 (another SM may have
// written them earlier in the same launch), and written back.
__device__ inline void load_state_cg(ScalarState& dst, const LatScalars* src) {
  const double* s = reinterpret_cast<const double*>(src);
  double* d = reinterpret_cast<double*>(&dst);
#pragma unroll
  for (int i = 0; i < kStateWords; ++i) d[i] = __ldcg(s + i);
}
__device__ inline void store_state(LatScalars* dst, const ScalarState& src) {
  const double* s = reinterpret_cast<const double*>(&src);
  double* d = reinterpret_cast<double*>(dst);
#pragma unroll
  for (int i = 0; i < kStateWords; ++i) d[i] = s[i];
}

// Energy sums of one pass for one lattice, already summed over the lattice.
struct PassSums {
  double EKpre, EKpost, EG, EV;   // normalised energies (pre / post kick)
  double EKA, EGA;                // U(1) electric (post kick) and magnetic
  double EKApre;                  // U(1) electric before the kick
};

// a^(alpha + k): by repeated multiplication when alpha is a small integer
// (alpha = 1 or 0 in the manual's scenarios), pow otherwise.  Double pow has
// a long dependent latency and this runs between two passes.
__device__ __forceinline__ double apow(const LatConst& L, double a, int m, int k) {
  // exponent m * alpha + k
  if (L.int_alpha) {
    int e = m * (int)L.alpha + k;
    const bool neg = e < 0;
    e = neg ? -e : e;
    double x = 1.0, b = a;
    while (e) {
      if (e & 1) x *= b;
      b *= b;
      e >>= 1;
    }
    return neg ? 1.0 / x : x;
  }
  return pow(a, m * L.alpha + k);
}

__device__ __forceinline__ double fixed_p(const LatConst& L) {
  return 2.0 / (3.0 * (1.0 + L.omega_eos) - 2.0 * L.alpha);
}

// Fixed power-law background, eq. ScaleFactorPowerLaw.
template <class SS>
__device__ __forceinline__ double a_fixed(const LatConst& L, const SS& S, double eta) {
  double p = fixed_p(L);
  return S.a0 * pow(1.0 + S.Hfix * (eta - S.eta0) / p, p);
}
template <class SS>
__device__ __forceinline__ double H_fixed(const LatConst& L, const SS& S, double eta) {
  double p = fixed_p(L);
  return S.Hfix / (1.0 + S.Hfix * (eta - S.eta0) / p);
}

// b' = K_a (Sec. 3.5.2 / Sec. 4.3): a^{2alpha+1}/3 (f_s/m_p)^2 [(alpha-2) E_K + alpha E_G
//        + (alpha-1)(E_K^A + E_G^A) + (alpha+1) E_V]
__device__ __forceinline__ double kernel_a(const LatConst& L, double a, double EK, double EG,
                                           double EV, double EKA, double EGA) {
  const double al = L.alpha;
  return apow(L, a, 2, 1) * (1.0 / 3.0) * L.fm2 *
         ((al - 2.0) * EK + al * EG + (al - 1.0) * (EKA + EGA) + (al + 1.0) * EV);
}

// Friedmann kicks of b (kick-out with the pre-kick momenta, then kick-in with
// the post-kick momenta, as in the velocity-Verlet step), then the drift of a
// by P.dnext and the drift coefficients of the next pass.
template <class SS>
__device__ inline void advance_scalars(const PassArgs& P, const LatConst& L, SS& S,
                                       const PassSums& E, bool have_sums) {
  const double a = S.a;
  if (have_sums && L.expansion == CL_EXP_SELF) {
    // K_a of both kicks share a^{2alpha+1}/3 (f_s/m_p)^2 (one FP64 chain on the critical path)
    const double al = L.alpha, pref = apow(L, a, 2, 1) * (1.0 / 3.0) * L.fm2;
    const double common = al * E.EG + (al + 1.0) * E.EV;
    S.b += P.wout * (pref * ((al - 2.0) * E.EKpre + common + (al - 1.0) * (E.EKApre + E.EGA)));
    S.b += P.win * (pref * ((al - 2.0) * E.EKpost + common + (al - 1.0) * (E.EKA + E.EGA)));
  }
}

// w_in dK_a/da + w_out dK_a/da of the two Friedmann kicks of a pass (scalar
// fields), at fixed fields and momenta: with E_K ~ a^-6, E_G ~ a^-2,
//   d/da [a^{2alpha+1} E] = a^{2alpha} (2alpha+1-s) E  for E ~ a^-s.
__device__ __forceinline__ double kernel_a_da(const PassArgs& P, const LatConst& L, double a,
                                              const PassSums& E) {
  const double al = L.alpha, w = P.win + P.wout;
  return apow(L, a, 2, 0) * (1.0 / 3.0) * L.fm2 *
         ((2.0 * al - 5.0) * (al - 2.0) * (P.win * E.EKpost + P.wout * E.EKpre) +
          w * ((2.0 * al - 1.0) * al * E.EG + (2.0 * al + 1.0) * (al + 1.0) * E.EV));
}

template <class SS>
__device__ inline void advance_drift(const PassArgs& P, const LatConst& L, SS& S) {
  const double a = S.a;
  if (P.dnext != 0.0) {
    double an;
    if (L.expansion == CL_EXP_SELF) an = a + P.dnext * S.b;
    else if (L.expansion == CL_EXP_FIXED) an = a_fixed(L, S, S.eta + P.dnext);
    else an = a;
    const double abar = 0.5 * (a + an);
    S.cd = P.dnext * apow(L, abar, 1, -3);
    S.cdA = P.dnext * apow(L, abar, 1, -1);
    S.a = an;
    S.eta += P.dnext;
    if (L.expansion == CL_EXP_FIXED) S.b = an * H_fixed(L, S, S.eta);
    S.apow1 = apow(L, an, 1, 1);
    S.apow3 = apow(L, an, 1, 3);
    S.apowm1 = apow(L, an, 1, -1);
  } else {
    S.cd = 0.0;
    S.cdA = 0.0;
  }
}

// Hubble-constraint monitor and energy bookkeeping of a measurement.
template <class SS>
__device__ inline void finish_obs(const PassArgs& P, const LatConst& L, SS& S, cl_energies_t& o) {
  double rho = o.EKA + o.EGA;
  for (int k = 0; k < 4; ++k) rho += o.EK[k] + o.EG[k] + o.EV[k];
  o.rho = rho;
  o.hubble_lhs = S.b * S.b;
  o.hubble_rhs = apow(L, S.a, 2, 2) * (1.0 / 3.0) * L.fm2 * rho;
  const double den = o.hubble_lhs + o.hubble_rhs;
  o.hubble_viol = den > 0.0 ? (o.hubble_lhs - o.hubble_rhs) / den : 0.0;
  if (P.set_rho0) S.rho0 = rho;
  o.energy_cons = S.rho0 != 0.0 ? 1.0 - rho / S.rho0 : 0.0;
  o.eta = S.eta;
  o.a = S.a;
  o.b = S.b;
}

}  // namespace clg
