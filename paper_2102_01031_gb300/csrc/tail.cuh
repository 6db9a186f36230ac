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

// The tail runs once per pass, on one thread, between passes: its cost is the
// number of FP64 operations (each takes tens of cycles on this part, even when
// independent), so integer powers use the fewest multiplications and general
// powers go through one out-of-line pow.
static __device__ __noinline__ double pow_out_of_line(double a, double e) { return pow(a, e); }

// x^n by squaring with the fewest products (x^2: one, x^4: two, x^0: none).
__device__ __forceinline__ double ipow(double x, int n) {
  const bool neg = n < 0;
  int m = neg ? -n : n;
  double r = 1.0, p = x;
  bool have = false;
  while (m) {
    if (m & 1) {
      r = have ? r * p : p;
      have = true;
    }
    m >>= 1;
    if (m) p = p * p;
  }
  return neg ? 1.0 / r : r;
}

// a^(m alpha + k): by multiplication when alpha is a small integer (alpha = 1
// or 0 in the manual's scenarios), pow otherwise.
__device__ __forceinline__ double apow(const LatConst& L, double a, int m, int k) {
  if (L.int_alpha) return ipow(a, m * L.alpha_i + k);
  return pow_out_of_line(a, m * L.alpha + k);
}

__device__ __forceinline__ double fixed_p(const LatConst& L) {
  return 2.0 / (3.0 * (1.0 + L.omega_eos) - 2.0 * L.alpha);
}

// Fixed power-law background, eq. ScaleFactorPowerLaw.
template <class SS>
__device__ __forceinline__ double a_fixed(const LatConst& L, const SS& S, double eta) {
  double p = fixed_p(L);
  return S.a0 * pow_out_of_line(1.0 + S.Hfix * (eta - S.eta0) / p, p);
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

// The factor a^{2alpha+1}/3 (f_s/m_p)^2 that both Friedmann kicks of a pass share.
__device__ __forceinline__ double kernel_a_pref(const LatConst& L, double a) {
  return apow(L, a, 2, 1) * (1.0 / 3.0) * L.fm2;
}

// Friedmann kicks of b (kick-out with the pre-kick momenta, then kick-in with
// the post-kick momenta, as in the velocity-Verlet step), pref = kernel_a_pref
// at the current a.
template <class SS>
__device__ inline void advance_scalars(const PassArgs& P, const LatConst& L, SS& S,
                                       const PassSums& E, bool have_sums, double pref) {
  if (have_sums && L.expansion == CL_EXP_SELF) {
    const double al = L.alpha;
    const double common = al * E.EG + (al + 1.0) * E.EV;
    S.b += P.wout * (pref * ((al - 2.0) * E.EKpre + common + (al - 1.0) * (E.EKApre + E.EGA)));
    S.b += P.win * (pref * ((al - 2.0) * E.EKpost + common + (al - 1.0) * (E.EKA + E.EGA)));
  }
}
template <class SS>
__device__ inline void advance_scalars(const PassArgs& P, const LatConst& L, SS& S,
                                       const PassSums& E, bool have_sums) {
  if (have_sums && L.expansion == CL_EXP_SELF) advance_scalars(P, L, S, E, true, kernel_a_pref(L, S.a));
}

// The two Friedmann kicks of a pass for the scalar models (no U(1) energies),
// merged:  b += pref [(alpha-2)(w_out E_K^pre + w_in E_K^post) + (w_out + w_in)(alpha E_G + (alpha+1) E_V)].
// FriedPre holds the factors that do not depend on the pass's sums.
struct FriedPre {
  double pref, am2, al, ap1, wout, win, ws;
};
__device__ __forceinline__ FriedPre friedmann_pre(const LatConst& L, double a, double wout, double win) {
  FriedPre F;
  F.pref = kernel_a_pref(L, a);
  F.al = L.alpha;
  F.am2 = L.alpha - 2.0;
  F.ap1 = L.alpha + 1.0;
  F.wout = wout;
  F.win = win;
  F.ws = wout + win;
  return F;
}
__device__ __forceinline__ double friedmann_kicks_scalar(const FriedPre& F, const PassSums& E, double b) {
  const double ek = fma(F.win, E.EKpost, F.wout * E.EKpre);
  const double common = fma(F.ap1, E.EV, F.al * E.EG);
  return fma(F.pref, fma(F.am2, ek, F.ws * common), b);
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

// The drift of a by P.dnext and the drift coefficients of the next pass:
//   a' = a + dnext b (self-consistent) or a(eta + dnext) (fixed power law),
//   cd = dnext abar^{alpha-3}, cdA = dnext abar^{alpha-1}, abar = (a + a')/2,
//   and the kick's a'^{1+alpha}, a'^{3+alpha}, a'^{alpha-1}.
// Few FP64 operations: alpha's exponents are read once, negative powers are
// reciprocals of positive ones, and alpha = 1 (the manual's default) is
// straight-line code.
// Drift coefficients of a drift dn at the midpoint scale factor abar: fields
// h abar^{alpha-3}, links h abar^{alpha-1} (Sec. 3.5.2; Sec. 4.3 for the links).
__device__ inline void drift_coefficients(const LatConst& L, double abar, double dn, double& cd, double& cdA) {
  const int ia = L.alpha_i;
  if (L.int_alpha && ia == 1) {
    cd = dn * (1.0 / (abar * abar));
    cdA = dn;
  } else if (L.int_alpha) {
    cd = dn * ipow(abar, ia - 3);
    cdA = dn * ipow(abar, ia - 1);
  } else {
    cd = dn * pow_out_of_line(abar, L.alpha - 3.0);
    cdA = dn * pow_out_of_line(abar, L.alpha - 1.0);
  }
}

template <class SS>
__device__ inline void advance_drift(const PassArgs& P, const LatConst& L, SS& S) {
  const double a = S.a, dn = P.dnext;
  if (dn == 0.0) {
    S.cd = 0.0;
    S.cdA = 0.0;
    return;
  }
  double an;
  if (L.expansion == CL_EXP_SELF) an = fma(dn, S.b, a);
  else if (L.expansion == CL_EXP_FIXED) an = a_fixed(L, S, S.eta + dn);
  else an = a;
  const double abar = 0.5 * (a + an);
  S.a = an;
  S.eta += dn;
  if (L.expansion == CL_EXP_FIXED) S.b = an * H_fixed(L, S, S.eta);
  const int ia = L.alpha_i;
  drift_coefficients(L, abar, dn, S.cd, S.cdA);
  if (L.int_alpha && ia == 1) {
    const double an2 = an * an;
    S.apow1 = an2;
    S.apow3 = an2 * an2;
    S.apowm1 = 1.0;
  } else if (L.int_alpha) {
    S.apow1 = ipow(an, ia + 1);
    S.apow3 = S.apow1 * (an * an);
    S.apowm1 = ipow(an, ia - 1);
  } else {
    S.apow1 = pow_out_of_line(an, L.alpha + 1.0);
    S.apow3 = S.apow1 * (an * an);
    S.apowm1 = pow_out_of_line(an, L.alpha - 1.0);
  }
}

// Hubble-constraint monitor and energy bookkeeping of a measurement.
template <class SS>
__device__ inline void finish_obs(const PassArgs& P, const LatConst& L, SS& S, cl_energies_t& o) {
  double rho = o.EKA + o.EGA + o.EKB + o.EGB;
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
