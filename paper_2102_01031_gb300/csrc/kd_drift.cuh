// kd_drift.cuh -- the drift coefficients of the kick-then-drift passes (the
// U(1) pass and the doublet passes without self-consistent expansion).
#pragma once

#include "tail.cuh"

namespace clg {

// The drift coefficients of a pass that drifts each site right after its kick,
// for a scale factor that does not wait for the pass's sums (no expansion, or a
// fixed power-law background): the drift over [eta, eta + dn] at the mean of
// a(eta) and a(eta + dn), the values the deferred form computes in the tail of
// the pass before.
__device__ inline void kd_drift_coefficients(const LatConst& L, const LatScalars* SC, double dn, double& cd,
                                             double& cdA) {
  ScalarState W;
  load_state_cg(W, SC);
  const double an = L.expansion == CL_EXP_FIXED ? a_fixed(L, W, W.eta + dn) : W.a;
  drift_coefficients(L, 0.5 * (W.a + an), dn, cd, cdA);
}

}  // namespace clg
