"""Pins of the oracle's modulus spectra of lphi4SU2U1's two charged fields (Sec. 4.5
outputs spectra_norm_SU2Doublet_scalar and spectra_norm_cmplx_scalar; eqs.
discretePS and OccuppationNum): which = 0 the doublet Phi, which = 1 the
U(1)-charged scalar vphi.

  * With q_G = q_H = 0 the doublet's outputs are the (separately pinned)
    doublet model's for the same state, bit for bit.
  * The mass of the occupation number is the curvature of eq. PotGauge along
    each field's canonical modulus rho = sqrt2 |field|, averaged over the
    lattice: the test differentiates the potential numerically along rho at
    every site (a dropped coupling, or a factor 2 on q_H, fails it).
  * Gauge invariance: an SU(2) x U(1) transformation, the charged scalar
    rotated with its own charge, leaves both fields' outputs unchanged.
"""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle_full import dump, full_params, full_state, load
from tests.test_oracle_su2 import gauge_transform

N, KIR = 8, 0.8


def potential(d2, s, v2, lam, v, qG, qH):
    """eq. PotGauge in program units: |Phi|^2 = d2, phi_s = s, |vphi|^2 = v2."""
    return lam * (d2 - v * v) ** 2 + qG * d2 * s * s + 2.0 * qH * d2 * v2


def curvature_mean(arrays, which, lam, v, qG, qH, h=1e-3):
    """<d^2 V/drho^2> over the sites, by central differences along the modulus rho."""
    d2 = 0.5 * sum(arrays[c] ** 2 for c in range(4))
    s = arrays[35]
    v2 = 0.5 * (arrays[37] ** 2 + arrays[38] ** 2)
    rho = np.sqrt(2.0 * (d2 if which == 0 else v2))

    def V(r):  # the potential with the chosen modulus set to r (the others fixed)
        m2 = 0.5 * r * r
        return potential(m2, s, v2, lam, v, qG, qH) if which == 0 else potential(d2, s, m2, lam, v, qG, qH)

    return float(np.mean((V(rho + h) - 2.0 * V(rho) + V(rho - h)) / (h * h)))


def occupation_from(k, d, dp, m, m2, fo2, dx):
    """eq. OccuppationNum at a = 1, a' = 0 from the shell sums behind Delta_r, Delta_r'."""
    V = float(N ** 3)
    C = (N * dx) ** 3 / (2.0 * V * V) * fo2
    nbar = k / KIR
    sh = k ** 3 / (2 * np.pi ** 2) * (dx / N) ** 3 / (4 * np.pi * nbar ** 2)
    s1, s2 = d / sh, dp / sh
    w = np.sqrt(k ** 2 + m2)
    return 2.0 * C * (w * s1 + s2 / w) / m


def test_doublet_reduces_to_the_doublet_model(oracle_mod):
    s = full_state(N, 3)
    kw = dict(expansion=O.EXP_OFF, v=0.3)
    F = O.Oracle(O.MODEL_LPHI4_SU2U1, N, KIR, 0.5, 1, full_params(qG=0.0, qH=0.0, **kw))
    D = O.Oracle(O.MODEL_SU2U1_HIGGS, N, KIR, 0.5, 1, full_params(**kw))
    load(F, s)
    load(D, s[:35])
    for L in (F, D):
        L.set_scalars(0.0, 1.3, 0.4)
    rf, rd = F.norm_spectrum(fo2=2.0, which=0), D.norm_spectrum(fo2=2.0)
    for x, y in zip(rf, rd):
        assert np.array_equal(x, y)
    with pytest.raises(ValueError):
        D.norm_spectrum(fo2=2.0, which=1)   # the doublet model has no second charged field


@pytest.mark.parametrize("which", [0, 1])
def test_mass_is_the_curvature_along_the_modulus(oracle_mod, which):
    lam, v, qG, qH = 1.0, 0.2, 1.5, 0.8
    s = full_state(N, 5)
    L = O.Oracle(O.MODEL_LPHI4_SU2U1, N, KIR, 1.0, 1,
                 full_params(lam=lam, v=v, qG=qG, qH=qH, expansion=O.EXP_OFF))
    load(L, s)
    L.set_scalars(0.0, 1.0, 0.0)
    k, d, dp, n, m = L.norm_spectrum(fo2=2.0, which=which)
    m2 = curvature_mean(s, which, lam, v, qG, qH)
    assert m2 > 0
    dx = 2 * np.pi / (N * KIR)
    sel = m > 0
    ref = occupation_from(k[sel], d[sel], dp[sel], m[sel], m2, 2.0, dx)
    assert np.abs(n[sel] - ref).max() < 1e-6 * np.abs(ref).max()
    # the other field's couplings matter: without them the occupation numbers move
    m2_bare = curvature_mean(s, which, lam, v, 0.0, 0.0 if which == 0 else 1e-9)
    bare = occupation_from(k[sel], d[sel], dp[sel], m[sel], m2_bare, 2.0, dx)
    assert np.abs(n[sel] - bare).max() > 1e-3 * np.abs(ref).max()


def test_gauge_invariance_of_both_moduli(oracle_mod):
    gQ, Qc = 0.6, 0.7
    dx = 2 * np.pi / (N * KIR)
    rng = np.random.default_rng(31)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    beta = rng.standard_normal((N, N, N))
    s = full_state(N, 9)
    t = gauge_transform(s[:35], om, beta, gQ, dx) + [x.copy() for x in s[35:]]
    ph = np.exp(1j * Qc * beta)
    for base in (37, 39):
        z = ph * (s[base] + 1j * s[base + 1])
        t[base], t[base + 1] = z.real, z.imag
    A = O.Oracle(O.MODEL_LPHI4_SU2U1, N, KIR, 1.0, 1, full_params(Qc=Qc, gQ=gQ))
    B = O.Oracle(O.MODEL_LPHI4_SU2U1, N, KIR, 1.0, 1, full_params(Qc=Qc, gQ=gQ))
    load(A, s)
    load(B, t)
    for L in (A, B):
        L.set_scalars(0.0, 1.2, 0.3)
    for which in (0, 1):
        ra, rb = A.norm_spectrum(fo2=2.0, which=which), B.norm_spectrum(fo2=2.0, which=which)
        for x, y in zip(ra, rb):
            assert np.allclose(x, y, rtol=1e-10, atol=1e-14 * np.abs(x).max()), which
    # the component arrays themselves did change
    assert np.abs(dump(A)[37] - dump(B)[37]).max() > 1e-2
