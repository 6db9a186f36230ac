"""Pins of the oracle's modulus ("norm") spectra of the charged fields
(clo_norm_spectrum: Delta of r = |phi|, of r', and the occupation number of the
canonical modulus sqrt2 r;
gauge models' spectrum outputs, Sec. 4.5, with eqs. discretePS and
OccuppationNum).

  * Reduction to the (separately pinned) singlet spectra and occupation number:
    a U(1) state phi_0 = s (s > 0), phi_1 = 0 has r = s/sqrt2, r' = s'/sqrt2 and
    the canonical modulus rho = sqrt2 r = s; with V = lam (r^2 - v^2)^2, lam = 1,
    v = 0 its potential is rho^4/4, that of the lphi4 model (the U(1) model with
    phi_1 = 0 is then the lphi4 model for phi_0).  So Delta_r and Delta_r' are
    half the lphi4 oracle's for phi = s and n equals it -- at a != 1 and a' != 0
    (the powers of a and the a'/a term), alpha = 0.5.
  * The same through a random SU(2) rotation of the doublet (|Phi| = s/sqrt2).
  * The occupation number of the modulus is an adiabatic invariant: a small
    radial ripple on the vacuum keeps its n while a doubles in a radiation era
    (this fixes the a^2 in front of the mass at a != 1 and the canonical
    normalisation).
  * Gauge invariance: a random U(1) transformation of a generic U(1) state, and
    a random SU(2) x U(1) transformation of a doublet state, leave every output
    unchanged (the component spectra change).
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import smooth_field, su2_doublet_state
from tests.test_oracle_su2 import gauge_transform, mat

N, KIR, ALPHA = 12, 0.7, 0.5


def scalar_ref(s, p, a, b):
    L = O.Oracle(O.MODEL_LPHI4, N, KIR, ALPHA, 1, O.make_params(fluct_amp2=0.0))
    L.set(0, 0, s)
    L.set(0, 1, p)
    L.set_scalars(0.0, a, b)
    k, d, m = L.spectrum(0, 0)
    _, dp, _ = L.spectrum(0, 1)
    _, n, _ = L.occupation(0, fo2=2.5)
    return k, d, dp, n, m


def test_u1_modulus_reduces_to_the_singlet(oracle_mod):
    s = smooth_field(N, 3, amp=0.4, offset=1.0)
    p = smooth_field(N, 4, amp=0.3)
    assert s.min() > 0
    a, b = 1.3, 0.4
    L = O.Oracle(O.MODEL_U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(lam=1.0, v=0.0, gQ=0.5, fluct_amp2=0.0))
    zero = np.zeros_like(s)
    L.set(0, 0, s); L.set(1, 0, zero)
    L.set(0, 1, p); L.set(1, 1, zero)
    L.set_scalars(0.0, a, b)
    k, d, dp, n, m = L.norm_spectrum(fo2=2.5)
    k0, d0, dp0, n0, m0 = scalar_ref(s, p, a, b)
    assert np.array_equal(m, m0) and np.abs(k - k0).max() < 1e-13
    assert np.abs(d - 0.5 * d0).max() <= 1e-12 * np.abs(d0).max()
    # r' = a^{alpha-3} pi/sqrt2: half the singlet's momentum spectrum times a^{2(alpha-3)}
    assert np.abs(dp - 0.5 * a ** (2 * (ALPHA - 3)) * dp0).max() <= 1e-12 * np.abs(dp).max()
    assert np.abs(n - n0).max() <= 1e-12 * np.abs(n0).max()


def test_doublet_modulus_through_an_su2_rotation(oracle_mod):
    s = smooth_field(N, 5, amp=0.4, offset=1.0)
    p = smooth_field(N, 6, amp=0.3)
    a, b = 0.8, -0.2
    rng = np.random.default_rng(2)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    Om = mat(om)
    # psi = Omega (s, 0), pi_psi = Omega (p, 0): sqrt2 |Phi| = s, sqrt2 |Phi|' = a^{alpha-3} p
    f = np.einsum("...ij,...j->...i", Om, np.stack([s + 0j, 0 * s + 0j], -1))
    g = np.einsum("...ij,...j->...i", Om, np.stack([p + 0j, 0 * p + 0j], -1))
    L = O.Oracle(O.MODEL_SU2U1_HIGGS, N, KIR, ALPHA, 1,
                 O.make_params(lam=1.0, v=0.0, gQ=0.5, gQB=0.7, fluct_amp2=0.0))
    for c, x in enumerate((f[..., 0].real, f[..., 0].imag, f[..., 1].real, f[..., 1].imag)):
        L.set_array(c, x)
    for c, x in enumerate((g[..., 0].real, g[..., 0].imag, g[..., 1].real, g[..., 1].imag)):
        L.set_array(4 + c, x)
    L.set_scalars(0.0, a, b)
    k, d, dp, n, m = L.norm_spectrum(fo2=2.5)
    k0, d0, dp0, n0, m0 = scalar_ref(s, p, a, b)
    assert np.array_equal(m, m0)
    assert np.abs(d - 0.5 * d0).max() <= 1e-12 * np.abs(d0).max()
    assert np.abs(dp - 0.5 * a ** (2 * (ALPHA - 3)) * dp0).max() <= 1e-12 * np.abs(dp).max()
    assert np.abs(n - n0).max() <= 1e-12 * np.abs(n0).max()


def test_u1_gauge_invariance(oracle_mod):
    kw = dict(lam=1.0, v=0.5, gQ=0.5, fluct_amp2=0.0)
    A = O.Oracle(O.MODEL_U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(**kw))
    B = O.Oracle(O.MODEL_U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(**kw))
    f = [smooth_field(N, 10 + i, amp=0.5, offset=0.7) for i in range(4)]
    th = np.random.default_rng(3).standard_normal((N, N, N))
    c, s_ = np.cos(th), np.sin(th)
    for L, rot in ((A, False), (B, True)):
        for w in (0, 1):
            x, y = f[2 * w], f[2 * w + 1]
            if rot:
                x, y = c * x - s_ * y, s_ * x + c * y
            L.set(0, w, x)
            L.set(1, w, y)
        L.set_scalars(0.0, 1.2, 0.3)
    ra, rb = A.norm_spectrum(fo2=2.0), B.norm_spectrum(fo2=2.0)
    for x, y in zip(ra, rb):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(x).max(), 1e-300)
    # the components' own spectrum is not invariant
    assert np.abs(A.spectrum(0, 0)[1] - B.spectrum(0, 0)[1]).max() > 1e-3 * np.abs(A.spectrum(0, 0)[1]).max()


def test_doublet_gauge_invariance(oracle_mod):
    kw = dict(lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3, fluct_amp2=0.0)
    dx = 2 * np.pi / (N * KIR)
    st = su2_doublet_state(N, 12)
    rng = np.random.default_rng(8)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    beta = rng.standard_normal((N, N, N))
    A = O.Oracle(O.MODEL_SU2U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(**kw))
    B = O.Oracle(O.MODEL_SU2U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(**kw))
    for i, x in enumerate(st):
        A.set_array(i, x)
    for i, x in enumerate(gauge_transform(st, om, beta, kw["gQ"], dx)):
        B.set_array(i, x)
    ra, rb = A.norm_spectrum(fo2=2.0), B.norm_spectrum(fo2=2.0)
    for x, y in zip(ra, rb):
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(x).max(), 1e-300)


def test_scalar_models_refused(oracle_mod):
    L = O.Oracle(O.MODEL_LPHI4, 8, 1.0, 1.0, 1, O.make_params(fluct_amp2=1e-2))
    with pytest.raises(ValueError):
        L.norm_spectrum(fo2=1.0)


def plane_waves(N, modes, amp, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    f = np.zeros((N, N, N))
    for m in modes:
        f += amp * rng.uniform(0.5, 1.0) * np.cos(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / N
                                                   + rng.uniform(0, 2 * np.pi))
    return f


@pytest.mark.parametrize("alpha", [1.0, 0.0])
def test_modulus_occupation_is_an_adiabatic_invariant(oracle_mod, alpha):
    """A small radial ripple on the vacuum |phi| = v of the U(1) model (phi_1 = 0,
    so the current and the gauge fields stay zero) is a free field of mass^2
    d^2V/drho^2 = 4 lam v^2 for the canonical modulus rho = sqrt2 |phi|.  In a
    radiation-dominated background (a linear in conformal time, so a''/a = 0)
    each mode a rho_k is an oscillator of frequency w^2 = k^2 + a^2 m^2 that
    changes slowly (w'/w^2 < 0.01 here), so its occupation number is conserved
    while a doubles.  Bins of width 0.04 hold one |n| each, so the bin's k is the
    mode's (the manual's shell-mean k is exact there); the modes' lattice and
    continuum k differ by < 0.6 % in w.  A wrong power of a in front of the mass
    (a^0, a^4) or the uncanonical modulus (mass V''(r), no factor 2) breaks the
    1 % bound; the a'/a term (H/w < 1 %) is left to the reduction pin."""
    N, kIR, H0, dt, lam, v = 12, 0.5, 0.025, 0.05, 2.0, 1.0
    p = O.make_params(dt=dt, integrator=O.VV4, lam=lam, v=v, gQ=0.5, fluct_amp2=0.0,
                      phi0=[np.sqrt(2) * v, 0.0], expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0, H0=H0,
                      fstar_over_mp=0.5)
    L = O.Oracle(O.MODEL_U1_HIGGS, N, kIR, alpha, 1, p)
    L.set(0, 0, np.sqrt(2) * v + plane_waves(N, [(1, 0, 0), (0, 1, 1), (1, -1, 1), (0, 2, 0)], 1e-4, 7))
    k0, _, _, n0, m0 = L.norm_spectrum(dk_bin=0.04, fo2=1.0)
    hit = np.nonzero(n0 > 1e-20)[0]
    assert np.allclose(k0[hit] / kIR, np.sqrt([1.0, 2.0, 3.0, 4.0]), rtol=1e-12)
    # a = 1 + H0 eta (alpha = 1), a = sqrt(1 + 2 H0 t) (alpha = 0): a = 2 at the end
    L.step(800 if alpha == 1.0 else 1200)
    assert abs(L.scalars()[1] - 2.0) < 1e-9
    k1, _, _, n1, m1 = L.norm_spectrum(dk_bin=0.04, fo2=1.0)
    assert np.array_equal(m0, m1)
    rel = np.abs(n1[hit] / n0[hit] - 1.0)
    assert rel.max() < 0.01, rel


def test_doublet_modulus_occupation_is_an_adiabatic_invariant(oracle_mod):
    """The same radial ripple on the doublet's vacuum (real upper component, links
    at the identity): the U(1) and SU(2) currents Im(psi^dag sigma W psi) vanish
    for a real upper component, so the gauge fields stay zero and n of the
    canonical modulus is conserved while a doubles (conformal time)."""
    N, kIR, H0, dt, lam, v = 12, 0.5, 0.025, 0.05, 2.0, 1.0
    p = O.make_params(dt=dt, integrator=O.VV4, lam=lam, v=v, gQ=0.5, gQB=0.7, fluct_amp2=0.0,
                      phi0=[np.sqrt(2) * v, 0.0, 0.0, 0.0], expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0,
                      H0=H0, fstar_over_mp=0.5)
    L = O.Oracle(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 1, p)
    L.set_array(0, np.sqrt(2) * v + plane_waves(N, [(1, 0, 0), (0, 1, 1), (1, -1, 1), (0, 2, 0)], 1e-4, 7))
    _, _, _, n0, m0 = L.norm_spectrum(dk_bin=0.04, fo2=1.0)
    hit = np.nonzero(n0 > 1e-20)[0]
    assert len(hit) == 4
    L.step(800)
    assert abs(L.scalars()[1] - 2.0) < 1e-9
    _, _, _, n1, m1 = L.norm_spectrum(dk_bin=0.04, fo2=1.0)
    assert np.array_equal(m0, m1)
    rel = np.abs(n1[hit] / n0[hit] - 1.0)
    assert rel.max() < 0.01, rel
