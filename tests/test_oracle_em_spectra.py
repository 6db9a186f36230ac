"""Pins of the oracle's electric and magnetic field spectra of the U(1) model
(clo_em_spectrum; E_i = a^{alpha-1} pi_A,i, B_i = (1/2) eps_ijk sin(theta_jk)/(gQ dx^2)):

* each equals the sum over components of the scalar spectrum (clo_spectrum,
  pinned by Parseval and the naive DFT elsewhere) of the component fields,
  built here from the definitions: E from the link momenta and a, B as the
  forward-difference curl of A, which the compact form reaches for small
  angles (sin theta = theta + O(theta^3));
* links that are a pure gauge (A_i = grad_i chi) have no magnetic field;
* a lattice gauge transformation leaves both spectra unchanged.
"""
import numpy as np
import pytest

import oracle as O


def u1(N=8, gQ=0.5, amp=0.05, seed=5, expansion=O.EXP_OFF):
    p = O.make_params(dt=0.05, integrator=O.LF, lam=1.0, v=1.0, gQ=gQ, fstar_over_omegastar=0.8,
                      phi0=[1.0, 1.0], fluct_amp2=amp, expansion=expansion, fstar_over_mp=2.0)
    return O.Oracle(O.MODEL_U1_HIGGS, N, 1.0, 1.0, seed, p)


def scalar_spectrum_sum(N, comps, dk):
    """Sum over components of clo_spectrum of each component loaded as a scalar field."""
    s = O.Oracle(O.MODEL_LPHI4, N, 1.0, 1.0, 1, O.make_params(dt=0.01, phi0=[0.0], fluct_amp2=0.0))
    tot = None
    for f in comps:
        s.set(0, 0, f)
        k, d, m = s.spectrum(0, 0, dk)
        tot = d if tot is None else tot + d
    return k, tot, m


def fwd(u, ax):   # forward difference along array axis ax ([z][y][x])
    return np.roll(u, -1, axis=ax) - u


@pytest.mark.parametrize("dk", [1.0, 1.5])
def test_electric_spectrum_is_the_momenta_spectrum(oracle_mod, dk):
    L = u1(expansion=O.EXP_SELF)
    L.step(20)
    eta, a, b = L.scalars()
    assert a > 1.01
    E = [a ** (1.0 - 1.0) * L.get(2 + i, 1) for i in range(3)]   # alpha = 1: a^{alpha-1} = 1
    k, d, m = L.em_spectrum(0, dk)
    ks, ds, ms = scalar_spectrum_sum(8, E, dk)
    assert np.array_equal(m, ms) and np.allclose(k, ks, rtol=1e-14, atol=0)
    assert np.abs(d - ds).max() < 1e-12 * np.abs(ds).max()


def test_electric_spectrum_scale_factor_power(oracle_mod):
    """alpha = 0: E_i = pi_A,i / a."""
    p = O.make_params(dt=0.05, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=0.8,
                      phi0=[1.0, 1.0], fluct_amp2=0.05, expansion=O.EXP_SELF, fstar_over_mp=2.0)
    L = O.Oracle(O.MODEL_U1_HIGGS, 8, 1.0, 0.0, 5, p)
    L.step(20)
    a = L.scalars()[1]
    assert abs(a - 1.0) > 0.01   # (this background decelerates and contracts)
    k, d, m = L.em_spectrum(0)
    ks, ds, ms = scalar_spectrum_sum(8, [L.get(2 + i, 1) / a for i in range(3)], 1.0)
    assert np.abs(d - ds).max() < 1e-12 * np.abs(ds).max()


def test_magnetic_spectrum_small_angle_curl(oracle_mod):
    N, gQ = 8, 0.5
    dx = 2 * np.pi / N
    L = u1(N=N, gQ=gQ)
    rng = np.random.default_rng(3)
    A = [1e-5 * rng.standard_normal((N, N, N)) for _ in range(3)]
    for i in range(3):
        L.set(2 + i, 0, A[i])
    ax = {0: 2, 1: 1, 2: 0}   # direction i -> array axis
    F = lambda i, j: (fwd(A[j], ax[i]) - fwd(A[i], ax[j])) / dx
    B = [F(1, 2), -F(0, 2), F(0, 1)]   # B_x = F_yz, B_y = -F_xz, B_z = F_xy
    k, d, m = L.em_spectrum(1)
    ks, ds, ms = scalar_spectrum_sum(N, B, 1.0)
    assert np.abs(d - ds).max() < 1e-8 * np.abs(ds).max()


def test_pure_gauge_has_no_magnetic_field(oracle_mod):
    N = 8
    dx = 2 * np.pi / N
    L = u1(N=N)
    L.step(5)
    k, d0, m = L.em_spectrum(1)
    assert d0.max() > 0
    chi = np.random.default_rng(4).standard_normal((N, N, N))
    for i, ax in enumerate((2, 1, 0)):
        L.set(2 + i, 0, fwd(chi, ax) / dx)
    k, d, m = L.em_spectrum(1)
    assert d.max() < 1e-24 * d0.max()


def test_gauge_invariance(oracle_mod):
    N, gQ = 8, 0.5
    dx = 2 * np.pi / N
    L = u1(N=N, gQ=gQ)
    L.step(5)
    before = [L.em_spectrum(w)[1] for w in (0, 1)]
    al = np.random.default_rng(9).standard_normal((N, N, N))
    th = gQ * al
    c, s = np.cos(th), np.sin(th)
    for what in (0, 1):
        x, y = L.get(0, what), L.get(1, what)
        L.set(0, what, c * x - s * y)
        L.set(1, what, s * x + c * y)
    for i, ax in enumerate((2, 1, 0)):
        L.set(2 + i, 0, L.get(2 + i, 0) + fwd(al, ax) / dx)
    after = [L.em_spectrum(w)[1] for w in (0, 1)]
    for b, a in zip(before, after):
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_scalar_models_refused(oracle_mod):
    o = O.Oracle(O.MODEL_LPHI4, 8, 1.0, 1.0, 1, O.make_params(dt=0.01, phi0=[1.0], fluct_amp2=1e-4))
    with pytest.raises(ValueError):
        o.em_spectrum(0)
