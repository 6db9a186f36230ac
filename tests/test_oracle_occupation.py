"""Pins of the oracle's lattice occupation number (eq. OccuppationNum):

* at the initial conditions every drawn mode's contribution follows from its
  two Rayleigh draws alone, n = C [w |F|^2 + |G + H F|^2/w] with
  F = (z1 + z2)/sqrt2 and G + H F = a^{alpha-1} i omega (z1 - z2)/sqrt2 (the IC
  map, pinned separately); the bins are rebuilt here from the draws, so the
  FFT normalisation, the shell binning, the conversion pi -> phi' and the
  constant a^2 L^3 (f*/omega*)^2/(2 N^6) are all checked;
* the vacuum gives n = 1/2 on average;
* a massless field in a radiation-dominated background (fixed power law,
  w = 1/3) is conformal, so n_k is conserved while a grows threefold, in
  conformal (alpha = 1) and cosmic (alpha = 0) time; a missing power of a or a
  missing a'/a term changes it by order one.
"""
import numpy as np
import pytest

import oracle as O


def bins_of(N, dk):
    idx = np.arange(N ** 3)
    x, y, z = idx % N, (idx // N) % N, idx // (N * N)
    s = lambda u: np.where(u <= N // 2, u, u - N)
    nn = np.sqrt(s(x) ** 2 + s(y) ** 2 + s(z) ** 2)
    nb = int(np.floor(np.sqrt(3.0) * (N // 2) / dk)) + 1
    b = np.minimum(np.floor(nn / dk).astype(int), nb - 1)
    partner = (-x) % N + N * ((-y) % N + N * ((-z) % N))
    return idx, nn, b, nb, partner


@pytest.mark.parametrize("field,m2", [(0, 3.0), (1, 100.0)])
def test_occupation_from_ic_draws(oracle_mod, field, m2):
    N, kIR, seed, dk = 12, 0.5, 3, 1.0
    kw = dict(dt=0.01, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-8,
              expansion=O.EXP_SELF, fstar_over_mp=2.0)
    p = O.make_params(**kw)
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p)
    eta, a, bsc = o.scalars()
    assert a == 1.0 and bsc > 0.5            # H = a'/a enters
    k, n, m = o.occupation(field, dk)
    idx, nn, b, nb, partner = bins_of(N, dk)
    canon = np.minimum(idx, partner)         # the drawn member of each pair
    dr = O.ic_draws(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p, canon)[:, field]
    z1 = dr[:, 0] * np.exp(1j * dr[:, 1])
    z2 = dr[:, 2] * np.exp(1j * dr[:, 3])
    F = (z1 + z2) / np.sqrt(2.0)
    GH = 1j * dr[:, 4] * (z1 - z2) / np.sqrt(2.0)
    sc = partner == idx                      # self-conjugate sites keep the real part
    F = np.where(sc, F.real, F)
    GH = np.where(sc, GH.real, GH)
    L = N * 2 * np.pi / (N * kIR)
    C = a ** 2 * L ** 3 / (2.0 * N ** 6) / kw["fluct_amp2"]
    for bb in range(nb):
        sel = (b == bb) & (idx != 0)
        if not sel.any():
            assert m[bb] == 0
            continue
        assert m[bb] == sel.sum()
        kb = kIR * nn[sel].mean()
        assert abs(k[bb] - kb) < 1e-12 * kb
        w = np.sqrt(kb ** 2 + a ** 2 * m2)   # the homogeneous mass: <V''> differs by O(1e-8)
        want = C * np.mean(w * np.abs(F[sel]) ** 2 + np.abs(GH[sel]) ** 2 / w)
        assert abs(n[bb] - want) < 1e-6 * want, (bb, n[bb], want)
    # the vacuum: one half per mode on average
    assert abs(np.sum(n * m) / np.sum(m) - 0.5) < 0.05


@pytest.mark.parametrize("alpha", [1.0, 0.0])
def test_occupation_conserved_in_radiation_era(oracle_mod, alpha):
    p = O.make_params(dt=0.01, integrator=O.VV4, phi0=[0.0], fluct_amp2=1e-8, expansion=O.EXP_FIXED,
                      omega_eos=1.0 / 3.0, H0=1.0, fstar_over_mp=0.5)
    o = O.Oracle(O.MODEL_LPHI4, 16, 0.25, alpha, 5, p)
    k0, n0, m0 = o.occupation(0)
    o.step(200)
    assert o.scalars()[1] > 2.2
    k1, n1, m1 = o.occupation(0)
    assert np.array_equal(m0, m1)
    rel = np.abs(n1[1:5] / n0[1:5] - 1.0)
    assert rel.max() < 0.05, rel


def test_occupation_arguments(oracle_mod):
    p = O.make_params(dt=0.01, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4)
    o = O.Oracle(O.MODEL_LPHI4_CHI, 8, 1.0, 1.0, 2, p)
    k, n1, m = o.occupation(1, 1.0, fo2=1.0)
    k, n2, m = o.occupation(1, 1.0, fo2=3.0)
    assert np.allclose(n2, 3.0 * n1, rtol=1e-14, atol=0)
    with pytest.raises(ValueError):
        o.occupation(2)
    with pytest.raises(ValueError):
        o.occupation(0, fo2=-1.0)
    u = O.Oracle(O.MODEL_U1_HIGGS, 8, 1.0, 1.0, 1, O.make_params(dt=0.01, lam=1.0, v=1.0, gQ=0.5,
                                                                 phi0=[1.0, 1.0], fluct_amp2=1e-2))
    with pytest.raises(ValueError):
        u.occupation(0)
