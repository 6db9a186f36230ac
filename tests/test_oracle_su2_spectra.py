"""Pins of the oracle's electric and magnetic spectra of the doublet model's
gauge fields (clo_em_spectrum, which = 0..3; the spectra_norm_[U1/SU2] outputs of
Sec. 4.5 with eq. discretePS; G from the plaquette as in the SU(N) toolkit).

  * SU(2) electric: the sum over the 9 components (colour a, direction i) of the
    (separately pinned) singlet spectrum of a^{alpha-1} pi_B,i^a, at a != 1.
  * SU(2) magnetic: pure-gauge links (U_i(n) = Omega(n) Omega^dag(n+i)) give zero;
    small random fields give the spectrum of the forward-difference curl of B^a
    (the toolkit's small-angle limit), to the non-Abelian correction.
  * A global SU(2) rotation of links and momenta leaves both unchanged.
  * The doublet model's U(1) spectra are the U(1) model's for the same links.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import smooth_field, su2_doublet_state
from tests.test_oracle_su2 import mat, quat

N, KIR, ALPHA = 12, 0.7, 0.5
DX = 2 * np.pi / (N * KIR)
KW = dict(lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3, fluct_amp2=0.0)


def doublet(arrays, a=1.0):
    L = O.Oracle(O.MODEL_SU2U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(**KW))
    for i, x in enumerate(arrays):
        L.set_array(i, x)
    L.set_scalars(0.0, a, 0.0)
    return L


def summed_spectrum(fields):
    """sum over the given real fields of the singlet spectrum (k, delta, mult)."""
    S = O.Oracle(O.MODEL_LPHI4, N, KIR, ALPHA, 1, O.make_params(fluct_amp2=0.0))
    tot = None
    for f in fields:
        S.set(0, 0, f)
        k, d, m = S.spectrum(0, 0)
        tot = d if tot is None else tot + d
    return k, tot, m


def test_su2_electric_is_the_sum_of_component_spectra(oracle_mod):
    st = su2_doublet_state(N, 3)
    a = 1.25
    L = doublet(st, a)
    k, d, m = L.em_spectrum(2)
    ae = a ** (ALPHA - 1.0)
    k0, d0, m0 = summed_spectrum([ae * st[26 + c] for c in range(9)])
    assert np.array_equal(m, m0) and np.abs(k - k0).max() < 1e-13
    assert np.abs(d - d0).max() <= 1e-12 * np.abs(d0).max()


def test_su2_magnetic_of_pure_gauge_links_is_zero(oracle_mod):
    rng = np.random.default_rng(5)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    Om = mat(om)
    st = su2_doublet_state(N, 4)
    for i, ax in enumerate((2, 1, 0)):
        Op = np.roll(Om, -1, axis=ax)
        st[14 + 4 * i: 18 + 4 * i] = quat(Om @ np.conj(np.swapaxes(Op, -1, -2)))
    _, d, _ = doublet(st).em_spectrum(3)
    _, dref, _ = doublet(su2_doublet_state(N, 4)).em_spectrum(3)
    assert np.abs(d).max() < 1e-24 * np.abs(dref).max()


def test_su2_magnetic_small_field_limit_is_the_lattice_curl(oracle_mod):
    eps, gB = 1e-4, KW["gQB"]
    B = [[eps * smooth_field(N, 40 + 3 * i + a, amp=1.0) for a in range(3)] for i in range(3)]  # B[i][a]
    st = su2_doublet_state(N, 6)
    for i in range(3):
        u = np.empty((4, N, N, N))
        th = np.stack([gB * DX * B[i][a] for a in range(3)], 0)
        for idx in np.ndindex(N, N, N):
            u[(slice(None),) + idx] = O.su2_exp(th[(slice(None),) + idx])
        st[14 + 4 * i: 18 + 4 * i] = list(u)
    _, d, _ = doublet(st).em_spectrum(3)

    def fwd(f, d_):   # forward difference along direction d_ (arrays are [z][y][x])
        return (np.roll(f, -1, axis=2 - d_) - f) / DX
    curl = []
    for i in range(3):
        j, l = (i + 1) % 3, (i + 2) % 3
        for a in range(3):
            curl.append(fwd(B[l][a], j) - fwd(B[j][a], l))
    _, d0, _ = summed_spectrum(curl)
    assert np.abs(d - d0).max() <= 1e-5 * np.abs(d0).max()   # measured 4e-7: O(eps) corrections


def test_global_rotation_leaves_both_unchanged(oracle_mod):
    st = su2_doublet_state(N, 7)
    q = np.array([0.3, -0.5, 0.7, 0.4])
    q /= np.linalg.norm(q)
    Om = mat([np.full((N, N, N), x) for x in q])
    Od = np.conj(np.swapaxes(Om, -1, -2))
    rot = [x.copy() for x in st]
    sig = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]
    for i in range(3):
        rot[14 + 4 * i: 18 + 4 * i] = quat(Om @ mat(st[14 + 4 * i: 18 + 4 * i]) @ Od)
        P = sum(st[26 + 3 * i + a][..., None, None] * sig[a] / 2 for a in range(3))
        Pn = Om @ P @ Od
        for a in range(3):
            rot[26 + 3 * i + a] = np.einsum("...ij,ji->...", Pn, sig[a]).real
    for which in (2, 3):
        _, d1, _ = doublet(st).em_spectrum(which)
        _, d2, _ = doublet(rot).em_spectrum(which)
        assert np.abs(d1 - d2).max() <= 1e-12 * np.abs(d1).max()


def test_doublet_u1_spectra_are_the_u1_models(oracle_mod):
    st = su2_doublet_state(N, 9)
    D = doublet(st, 1.1)
    U = O.Oracle(O.MODEL_U1_HIGGS, N, KIR, ALPHA, 1, O.make_params(lam=1.0, v=0.5, gQ=KW["gQ"], fluct_amp2=0.0))
    for i in range(3):
        U.set(2 + i, 0, st[8 + i])
        U.set(2 + i, 1, st[11 + i])
    U.set_scalars(0.0, 1.1, 0.0)
    for which in (0, 1):
        _, d1, _ = D.em_spectrum(which)
        _, d2, _ = U.em_spectrum(which)
        assert np.abs(d1 - d2).max() <= 1e-13 * np.abs(d2).max()
    with pytest.raises(ValueError):
        U.em_spectrum(2)
