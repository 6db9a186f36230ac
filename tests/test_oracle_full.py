"""Pins of the oracle's lphi4SU2U1 model (Sec. 4.5): the SU(2) x U(1) doublet
Phi, a singlet phi_s and a U(1)-charged scalar vphi coupled through
V = lam (|Phi|^2 - v^2)^2 + q_G |Phi|^2 phi_s^2 + 2 q_H |Phi|^2 |vphi|^2
(eq. PotGauge in program units; the manual's example has lam = 1, v = 0).

What fixes the new terms, independently of their own formulas:
  * with q_G = q_H = 0 and the charged scalar uncharged, the doublet and both
    gauge fields evolve bit for bit as the doublet model (itself pinned);
  * with q_G = 0 the singlet is the massless field chi of the lphi4 + chi model
    at phi = 0, bit for bit;
  * with the doublet at zero and charge 1, (vphi, A) is the U(1) model without
    potential, with self-consistent expansion (fields, links, a, a');
  * the kernels are the exact gradients of the lattice energy: each momentum's
    rate equals minus the derivative of N^3 rho (times (f*/omega*)^2 for the
    links) with respect to its field, by central differences at random sites
    -- a dropped, doubled or sign-flipped force term fails it;
  * both Gauss laws, the U(1) one with two charges, conserved to roundoff on
    random states, and held by the initial conditions;
  * gauge covariance with the charged scalar transformed with its own charge
    (and not with the doublet's);
  * energy conservation at second order, and the Hubble constraint at orders
    2 (VV2) and 4 (VV4) under self-consistent expansion.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests.inputs import su2_doublet_state
from tests.test_oracle_su2 import gauge_transform, load as load35

NA = 41


def full_params(**kw):
    base = dict(dt=0.02, integrator=O.VV2, lam=1.0, v=0.0, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
                fluct_amp2=1e-2, phi0=[0.5] * 4, dphi0=[0.1] * 4, expansion=O.EXP_OFF, fstar_over_mp=0.5,
                qG=1.5, qH=0.8, Qc=0.7)
    base.update(kw)
    return O.make_params(**base)


def full_state(N, seed, amp=0.3):
    """The 41 arrays: a doublet-model state, then singlet, charged scalar and momenta."""
    rng = np.random.default_rng(seed + 1000)
    extra = [amp * rng.standard_normal((N, N, N)) for _ in range(6)]
    return su2_doublet_state(N, seed) + extra


def load(L, arrays):
    for a, x in enumerate(arrays):
        L.set_array(a, x)


def dump(L, n=NA):
    return [L.get_array(a).copy() for a in range(n)]


def test_reduces_to_the_doublet_model(oracle_mod):
    N, kIR = 8, 0.8
    kw = dict(integrator=O.LF, v=0.5, fluct_amp2=3e-2)
    full = O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 5, full_params(qG=0.0, qH=0.0, Qc=0.0, **kw))
    dbl = O.Oracle(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 5, full_params(**kw))
    a, b = dump(full), dump(dbl, 35)
    for i in range(35):
        assert np.array_equal(a[i], b[i]), i
    assert np.abs(a[35]).max() > 0 and np.abs(a[37]).max() > 0   # the extra fields fluctuate
    full.step(10)
    dbl.step(10)
    a, b = dump(full), dump(dbl, 35)
    for i in range(35):
        assert np.array_equal(a[i], b[i]), i


def test_singlet_is_the_free_chi_field(oracle_mod):
    N, kIR = 8, 0.8
    rng = np.random.default_rng(2)
    s, ps = 0.3 * rng.standard_normal((N, N, N)), 0.3 * rng.standard_normal((N, N, N))
    full = O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 5, full_params(qG=0.0))
    load(full, full_state(N, 3))
    full.set_array(35, s)
    full.set_array(36, ps)
    chi = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 5, O.make_params(dt=0.02, integrator=O.VV2, q=100.0))
    zero = np.zeros((N, N, N))
    chi.set(0, 0, zero)
    chi.set(0, 1, zero)
    chi.set(1, 0, s)
    chi.set(1, 1, ps)
    full.step(12)
    chi.step(12)
    assert np.array_equal(full.get_array(35), chi.get(1, 0))
    assert np.array_equal(full.get_array(36), chi.get(1, 1))


def test_charged_scalar_is_the_u1_model(oracle_mod):
    N, kIR, g1, fo = 8, 0.8, 0.45, 1.3
    dx = 2 * np.pi / (N * kIR)
    rng = np.random.default_rng(4)
    vp = [0.8 + 0.2 * rng.standard_normal((N, N, N)), 0.6 + 0.2 * rng.standard_normal((N, N, N))]
    pv = [0.3 * rng.standard_normal((N, N, N)) for _ in range(2)]
    A = [0.3 * rng.standard_normal((N, N, N)) for _ in range(3)]
    pA = [0.3 * rng.standard_normal((N, N, N)) for _ in range(3)]
    common = dict(dt=0.03, integrator=O.VV4, fstar_over_omegastar=fo, expansion=O.EXP_SELF, fstar_over_mp=2.0,
                  gQ=g1)
    u1 = O.Oracle(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, O.make_params(lam=0.0, v=0.5, phi0=[0.8, 0.6], **common))
    full = O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 1, full_params(qH=2.0, Qc=1.0, v=0.0, fluct_amp2=0.0,
                                                                     **common))
    for f in range(2):
        u1.set(f, 0, vp[f])
        u1.set(f, 1, pv[f])
    for i in range(3):
        u1.set(2 + i, 0, A[i])
        u1.set(2 + i, 1, pA[i])
    zero, one = np.zeros((N, N, N)), np.ones((N, N, N))
    arrays = [zero] * 8 + A + pA
    for i in range(3):
        arrays += [one, zero, zero, zero]
    arrays += [zero] * 9 + [zero, zero] + vp + pv
    load(full, arrays)
    b0 = np.sqrt(2.0 ** 2 * u1.energies()["rho"] / 3.0)   # a' from the Hubble law (f*/m_p = 2)
    for L in (u1, full):
        L.set_scalars(0.0, 1.0, b0)
    e1, e2 = u1.energies(), full.energies()
    assert abs(e1["rho"] - e2["rho"]) < 1e-13 * e1["rho"]
    assert abs(e1["EG"][0] - e2["EG"][2]) < 1e-13 * e1["EG"][0]
    u1.step(10)
    full.step(10)
    assert abs(u1.scalars()[1] - full.scalars()[1]) < 1e-13 and u1.scalars()[1] > 1.01
    assert abs(u1.scalars()[2] - full.scalars()[2]) < 1e-13
    for f in range(2):
        assert np.abs(full.get_array(37 + f) - u1.get(f, 0)).max() < 1e-11
        assert np.abs(full.get_array(39 + f) - u1.get(f, 1)).max() < 1e-11
    for i in range(3):
        assert np.abs(full.get_array(8 + i) - u1.get(2 + i, 0)).max() < 1e-11
        assert np.abs(full.get_array(11 + i) - u1.get(2 + i, 1)).max() < 1e-11
    for a in range(8):
        assert np.abs(full.get_array(a)).max() == 0.0


# momentum array -> (field array, factor on the energy gradient)
FORCES = [(4, 0, 1.0), (6, 2, 1.0), (11, 8, None), (13, 10, None), (36, 35, 1.0), (39, 37, 1.0), (40, 38, 1.0)]


def test_kernels_are_gradients_of_the_lattice_energy(oracle_mod):
    """At a = 1, alpha = 1 the lattice Hamiltonian is N^3 rho for the scalars and
    (f*/omega*)^2 N^3 rho for the link fields (their kinetic term carries the
    inverse), so pi' = -dH/dq: checked by central differences of rho at
    random sites, for the doublet, the singlet, the charged scalar and the U(1) links."""
    N, kIR, eps = 6, 0.8, 1e-5
    p = full_params(v=0.3, fluct_amp2=0.0)
    fo2 = 1.3 ** 2
    L = O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 1, p)
    st = full_state(N, 9)
    load(L, st)
    rng = np.random.default_rng(5)
    V = N ** 3
    for mom, field, fac in FORCES:
        K = L.kernel(mom)
        scale = np.abs(K).max()
        assert scale > 1e-3
        for _ in range(4):
            z, y, x = rng.integers(0, N, 3)
            grad = []
            for sgn in (+1, -1):
                arr = st[field].copy()
                arr[z, y, x] += sgn * eps
                L.set_array(field, arr)
                grad.append(L.energies()["rho"] * V)
            L.set_array(field, st[field])
            dH = (grad[0] - grad[1]) / (2 * eps)
            f = fo2 if fac is None else fac
            assert abs(K[z, y, x] + f * dH) < 1e-6 * scale, (mom, K[z, y, x], -f * dH)


@pytest.mark.parametrize("integ,expansion", [(O.VV2, O.EXP_OFF), (O.VV4, O.EXP_SELF)])
def test_gauss_laws_conserved_with_two_charges(oracle_mod, integ, expansion):
    N = 8
    L = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 7, full_params(integrator=integ, expansion=expansion))
    load(L, full_state(N, 11))
    r0 = [L.gauss_residual(g).copy() for g in range(4)]
    assert min(np.abs(r).max() for r in r0) > 0.1
    L.step(6)
    for g in range(4):
        assert np.abs(L.gauss_residual(g) - r0[g]).max() < 2e-13, g


def test_initial_conditions_hold_the_gauss_laws(oracle_mod):
    L = O.Oracle(O.MODEL_LPHI4_SU2U1, 8, 0.8, 1.0, 3, full_params(fluct_amp2=3e-2))
    rel, lhs, rhs, mx = L.gauss()
    assert rhs > 1e-4 and rel < 1e-13 and mx < 1e-13
    # the charged scalar's density is part of the U(1) law: without it the law fails
    ref = O.Oracle(O.MODEL_LPHI4_SU2U1, 8, 0.8, 1.0, 3, full_params(fluct_amp2=3e-2, Qc=0.0))
    assert np.abs(L.get_array(11) - ref.get_array(11)).max() > 1e-6
    assert np.array_equal(L.get_array(26), ref.get_array(26))   # the SU(2) laws do not see it
    L.step(30)
    assert L.gauss()[0] < 1e-12


def test_gauge_covariance_with_two_charges(oracle_mod):
    N, gQ, Qc = 8, 0.6, 0.7
    dx = 2 * np.pi / (N * 0.8)
    rng = np.random.default_rng(21)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    beta = rng.standard_normal((N, N, N))

    def transform(arrays, q):
        out = gauge_transform(arrays[:35], om, beta, gQ, dx) + [x.copy() for x in arrays[35:]]
        ph = np.exp(1j * q * beta)
        for base in (37, 39):
            z = ph * (arrays[base] + 1j * arrays[base + 1])
            out[base], out[base + 1] = z.real, z.imag
        return out

    s = full_state(N, 8)
    L1 = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 1, full_params(expansion=O.EXP_SELF, Qc=Qc))
    L2 = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 1, full_params(expansion=O.EXP_SELF, Qc=Qc))
    load(L1, s)
    load(L2, transform(s, Qc))
    e1, e2 = L1.energies(), L2.energies()
    for k in ("EK", "EG", "EV"):
        for i in range(3):
            assert abs(e1[k][i] - e2[k][i]) < 1e-13 * abs(e1[k][i]), (k, i)
    L1.step(8)
    L2.step(8)
    assert abs(L1.scalars()[1] - L2.scalars()[1]) < 1e-14
    ref, got = transform(dump(L1), Qc), dump(L2)
    for a in range(NA):
        assert np.abs(ref[a] - got[a]).max() < 1e-11, a
    # the charged scalar rotated with the doublet's charge instead: not a symmetry
    L3 = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 1, full_params(Qc=Qc))
    load(L3, transform(s, 1.0))
    assert abs(L3.energies()["EG"][2] - e1["EG"][2]) > 1e-3 * e1["EG"][2]


def test_energy_conservation_second_order(oracle_mod):
    N, T, errs = 8, 0.4, []
    for dt in (0.04, 0.02, 0.01):
        L = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 1, full_params())
        load(L, full_state(N, 3))
        r0 = L.energies()["rho"]
        L.step(int(round(T / dt)), h=dt)
        errs.append(abs(L.energies()["rho"] - r0))
    for e0, e1 in zip(errs, errs[1:]):
        assert abs(math.log(e0 / e1, 2) - 2.0) < 0.05, errs


@pytest.mark.parametrize("integ,order", [(O.VV2, 2), (O.VV4, 4)])
def test_hubble_constraint_order(oracle_mod, integ, order):
    N, T, v = 8, 0.8, []
    st = full_state(N, 17)
    for dt in (0.04, 0.02):
        L = O.Oracle(O.MODEL_LPHI4_SU2U1, N, 0.8, 1.0, 1, full_params(dt=dt, integrator=integ,
                                                                      expansion=O.EXP_SELF))
        load(L, st)
        rho = L.energies()["rho"]
        L.set_scalars(0.0, 1.0, np.sqrt(0.5 ** 2 * rho / 3.0))
        L.step(int(round(T / dt)))
        e = L.energies()
        assert e["a"] > 1.3 and e["EG"][1] > 0 and e["EG"][2] > 0
        v.append(abs(e["hubble_viol"]))
    slope = math.log(v[0] / v[1], 2)
    assert abs(slope - order) < 0.1, (v, slope)


def test_state_access(oracle_mod):
    L = O.Oracle(O.MODEL_LPHI4_SU2U1, 8, 0.8, 1.0, 1, full_params())
    assert L.nfields() == 10
    for f, a in ((7, 35), (8, 37), (9, 38)):
        assert np.array_equal(L.get(f, 0), L.get_array(a))
        assert np.array_equal(L.get(f, 1), L.get_array(a + (1 if f == 7 else 2)))
    with pytest.raises(IndexError):
        L.get_array(41)
