"""GPU parity of the U(1) Abelian-Higgs path (C ABI, sm_103a kernels) against
the FP64 CPU oracle, on the same seeds / the same seeded input states.

Tolerances (normwise: max |gpu - oracle| / max |oracle| per array):
  FP64 storage: 1e-10 pointwise, 1e-10 on volume averages, Gauss-law
                residual <= 1.05 x the oracle's (both at roundoff);
  FP32 storage: 1e-4 pointwise after 100 steps, 1e-5 on volume averages;
                Gauss-law residual below 50 eps_32 sqrt(steps) (roundoff).
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.parity import assert_bins

pytestmark = pytest.mark.gpu

NARR = 5   # fields: phi_0, phi_1, A_x, A_y, A_z (each with a momentum)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def both(P, N, kIR, alpha, seed, precision=0, **kw):
    po = O.make_params(**kw)
    pg = P.make_params(precision=precision, **kw)
    return (P.Lattice(O.MODEL_U1_HIGGS, N, kIR, alpha, seed, pg),
            O.Oracle(O.MODEL_U1_HIGGS, N, kIR, alpha, seed, po))


def compare_state(g, o, tol):
    for f in range(NARR):
        for w in (0, 1):
            ref = o.get(f, w)
            if np.abs(ref).max() == 0.0:
                assert np.abs(g.get(f, w)).max() == 0.0, (f, w)
                continue
            e = nrel(g.get(f, w), ref)
            assert e < tol, (f, w, e)


def compare_energies(eg, eo, tol):
    for k in ("EK", "EG", "EV"):
        assert abs(eg[k][0] - eo[k][0]) <= tol * abs(eo[k][0]), (k, eg[k][0], eo[k][0])
    for k in ("EKA", "EGA"):
        assert abs(eg[k] - eo[k]) <= tol * max(abs(eo[k]), 1e-300), (k, eg[k], eo[k])
    for k in ("a", "b", "eta", "rho"):
        assert abs(eg[k] - eo[k]) <= tol * max(abs(eo[k]), 1e-300), (k, eg[k], eo[k])
    for c in range(2):
        scale = {"mean_phi": np.sqrt(eo["mean_phi2"][c]), "mean_phi2": eo["mean_phi2"][c],
                 "mean_pi2": eo["mean_pi2"][c]}
        for k, sc in scale.items():
            assert abs(eg[k][c] - eo[k][c]) <= tol * max(sc, 1e-300), (k, c, eg[k][c], eo[k][c])


# the Abelian-Higgs workload: |phi| at the vacuum v, vacuum fluctuations,
# link momenta from the lattice Gauss law, leapfrog, no expansion
C3 = dict(dt=0.01, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
          phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5)


def test_initial_conditions_match(P):
    g, o = both(P, 24, 0.5, 1.0, 7, **C3)
    compare_state(g, o, 1e-12)
    compare_energies(g.energies(), o.energies(), 1e-12)
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg < 1e-12 and ro < 1e-13


@pytest.mark.parametrize("N,kw,nsteps", [
    (16, C3, 200),                                               # 1 warp-row per 16 threads
    (24, dict(C3, integrator=O.VV2), 100),                       # BY = 12, rows straddle warps
    (32, dict(C3, integrator=O.VV4, expansion=O.EXP_SELF), 40),  # Friedmann sums, carried pre-kick sums
    (16, dict(C3, expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0, H0=0.3), 60),
])
def test_fp64_evolution(P, N, kw, nsteps):
    g, o = both(P, N, 0.5, 1.0, 3, **kw)
    g.step(nsteps)
    o.step(nsteps)
    compare_state(g, o, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10)
    if kw["expansion"] == O.EXP_SELF:
        assert eg["a"] > 1.0001
        assert abs(eg["hubble_viol"]) <= 1.05 * abs(eo["hubble_viol"]) + 1e-15
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg <= 1.05 * ro + 1e-13, (rg, ro)


def test_rough_seeded_state_large_angles(P):
    """Shared seeded state with link angles beyond pi/4 (the library branch of
    the FP32 sine) and O(1) charged-field gradients, alpha = 0."""
    N, kIR, gQ = 16, 0.5, 1.5
    kw = dict(C3, gQ=gQ, fluct_amp2=0.0)
    dx = 2 * np.pi / (N * kIR)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        g, o = both(P, N, kIR, 0.0, 1, precision=prec, **kw)
        for f in range(NARR):
            for w in (0, 1):
                x = inputs.random_field(N, 100 + 2 * f + w)
                scale = (1.2 / (gQ * dx)) if (f >= 2 and w == 0) else 0.5
                x = (scale * x).astype(np.float32).astype(np.float64) if prec else scale * x
                g.set(f, w, x)
                o.set(f, w, x)
        g.step(10)
        o.step(10)
        compare_state(g, o, tol)
        compare_energies(g.energies(), o.energies(), tol)


def test_fp32_storage_100_steps(P):
    g, o = both(P, 32, 0.5, 1.0, 3, precision=1, **C3)
    g.step(100)
    o.step(100)
    compare_state(g, o, 1e-4)
    compare_energies(g.energies(), o.energies(), 1e-5)
    assert g.gauss()[0] < 50 * 2 ** -24 * np.sqrt(100)


def test_gauge_invariance(P):
    """A gauge transform of the state (phi -> e^{i gQ alpha} phi, A -> A + grad alpha)
    leaves the energies and |phi| of the evolution unchanged."""
    N, kIR = 16, 0.5
    dx = 2 * np.pi / (N * kIR)
    gQ = C3["gQ"]
    a = P.Lattice(O.MODEL_U1_HIGGS, N, kIR, 1.0, 5, P.make_params(**C3))
    b = P.Lattice(O.MODEL_U1_HIGGS, N, kIR, 1.0, 5, P.make_params(**C3))
    al = inputs.random_field(N, 77)
    th = gQ * al
    c, s = np.cos(th), np.sin(th)
    for w in (0, 1):
        x, y = b.get(0, w), b.get(1, w)
        b.set(0, w, c * x - s * y)
        b.set(1, w, s * x + c * y)
    for i, ax in enumerate((2, 1, 0)):   # arrays are [z][y][x]
        grad = (np.roll(al, -1, axis=ax) - al) / dx
        b.set(2 + i, 0, b.get(2 + i, 0) + grad)
    a.step(30)
    b.step(30)
    ea, eb = a.energies(), b.energies()
    for k in ("EK", "EG", "EV"):
        assert abs(ea[k][0] - eb[k][0]) < 1e-10 * abs(ea[k][0])
    assert abs(ea["EKA"] - eb["EKA"]) < 1e-10 * abs(ea["EKA"]) + 1e-18
    m1 = a.get(0, 0) ** 2 + a.get(1, 0) ** 2
    m2 = b.get(0, 0) ** 2 + b.get(1, 0) ** 2
    assert np.abs(m1 - m2).max() < 1e-10
    for i in range(3):
        assert np.abs(a.get(2 + i, 1) - b.get(2 + i, 1)).max() < 1e-10


def test_single_pass_launches_match_multi_pass(P):
    kw = dict(C3, integrator=O.VV2, expansion=O.EXP_SELF)
    a = P.Lattice(O.MODEL_U1_HIGGS, 32, 0.5, 1.0, 8, P.make_params(precision=1, **kw))
    b = P.Lattice(O.MODEL_U1_HIGGS, 32, 0.5, 1.0, 8, P.make_params(precision=1, **kw))
    a.step(12)
    for _ in range(12):
        b.step(1)
    for f in range(NARR):
        for w in (0, 1):
            assert np.array_equal(a.get(f, w), b.get(f, w)), (f, w)


def test_time_reversal(P):
    g = P.Lattice(O.MODEL_U1_HIGGS, 24, 0.5, 1.0, 4,
                  P.make_params(**dict(C3, integrator=O.VV4, expansion=O.EXP_SELF)))
    s0 = [g.get(f, w) for f in range(NARR) for w in (0, 1)]
    g.step(30)
    g.step(30, h=-C3["dt"])
    for x, y in zip(s0, [g.get(f, w) for f in range(NARR) for w in (0, 1)]):
        if np.abs(x).max() > 0:
            assert nrel(y, x) < 1e-10


def test_full_size_fp32_leapfrog(P):
    """256^3, FP32, leapfrog, no expansion (the Abelian-Higgs benchmark
    configuration), checked by properties that hold at any size: the Gauss
    law kept to roundoff, energy conserved to the integrator's accuracy, a
    finite state, and time reversal to FP32 roundoff."""
    N, kIR = 256, 0.1
    g = P.Lattice(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, P.make_params(precision=1, **C3))
    r0 = g.gauss()
    e0 = g.energies()
    # phi_0, pi_0, pi_A,x (the links themselves start at zero)
    sel = ((0, 0), (0, 1), (2, 1))
    s0 = [g.get(f, w) for f, w in sel]
    g.step(40)
    e1 = g.energies()
    r1 = g.gauss()
    ax = np.abs(g.get(2, 0)).max()
    assert e1["nonfinite"] == 0 and ax > 0.0
    assert abs(e1["rho"] / e0["rho"] - 1.0) < 5e-3
    assert r1[0] < 50 * 2 ** -24 * np.sqrt(40) and r0[0] < 1e-6
    g.step(40, h=-C3["dt"])
    for x, (f, w) in zip(s0, sel):
        assert nrel(g.get(f, w), x) < 1e-4, (f, w)
    assert np.abs(g.get(2, 0)).max() < 1e-3 * ax
    g.close()


def test_errors(P):
    with pytest.raises(P.ClError) as e:
        P.Lattice(O.MODEL_U1_HIGGS, 16, 0.5, 1.0, 1, P.make_params(**dict(C3, gQ=0.0)))
    assert e.value.status == P.CL_EINVAL
    g = P.Lattice(O.MODEL_U1_HIGGS, 16, 0.5, 1.0, 1, P.make_params(**C3))
    assert g.nfields() == NARR
    with pytest.raises(P.ClError):
        g.get(5, 0)


@pytest.mark.parametrize("precision,alpha", [(0, 1.0), (0, 0.0), (1, 1.0)])
def test_electric_and_magnetic_spectra_match(P, precision, alpha):
    """cl_em_spectrum against the oracle on the same state and scalars, with
    self-consistent expansion (a != 1 enters E through a^{alpha-1})."""
    kw = dict(C3, expansion=O.EXP_SELF, fstar_over_mp=2.0)
    g, o = both(P, 24, 0.5, alpha, 6, precision=precision, **kw)
    g.step(30)
    for f in range(NARR):
        for w in (0, 1):
            o.set(f, w, g.get(f, w))
    o.set_scalars(*g.scalars())
    assert abs(g.scalars()[1] - 1.0) > 1e-3
    for which in (0, 1):
        for dk in (1.0, 1.5):
            kg, dg, mg = g.em_spectrum(which, dk)
            ko, do, mo = o.em_spectrum(which, dk)
            assert np.array_equal(mg, mo)
            assert np.abs(kg - ko).max() < 1e-12 * ko.max()
            assert_bins(dg, do, 1e-10, (which, dk))
    s = P.Lattice(O.MODEL_LPHI4, 16, 0.5, 1.0, 1, P.make_params(dt=0.01, phi0=[1.0], fluct_amp2=1e-4))
    with pytest.raises(P.ClError) as e:
        s.em_spectrum(0)
    assert e.value.status == P.CL_EUNSUPPORTED
