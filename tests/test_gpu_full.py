"""GPU parity of the lphi4SU2U1 model (Sec. 4.5: doublet, singlet, U(1)-charged
scalar, U(1) and SU(2) links, eq. PotGauge) against the FP64 oracle, on the
same seeds / the same seeded input states.

Tolerances (normwise per array, max |gpu - oracle| / max |oracle|):
  FP64: 1e-12 on the initial arrays, 1e-10 after 20 steps, 1e-10 on the
        energies per species; Gauss laws at roundoff (<= 1.05 x the oracle's
        relative residual + 1e-13);
  FP32: 1e-4 after 50 steps, 1e-5 on the energies.
"""
import numpy as np
import pytest

import oracle as O
from tests.inputs import su2_doublet_state
from tests.parity import assert_bins, nrel

pytestmark = pytest.mark.gpu

NA = 41
FULL = dict(dt=0.01, integrator=O.LF, lam=1.0, v=0.0, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
            phi0=[0.5] * 4, dphi0=[0.1] * 4, fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5,
            qG=1.5, qH=0.8, Qc=0.7)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def both(P, N, kIR, seed, precision=0, **kw):
    kw = dict(FULL, **kw)
    return (P.Lattice(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, seed, P.make_params(precision=precision, **kw)),
            O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, seed, O.make_params(**kw)))


def compare_state(g, o, tol):
    for a in range(NA):
        ref, got = o.get_array(a), g.get_array(a)
        if np.abs(ref).max() == 0.0:
            assert np.abs(got).max() == 0.0, a
            continue
        e = nrel(got, ref)
        assert e < tol, (a, e)


def compare_energies(eg, eo, tol):
    """Relative per energy, with an absolute floor of 1e-13 of the total energy
    density: the magnetic energies of links near the identity are tiny sums of
    2 - Tr U_ij (1 - cos theta for U(1)), which the oracle forms with the
    cancellation of two nearly equal numbers (~1e-16 absolute per plaquette)."""
    floor = 1e-13 * abs(eo["rho"])
    for k in ("EK", "EG", "EV"):
        for i in range(3):
            assert abs(eg[k][i] - eo[k][i]) <= tol * abs(eo[k][i]) + floor, (k, i, eg[k][i], eo[k][i])
    for k in ("EKA", "EGA", "EKB", "EGB", "rho"):
        assert abs(eg[k] - eo[k]) <= tol * abs(eo[k]) + floor, (k, eg[k], eo[k])
    for k in ("a", "b"):
        assert abs(eg[k] - eo[k]) <= tol * max(abs(eo[k]), 1e-300), (k, eg[k], eo[k])


def full_state(N, seed, amp=0.3):
    rng = np.random.default_rng(seed + 1000)
    return su2_doublet_state(N, seed) + [amp * rng.standard_normal((N, N, N)) for _ in range(6)]


@pytest.mark.parametrize("N,kIR", [(16, 0.8), (48, 0.5)])
def test_initial_conditions_match(P, N, kIR):
    g, o = both(P, N, kIR, 3)
    compare_state(g, o, 1e-12)
    compare_energies(g.energies(), o.energies(), 1e-12)
    assert np.abs(g.get_array(35)).max() > 0 and np.abs(g.get_array(38)).max() > 0
    rel = g.gauss()[0]
    assert rel < 1e-12


@pytest.mark.parametrize("integ,expansion,n", [(O.LF, O.EXP_OFF, 20), (O.VV4, O.EXP_SELF, 8),
                                               (O.VV2, O.EXP_FIXED, 15)])
def test_evolution_fp64(P, integ, expansion, n):
    kw = dict(integrator=integ, expansion=expansion, omega_eos=1.0 / 3.0, fstar_over_mp=2.0)
    g, o = both(P, 16, 0.8, 5, **kw)
    g.step(n)
    o.step(n)
    compare_state(g, o, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10)
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg <= 1.05 * ro + 1e-13, (rg, ro)
    if expansion == O.EXP_SELF:
        assert eg["a"] > 1.01
        assert abs(eg["hubble_viol"]) <= 1.05 * abs(eo["hubble_viol"]) + 1e-15


def test_seeded_random_state_tx16(P):
    """A rough seeded state on a 48^3 lattice (tiles 16 wide), all couplings on."""
    N = 48
    g, o = both(P, N, 0.5, 1, fluct_amp2=0.0, expansion=O.EXP_SELF, integrator=O.VV2)
    for a, x in enumerate(full_state(N, 7)):
        g.set_array(a, x)
        o.set_array(a, x)
    for side in (g, o):
        side.set_scalars(0.0, 1.0, 0.2)
    g.step(6)
    o.step(6)
    compare_state(g, o, 1e-10)
    compare_energies(g.energies(), o.energies(), 1e-10)


def test_fp32_storage(P):
    g, o = both(P, 32, 0.8, 2, precision=1)
    for a in range(NA):   # the same FP32-rounded start on both sides
        o.set_array(a, g.get_array(a))
    g.step(50)
    o.step(50)
    compare_state(g, o, 1e-4)
    compare_energies(g.energies(), o.energies(), 1e-5)


def test_singlet_and_charged_spectra(P):
    g, o = both(P, 16, 0.8, 9)
    g.step(10)
    o.step(10)
    for field in (7, 8, 9):
        for w in (0, 1):
            kg, dg, mg = g.spectrum(field, w)
            ko, do, mo = o.spectrum(field, w)
            assert np.array_equal(mg, mo)
            assert_bins(dg, do, 1e-10, (field, w))


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_modulus_spectra_of_both_charged_fields(P, precision, tol):
    """cl_norm_spectrum_of against the oracle, bin by bin: Delta of the doublet's
    modulus |Phi| and of vphi's |vphi|, of their rates, and their occupation
    numbers (the doublet's mass with its couplings to phi_s and vphi, vphi's from
    the doublet), with self-consistent expansion (a != 1)."""
    g, o = both(P, 32, 0.8, 2, precision=precision, integrator=O.VV2, expansion=O.EXP_SELF)
    g.step(10)
    o.step(10)
    for which in (0, 1):
        rg, ro = g.norm_spectrum(which=which), o.norm_spectrum(which=which)
        assert np.array_equal(rg[4], ro[4])
        assert np.abs(rg[0] - ro[0]).max() < 1e-12
        for i, (x, y) in enumerate(zip(rg[1:4], ro[1:4])):
            assert_bins(x, y, tol, (which, i))
    # the two fields' occupation numbers differ (different masses and spectra)
    assert np.abs(g.norm_spectrum(which=0)[3] - g.norm_spectrum(which=1)[3]).max() > 0


def test_time_reversal(P):
    g = P.Lattice(O.MODEL_LPHI4_SU2U1, 16, 0.8, 1.0, 4,
                  P.make_params(**dict(FULL, integrator=O.VV4, expansion=O.EXP_SELF, fstar_over_mp=2.0)))
    s0 = [g.get_array(a) for a in range(NA)]
    g.step(10)
    g.step(10, h=-FULL["dt"])
    for a, x in enumerate(s0):
        if np.abs(x).max() > 0:
            assert nrel(g.get_array(a), x) < 1e-10, a


def test_state_access_and_errors(P):
    g = P.Lattice(O.MODEL_LPHI4_SU2U1, 16, 0.8, 1.0, 1, P.make_params(**FULL))
    assert g.nfields() == 10
    assert np.array_equal(g.get(7, 0), g.get_array(35))
    assert np.array_equal(g.get(8, 1), g.get_array(39))
    assert np.array_equal(g.get(9, 0), g.get_array(38))
    with pytest.raises(P.ClError) as e:
        g.get_array(41)
    assert e.value.status == P.CL_EINVAL
    with pytest.raises(P.ClError) as e:
        g.norm_spectrum(which=2)
    assert e.value.status == P.CL_EINVAL
    with pytest.raises(P.ClError) as e:
        P.Lattice(O.MODEL_LPHI4_SU2U1, 24, 0.8, 1.0, 1, P.make_params(**FULL))   # N % 16
    assert e.value.status == P.CL_EUNSUPPORTED
