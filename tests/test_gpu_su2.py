"""GPU parity of the SU(2) x U(1) doublet path (C ABI, sm_103a kernels)
against the FP64 CPU oracle, on the same seeds or the same seeded states.

Tolerances (normwise: max |gpu - oracle| / max |oracle| per array):
  FP64 storage: 1e-10 pointwise and on volume averages; Gauss residuals
                <= 1.05 x the oracle's (both at roundoff).  E_G^B also
                allows the oracle's own rounding: it sums 2 - Tr U_ij, whose
                absolute error is a few eps_64 per plaquette however small
                the field (the kernel forms 1 - Tr U_ij/2 as |p|^2/(1 + p_0),
                exact for unit quaternions), i.e. 100 eps_64 times the
                energy per unit of <2 - Tr U_ij>;
  FP32 storage: 1e-4 pointwise after 40 steps, 1e-5 on volume averages;
                Gauss residual below 50 eps_32 sqrt(steps).
Lattice sizes: 16^3 (16 x 8 tiles), 48^3 (16-wide tiles, runs that cross
tile boundaries and wrap in z), 64^3 (32 x 8 tiles, several planes per CTA).
"""
import numpy as np
import pytest

import oracle as O
from tests.parity import assert_bins
from tests.inputs import su2_doublet_state
from tests.test_oracle_su2 import gauge_transform

pytestmark = pytest.mark.gpu

NA = 35


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# the doublet workload: equal homogeneous components (the manual's choice,
# zero homogeneous charge), vacuum fluctuations, links at the identity,
# electric fields from the Gauss laws
SU2 = dict(dt=0.01, integrator=O.LF, lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
           phi0=[0.5] * 4, dphi0=[0.1] * 4, fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5)


def both(P, N, kIR, alpha, seed, precision=0, **kw):
    po = O.make_params(**kw)
    pg = P.make_params(precision=precision, **kw)
    return (P.Lattice(O.MODEL_SU2U1_HIGGS, N, kIR, alpha, seed, pg),
            O.Oracle(O.MODEL_SU2U1_HIGGS, N, kIR, alpha, seed, po))


def load_both(g, o, arrays, fp32=False):
    for a, x in enumerate(arrays):
        if fp32:
            x = x.astype(np.float32).astype(np.float64)
        g.set_array(a, x)
        o.set_array(a, x)


def compare_state(g, o, tol):
    for a in range(NA):
        ref = o.get_array(a)
        got = g.get_array(a)
        if np.abs(ref).max() == 0.0:
            assert np.abs(got).max() == 0.0, a
            continue
        e = nrel(got, ref)
        assert e < tol, (a, e)


def egb_floor(N, kIR, kw, a=1.0):
    """100 eps_64 x the E_G^B of a unit of <sum_{i<j} (2 - Tr U_ij)> per site."""
    dx = 2 * np.pi / (N * kIR)
    unit = 2.0 / (kw["fstar_over_omegastar"] ** 2 * a ** 4 * (kw["gQB"] * dx * dx) ** 2)
    return 100 * 2.0 ** -52 * unit


def compare_energies(eg, eo, tol, floor=0.0):
    for k in ("EK", "EG", "EV"):
        assert abs(eg[k][0] - eo[k][0]) <= tol * abs(eo[k][0]), (k, eg[k][0], eo[k][0])
    for k in ("EKA", "EGA", "EKB", "EGB", "a", "b", "eta", "rho"):
        fl = floor if k in ("EGB", "rho") else 0.0
        assert abs(eg[k] - eo[k]) <= tol * max(abs(eo[k]), 1e-300) + fl, (k, eg[k], eo[k])
    for c in range(4):
        for k, sc in (("mean_phi", np.sqrt(eo["mean_phi2"][c])), ("mean_phi2", eo["mean_phi2"][c]),
                      ("mean_pi2", eo["mean_pi2"][c])):
            assert abs(eg[k][c] - eo[k][c]) <= tol * max(sc, 1e-300), (k, c, eg[k][c], eo[k][c])


@pytest.mark.parametrize("N", [16, 32])
def test_initial_conditions_match(P, N):
    g, o = both(P, N, 0.8, 1.0, 7, **SU2)
    compare_state(g, o, 1e-12)
    compare_energies(g.energies(), o.energies(), 1e-12, egb_floor(N, 0.8, SU2))
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg < 1e-12 and ro < 1e-13
    assert np.abs(g.get_array(26)).max() > 1e-6     # SU(2) electric field from the Gauss law


@pytest.mark.parametrize("N,kw,nsteps", [
    (16, dict(SU2, integrator=O.VV2), 30),
    (48, dict(SU2, integrator=O.VV4, expansion=O.EXP_SELF), 2),
    (64, SU2, 3),
    (16, dict(SU2, expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0, H0=0.3), 20),
    (16, dict(SU2, gQ=0.0), 20),                                 # no U(1) field
])
def test_fp64_evolution_from_ics(P, N, kw, nsteps):
    g, o = both(P, N, 0.8, 1.0, 3, **kw)
    g.step(nsteps)
    o.step(nsteps)
    compare_state(g, o, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10, egb_floor(N, 0.8, kw, eo["a"]))
    if kw["expansion"] == O.EXP_SELF:
        assert eg["a"] > 1.0001
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg <= 1.05 * ro + 1e-13, (rg, ro)


@pytest.mark.parametrize("N,alpha,integ", [(16, 1.0, O.VV2), (48, 0.0, O.LF)])
def test_fp64_random_non_abelian_state(P, N, alpha, integ):
    """Shared seeded state far from the identity (plaquettes and link angles
    beyond the FP32 Taylor ranges), self-consistent expansion."""
    kw = dict(SU2, integrator=integ, expansion=O.EXP_SELF, fluct_amp2=0.0)
    g, o = both(P, N, 0.8, alpha, 1, **kw)
    load_both(g, o, su2_doublet_state(N, 31, link_spread=1.0))
    g.step(4)
    o.step(4)
    compare_state(g, o, 1e-10)
    eo = o.energies()
    compare_energies(g.energies(), eo, 1e-10, egb_floor(N, 0.8, kw, eo["a"]))
    rg, ro = g.gauss()[0], o.gauss()[0]
    assert rg <= 1.05 * ro + 1e-13


def test_fp32_storage(P):
    g, o = both(P, 32, 0.8, 1.0, 3, precision=1, **SU2)
    g.step(40)
    o.step(40)
    compare_state(g, o, 1e-4)
    compare_energies(g.energies(), o.energies(), 1e-5)
    assert g.gauss()[0] < 50 * 2 ** -24 * np.sqrt(40)


def test_fp32_random_state(P):
    N = 16
    g, o = both(P, N, 0.8, 1.0, 1, precision=1, **dict(SU2, fluct_amp2=0.0, integrator=O.VV2))
    load_both(g, o, su2_doublet_state(N, 5, link_spread=1.0), fp32=True)
    g.step(10)
    o.step(10)
    compare_state(g, o, 1e-4)
    compare_energies(g.energies(), o.energies(), 1e-5)


@pytest.mark.parametrize("model,N", [(O.MODEL_SU2U1_HIGGS, 64), (O.MODEL_SU2U1_HIGGS, 48),
                                     (O.MODEL_LPHI4_SU2U1, 64)])
def test_kick_then_drift_pass_repeatable_and_pointwise(P, model, N):
    """Without expansion the doublet passes kick, then drift, with the planes and the
    own momenta streamed into shared memory by asynchronous copies.  Two runs from the
    same seed agree bit for bit (no copy is read before it lands, whatever the timing),
    and after 12 FP32 leapfrog steps every array agrees with the oracle started from
    the same FP32-rounded state.  N = 64: every CTA takes one short z-chunk, so most
    planes sit next to the end of a CTA's sequence; N = 48: tiles 16 wide."""
    kw = dict(SU2, v=0.0, qG=1.5, qH=0.8, Qc=0.7) if model == O.MODEL_LPHI4_SU2U1 else SU2
    na = 41 if model == O.MODEL_LPHI4_SU2U1 else 35
    runs = []
    for rep in range(2):
        g = P.Lattice(model, N, 0.5, 1.0, 4, P.make_params(precision=1, **kw))
        if rep == 0:
            o = O.Oracle(model, N, 0.5, 1.0, 4, O.make_params(**dict(kw, fluct_amp2=0.0)))
            for a in range(na):
                o.set_array(a, g.get_array(a))
            o.set_scalars(*g.scalars())
        g.step(12)
        runs.append([g.get_array(a) for a in range(na)])
        g.close()
    o.step(12)
    for a in range(na):
        assert np.array_equal(runs[0][a], runs[1][a]), a
        ref = o.get_array(a)
        if np.abs(ref).max() == 0.0:
            assert np.abs(runs[0][a]).max() == 0.0, a
        else:
            assert nrel(runs[0][a], ref) < 1e-4, (a, nrel(runs[0][a], ref))


def test_gauge_covariance(P):
    """A random SU(2) x U(1) gauge transformation of the initial state commutes
    with the evolution (the GPU's own runs, to roundoff)."""
    N, kIR = 16, 0.8
    dx = 2 * np.pi / (N * kIR)
    rng = np.random.default_rng(21)
    om = rng.standard_normal((4, N, N, N))
    om /= np.sqrt((om ** 2).sum(0))
    beta = rng.standard_normal((N, N, N))
    kw = dict(SU2, integrator=O.VV2, expansion=O.EXP_SELF)
    a = P.Lattice(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 5, P.make_params(**kw))
    b = P.Lattice(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 5, P.make_params(**kw))
    s = su2_doublet_state(N, 8)
    for i, x in enumerate(s):
        a.set_array(i, x)
    for i, x in enumerate(gauge_transform(s, om, beta, SU2["gQ"], dx)):
        b.set_array(i, x)
    a.step(10)
    b.step(10)
    ea, eb = a.energies(), b.energies()
    for k in ("EK", "EG", "EV"):
        assert abs(ea[k][0] - eb[k][0]) < 1e-11 * abs(ea[k][0])
    for k in ("EKA", "EGA", "EKB", "EGB", "a"):
        assert abs(ea[k] - eb[k]) < 1e-11 * abs(ea[k])
    ref = gauge_transform([a.get_array(i) for i in range(NA)], om, beta, SU2["gQ"], dx)
    for i in range(NA):
        assert np.abs(b.get_array(i) - ref[i]).max() < 1e-10, i


def test_time_reversal(P):
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, 32, 0.8, 1.0, 4,
                  P.make_params(**dict(SU2, integrator=O.VV4, expansion=O.EXP_SELF)))
    s0 = [g.get_array(a) for a in range(NA)]
    g.step(20)
    g.step(20, h=-SU2["dt"])
    for a, x in enumerate(s0):
        y = g.get_array(a)
        assert np.abs(y - x).max() < 1e-10 * max(1.0, np.abs(x).max()), a


def test_doublet_spectrum_matches(P):
    g, o = both(P, 32, 0.8, 1.0, 2, **SU2)
    g.step(10)
    o.step(10)
    for f in (0, 3):
        kg, dg, mg = g.spectrum(f, 0)
        ko, do, mo = o.spectrum(f, 0)
        assert np.array_equal(mg, mo)
        assert np.abs(kg - ko).max() < 1e-12
        assert_bins(dg, do, 1e-10, f)


def test_full_size_fp32(P):
    """256^3, FP32, leapfrog, no expansion (the size the bench times),
    checked by properties that hold at any size: both Gauss laws kept to
    roundoff, energy conserved to the integrator's accuracy, a finite state,
    links unitary, and time reversal to FP32 roundoff."""
    N, kIR = 256, 0.1
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 1, P.make_params(precision=1, **SU2))
    e0 = g.energies()
    r0 = g.gauss()
    sel = (0, 4, 26, 11)
    s0 = [g.get_array(a) for a in sel]
    g.step(40)
    e1 = g.energies()
    r1 = g.gauss()
    assert e1["nonfinite"] == 0
    assert abs(e1["rho"] / e0["rho"] - 1.0) < 5e-3
    assert r0[0] < 1e-6 and r1[0] < 50 * 2 ** -24 * np.sqrt(40)
    u = [g.get_array(14 + k) for k in range(4)]
    assert np.abs(sum(x * x for x in u) - 1.0).max() < 1e-6
    assert np.abs(u[1]).max() > 0.0
    g.step(40, h=-SU2["dt"])
    for x, a in zip(s0, sel):
        assert nrel(g.get_array(a), x) < 1e-4, a
    g.close()


def test_errors(P):
    with pytest.raises(P.ClError) as e:
        P.Lattice(O.MODEL_SU2U1_HIGGS, 16, 0.8, 1.0, 1, P.make_params(**dict(SU2, gQB=0.0)))
    assert e.value.status == P.CL_EINVAL
    with pytest.raises(P.ClError) as e:
        P.Lattice(O.MODEL_SU2U1_HIGGS, 24, 0.8, 1.0, 1, P.make_params(**SU2))
    assert e.value.status == P.CL_EUNSUPPORTED
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, 16, 0.8, 1.0, 1, P.make_params(**SU2))
    assert g.nfields() == 7
    with pytest.raises(P.ClError):
        g.get_array(35)
    with pytest.raises(P.ClError):
        g.get(7, 0)
    with pytest.raises(P.ClError) as e:
        g.em_spectrum(4)
    assert e.value.status == P.CL_EINVAL


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_modulus_spectra_match(P, precision, tol):
    """cl_norm_spectrum against the oracle: Delta of |Phi|, of |Phi|', and the
    occupation number of |Phi| (self-consistent expansion, a != 1)."""
    kw = dict(SU2, integrator=O.VV2, expansion=O.EXP_SELF)
    g, o = both(P, 32, 0.8, 1.0, 2, precision=precision, **kw)
    g.step(10)
    o.step(10)
    rg, ro = g.norm_spectrum(), o.norm_spectrum()
    assert np.array_equal(rg[4], ro[4])
    assert np.abs(rg[0] - ro[0]).max() < 1e-12
    for i, (x, y) in enumerate(zip(rg[1:4], ro[1:4])):
        assert_bins(x, y, tol, i)


def test_modulus_spectra_u1(P):
    kw = dict(dt=0.01, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
              phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5)
    g = P.Lattice(O.MODEL_U1_HIGGS, 32, 0.5, 1.0, 3, P.make_params(**kw))
    o = O.Oracle(O.MODEL_U1_HIGGS, 32, 0.5, 1.0, 3, O.make_params(**kw))
    g.step(20)
    o.step(20)
    rg, ro = g.norm_spectrum(), o.norm_spectrum()
    assert np.array_equal(rg[4], ro[4])
    for i, (x, y) in enumerate(zip(rg[1:4], ro[1:4])):
        assert_bins(x, y, 1e-10, i)
    s = P.Lattice(O.MODEL_LPHI4, 16, 0.5, 1.0, 1, P.make_params(fluct_amp2=1e-2))
    with pytest.raises(P.ClError) as e:
        s.norm_spectrum()
    assert e.value.status == P.CL_EUNSUPPORTED


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-5)])
def test_gauge_field_spectra_match(P, precision, tol):
    """cl_em_spectrum of the doublet model (U(1) E, B and SU(2) E, B) against the
    oracle, after 10 steps with self-consistent expansion."""
    kw = dict(SU2, integrator=O.VV2, expansion=O.EXP_SELF)
    g, o = both(P, 32, 0.8, 1.0, 4, precision=precision, **kw)
    g.step(10)
    o.step(10)
    for which in range(4):
        kg, dg, mg = g.em_spectrum(which)
        ko, do, mo = o.em_spectrum(which)
        assert np.array_equal(mg, mo)
        assert np.abs(kg - ko).max() < 1e-12
        assert_bins(dg, do, tol, which)
    nou1 = P.Lattice(O.MODEL_SU2U1_HIGGS, 16, 0.8, 1.0, 1, P.make_params(**dict(SU2, gQ=0.0)))
    with pytest.raises(P.ClError) as e:
        nou1.em_spectrum(1)
    assert e.value.status == P.CL_EUNSUPPORTED


def test_largest_lattice_fp32(P):
    """512^3 (the largest N the library takes; 37.6 GB of state): the initial
    Gauss laws, a finite leapfrog run with both laws kept to FP32 roundoff and
    the energy conserved to the integrator's accuracy."""
    N = 512
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, N, 0.05, 1.0, 1, P.make_params(precision=1, **SU2))
    e0 = g.energies()
    r0 = g.gauss()
    g.step(6)
    e1 = g.energies()
    r1 = g.gauss()
    assert e1["nonfinite"] == 0 and e1["EKB"] > 0.0
    assert r0[0] < 1e-6 and r1[0] < 50 * 2 ** -24 * np.sqrt(6)
    assert abs(e1["rho"] / e0["rho"] - 1.0) < 1e-3
    g.close()


def test_nonfinite_link_momentum_is_reported(P):
    """An infinite SU(2) link momentum planted on the host is counted by the
    doublet pass's measurement and reported as CL_ENONFINITE."""
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, 16, 0.8, 1.0, 1, P.make_params(precision=1, **SU2))
    x = g.get_array(27)
    x[2, 3, 4] = np.inf
    g.set_array(27, x)
    g.step(1)
    with pytest.raises(P.ClError) as e:
        g.energies()
    assert e.value.status == P.CL_ENONFINITE
    assert g.energies(allow_nonfinite=True)["nonfinite"] > 0


def test_checkpoint_resume_is_exact(P, tmp_path):
    path = str(tmp_path / "su2.ckpt")
    kw = dict(SU2, integrator=O.VV2, expansion=O.EXP_SELF)
    a = P.Lattice(O.MODEL_SU2U1_HIGGS, 32, 0.8, 1.0, 3, P.make_params(precision=1, **kw))
    a.step(5)
    a.save(path)
    a.step(6)
    b = P.Lattice(O.MODEL_SU2U1_HIGGS, 32, 0.8, 1.0, 8, P.make_params(precision=1, **kw))
    b.load(path)
    b.step(6)
    for i in range(NA):
        assert np.array_equal(a.get_array(i), b.get_array(i)), i
    assert a.scalars() == b.scalars()


def test_vv6_and_raw_state_round_trip(P):
    """The sixth-order composition on the doublet model matches the oracle, and
    the whole 35-array state round-trips through cl_download_state /
    cl_upload_state (the end-to-end path)."""
    kw = dict(SU2, integrator=O.VV6)
    g, o = both(P, 16, 0.8, 1.0, 6, **kw)
    g.step(3)
    o.step(3)
    compare_state(g, o, 1e-10)
    n = g.state_bytes()
    import ctypes
    buf = (ctypes.c_char * n)()
    g.download(ctypes.addressof(buf), n)
    s0 = [g.get_array(a) for a in range(NA)]
    g.step(2)
    g.upload(ctypes.addressof(buf), n)
    for a in range(NA):
        assert np.array_equal(g.get_array(a), s0[a]), a
