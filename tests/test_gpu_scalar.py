"""GPU parity of the scalar-field path (C ABI, sm_103a kernels) against the
FP64 CPU oracle, on the same seeds / the same seeded input states.

Tolerances (normwise: max |gpu - oracle| / max |oracle| per array):
  FP64 storage: 1e-10 pointwise after 200 steps, 1e-10 on volume averages,
                Hubble-constraint violation <= 1.05 x the oracle's;
  FP32 storage: 1e-4 pointwise after 100 steps, 1e-5 on volume averages.
"""
import numpy as np
import pytest

import oracle as O
from tests import inputs
from tests.parity import assert_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def both(P, model, N, kIR, alpha, seed, precision=0, **kw):
    po = O.make_params(**kw)
    pg = P.make_params(precision=precision, **kw)
    return P.Lattice(model, N, kIR, alpha, seed, pg), O.Oracle(model, N, kIR, alpha, seed, po)


def compare_state(g, o, nf, tol):
    for f in range(nf):
        for w in (0, 1):
            e = nrel(g.get(f, w), o.get(f, w))
            assert e < tol, (f, w, e)


def compare_energies(eg, eo, tol, keys=("EK", "EG", "EV")):
    for k in keys:
        for i in range(4):
            if eo[k][i] != 0.0:
                assert abs(eg[k][i] - eo[k][i]) <= tol * abs(eo[k][i]), (k, i, eg[k][i], eo[k][i])
    for k in ("a", "b", "eta", "rho"):
        assert abs(eg[k] - eo[k]) <= tol * max(abs(eo[k]), 1e-300), (k, eg[k], eo[k])


C1 = dict(dt=0.01, integrator=O.VV2, phi0=[1.0], fluct_amp2=1e-4, expansion=O.EXP_SELF,
          fstar_over_mp=0.5)
C2S = dict(dt=0.005, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4,
           expansion=O.EXP_SELF, fstar_over_mp=0.5)


# ---------------------------------------------------------------------------
# initial conditions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("model,N,kIR,kw", [
    (O.MODEL_LPHI4, 32, 0.5, C1),
    (O.MODEL_LPHI4_CHI, 48, 0.5, C2S),
    (O.MODEL_LPHI4_CHI, 24, 0.3, dict(C2S, kcut=1.0)),
    (O.MODEL_LPHI4_CHI, 8, 1.0, dict(C2S, dphi0=[0.2, 0.1], b0_mode=1)),
])
def test_initial_conditions_match(P, model, N, kIR, kw):
    g, o = both(P, model, N, kIR, 1.0, 7, **kw)
    compare_state(g, o, 1 if model == O.MODEL_LPHI4 else 2, 1e-12)
    compare_energies(g.energies(), o.energies(), 1e-12)


def test_initial_conditions_sampled_modes_at_256(P):
    """Full-size lattice: Fourier modes of the GPU field against the oracle's one-by-one values."""
    N, kIR = 256, 0.1
    kw = dict(C2S)
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, P.make_params(precision=P.FP64, **kw))
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.integers(0, N ** 3, 400), [1, N - 1, N * N, N ** 3 - 1, N // 2]])
    f, gg = O.ic_sample(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, O.make_params(**kw), idx)
    for fld, off in ((0, 1.0), (1, 0.0)):
        F = np.fft.fftn(g.get(fld, 0) - off).reshape(-1)[idx]
        G = np.fft.fftn(g.get(fld, 1)).reshape(-1)[idx]
        assert np.abs(F - f[:, fld]).max() < 1e-9 * np.abs(f[:, fld]).max()
        assert np.abs(G - gg[:, fld]).max() < 1e-9 * np.abs(gg[:, fld]).max()
    g.close()


# ---------------------------------------------------------------------------
# evolution, FP64 storage
# ---------------------------------------------------------------------------
def test_c1_vv2_200_steps(P):
    g, o = both(P, O.MODEL_LPHI4, 32, 0.5, 1.0, 1, **C1)
    g.step(200)
    o.step(200)
    compare_state(g, o, 1, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10)
    assert abs(eg["hubble_viol"]) <= 1.05 * abs(eo["hubble_viol"]) + 1e-15


@pytest.mark.parametrize("N,integ", [(32, O.VV4), (48, O.VV4), (24, O.LF), (16, O.VV6)])
def test_two_field_evolution(P, N, integ):
    kw = dict(C2S, integrator=integ)
    g, o = both(P, O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 3, **kw)
    n = 200 if integ in (O.VV4, O.LF) else 30
    g.step(n)
    o.step(n)
    compare_state(g, o, 2, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10)
    assert abs(eg["hubble_viol"]) <= 1.05 * abs(eo["hubble_viol"]) + 1e-15


@pytest.mark.parametrize("expansion", [O.EXP_OFF, O.EXP_FIXED])
def test_other_backgrounds(P, expansion):
    kw = dict(C2S, expansion=expansion, omega_eos=1.0 / 3.0, H0=0.3, fluct_amp2=1e-2)
    g, o = both(P, O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 5, **kw)
    g.step(100)
    o.step(100)
    compare_state(g, o, 2, 1e-10)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-10)
    if expansion == O.EXP_OFF:
        assert abs(eg["energy_cons"] - eo["energy_cons"]) < 1e-12


def test_seeded_rough_state_and_alpha0(P):
    """Shared seeded input state (rough, all scales) loaded into both sides, alpha = 0."""
    N = 72   # rows of 36 threads straddle warps
    kw = dict(C2S, fluct_amp2=0.0)
    g, o = both(P, O.MODEL_LPHI4_CHI, N, 0.7, 0.0, 1, **kw)
    for f, (phi, pi) in enumerate(inputs.scalar_state(N, 11, rough=True)):
        for side in (g, o):
            side.set(f, 0, phi)
            side.set(f, 1, pi)
    for side in (g, o):
        side.set_scalars(0.0, 1.0, 0.2)
    g.step(30)
    o.step(30)
    compare_state(g, o, 2, 1e-10)
    compare_energies(g.energies(), o.energies(), 1e-10)


def test_fp64_128_ragged_work_split(P):
    """128^3 FP64: 2048 plane tasks over the SMs, runs of unequal length crossing tiles."""
    kw = dict(C2S)
    g, o = both(P, O.MODEL_LPHI4_CHI, 128, 0.2, 1.0, 6, **kw)
    g.step(6)
    o.step(6)
    compare_state(g, o, 2, 1e-11)
    compare_energies(g.energies(), o.energies(), 1e-11)
    g.close()


def test_stream_of_kicks_is_invisible(P):
    """Measuring in between (closing and reopening the kick stream) changes nothing."""
    a = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 2, P.make_params(**C2S))
    b = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 2, P.make_params(**C2S))
    a.step(40)
    for _ in range(4):
        b.step(10)
        b.energies()
    for f in range(2):
        for w in range(2):
            assert nrel(a.get(f, w), b.get(f, w)) < 1e-12


def test_time_reversal(P):
    g = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 4, P.make_params(**C2S))
    s0 = [g.get(f, w) for f in range(2) for w in range(2)]
    e0, a0, b0 = g.scalars()
    g.step(50)
    g.step(50, h=-C2S["dt"])
    s1 = [g.get(f, w) for f in range(2) for w in range(2)]
    for x, y in zip(s0, s1):
        assert nrel(y, x) < 1e-11
    e1, a1, b1 = g.scalars()
    assert abs(a1 - a0) < 1e-13 and abs(b1 - b0) < 1e-13 and abs(e1 - e0) < 1e-12


def test_spectra_match(P):
    g, o = both(P, O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 9, **C2S)
    g.step(50)
    o.step(50)
    for f in range(2):
        for w in range(2):
            for dk in (1.0, 1.5):
                kg, dg, mg = g.spectrum(f, w, dk)
                ko, do, mo = o.spectrum(f, w, dk)
                assert np.array_equal(mg, mo)
                assert np.abs(kg - ko).max() < 1e-12 * ko.max()
                assert_bins(dg, do, 1e-9, (f, w, dk))


@pytest.mark.parametrize("alpha", [1.0, 0.5])
def test_occupation_number_matches(P, alpha):
    """cl_occupation against the oracle on the same synchronised state, with
    self-consistent expansion (a != 1, a' != 0), both fields, two bin widths."""
    kw = dict(C2S, expansion=O.EXP_SELF, fstar_over_mp=2.0)
    g, o = both(P, O.MODEL_LPHI4_CHI, 32, 0.5, alpha, 9, **kw)
    g.step(40)
    for f in range(2):
        for w in (0, 1):
            o.set(f, w, g.get(f, w))
    o.set_scalars(*g.scalars())
    assert g.scalars()[1] > 1.05
    for f in range(2):
        for dk in (1.0, 1.5):
            kg, ng, mg = g.occupation(f, dk)
            ko, no, mo = o.occupation(f, dk)
            assert np.array_equal(mg, mo)
            assert np.abs(kg - ko).max() < 1e-12 * ko.max()
            assert_bins(ng, no, 1e-10, (f, dk))


def test_occupation_number_fp32_and_vacuum(P):
    """FP32 storage: at the initial conditions the vacuum gives 1/2 per mode on
    average, and the GPU matches the oracle on the same FP32-rounded state."""
    kw = dict(C2S, expansion=O.EXP_SELF, fstar_over_mp=2.0)
    g, o = both(P, O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 4, precision=1, **kw)
    for f in range(2):
        for w in (0, 1):
            o.set(f, w, g.get(f, w))
    o.set_scalars(*g.scalars())
    for f in range(2):
        kg, ng, mg = g.occupation(f)
        ko, no, mo = o.occupation(f)
        assert np.array_equal(mg, mo)
        assert_bins(ng, no, 1e-9, f)
        assert abs(np.sum(ng * mg) / np.sum(mg) - 0.5) < 0.05
    # an explicit (f*/omega*)^2 scales it
    k3, n3, m3 = g.occupation(0, 1.0, fo2=3.0 / kw["fluct_amp2"])
    k1, n1, m1 = g.occupation(0, 1.0)
    assert np.allclose(n3, 3.0 * n1, rtol=1e-13, atol=0)
    u = P.Lattice(O.MODEL_U1_HIGGS, 16, 0.5, 1.0, 1,
                  P.make_params(dt=0.01, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, phi0=[1.0, 1.0],
                                fluct_amp2=1e-2, expansion=O.EXP_OFF))
    with pytest.raises(P.ClError) as e:
        u.occupation(0)
    assert e.value.status == P.CL_EUNSUPPORTED


# ---------------------------------------------------------------------------
# FP32 storage with FP64 reductions
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [32, 48])
def test_fp32_storage_100_steps(P, N):
    g, o = both(P, O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 3, precision=P.FP32, **C2S)
    g.step(100)
    o.step(100)
    compare_state(g, o, 2, 1e-4)
    eg, eo = g.energies(), o.energies()
    compare_energies(eg, eo, 1e-5)
    assert abs(eg["hubble_viol"] - eo["hubble_viol"]) < 1e-6


def test_fp32_full_size_bench_configuration(P):
    """256^3, two fields, VV4, self-consistent expansion, FP32 storage: the
    launch configuration the benchmark times, from a shared seeded state."""
    N, kIR = 256, 0.1
    kw = dict(C2S, fluct_amp2=0.0)
    g, o = both(P, O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, precision=P.FP32, **kw)
    for f, (phi, pi) in enumerate(inputs.scalar_state(N, 5)):
        for side in (g, o):
            side.set(f, 0, phi)
            side.set(f, 1, pi)
    for side in (g, o):
        side.set_scalars(0.0, 1.0, 0.15)
    g.step(2)
    o.step(2)
    compare_state(g, o, 2, 1e-5)
    compare_energies(g.energies(), o.energies(), 1e-6)
    g.close()


# ---------------------------------------------------------------------------
# boundary behaviour
# ---------------------------------------------------------------------------
def test_state_roundtrip_and_errors(P):
    g = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**C2S))
    x = inputs.random_field(16, 3)
    g.set(1, 0, x)
    assert np.array_equal(g.get(1, 0), x)
    with pytest.raises(P.ClError) as e:
        g.get(2, 0)
    assert e.value.status == P.CL_EINVAL
    with pytest.raises(P.ClError) as e:
        g.step(-1)
    assert e.value.status == P.CL_EINVAL
    for bad_N in (7, 20, 1024, 40 * 5):
        with pytest.raises(P.ClError) as e:
            P.Lattice(O.MODEL_LPHI4, bad_N, 0.5, 1.0, 1, P.make_params())
        assert e.value.status == P.CL_EINVAL
    with pytest.raises(P.ClError):
        P.Lattice(O.MODEL_LPHI4, 16, -1.0, 1.0, 1, P.make_params())
    g.step(0)
    nb = g.state_bytes()
    assert nb == 4 * 16 ** 3 * 8


def test_degenerate_cases(P):
    # no fluctuations: the lattice stays homogeneous and equals the N = 8 oracle
    kw = dict(C2S, fluct_amp2=0.0, phi0=[1.0, 0.2])
    g, o = both(P, O.MODEL_LPHI4_CHI, 8, 1.0, 1.0, 1, **kw)
    g.step(100)
    o.step(100)
    compare_state(g, o, 2, 1e-11)
    assert np.ptp(g.get(0, 0)) == 0.0
    # kcut = 0 removes every mode
    g2 = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**dict(C2S, kcut=0.0)))
    assert np.ptp(g2.get(0, 0)) == 0.0 and np.ptp(g2.get(1, 0)) == 0.0
    # a zero step changes nothing
    g3 = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**C2S))
    s = g3.get(0, 0)
    g3.step(3, h=0.0)
    assert np.array_equal(g3.get(0, 0), s)


def test_kernel_launch_count_and_pass_timing(P):
    g = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 1, P.make_params(**C2S))
    n0 = g.launches()
    g.enable_pass_timing(True)
    g.step(10)
    g.sync()
    g.enable_pass_timing(False)
    # VV4: 30 passes (one opening, 29 merged kicks) in one cooperative launch,
    # then the closing half kick
    assert g.launches() - n0 == 2
    ms, npass = g.pass_timing(reset=True)
    assert npass == 31 and ms > 0.0


def test_single_pass_launches_match_multi_pass(P):
    """cl_step(1) repeatedly (separate launches) == cl_step(n) (one cooperative launch)."""
    a = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 8, P.make_params(**dict(C2S, integrator=O.VV2)))
    b = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 8, P.make_params(**dict(C2S, integrator=O.VV2)))
    a.step(12)
    for _ in range(12):
        b.step(1)
    for f in range(2):
        for w in range(2):
            assert np.array_equal(a.get(f, w), b.get(f, w))


@pytest.mark.parametrize("precision", [0, 1])
def test_nonfinite_state_is_reported(P, precision):
    """Failure detection without a GPU fault: a NaN planted in one site's
    momentum on the host spreads through the passes; the fused measurement
    counts the non-finite momenta and cl_energies returns CL_ENONFINITE (the
    data are still returned); a clean context is unaffected."""
    g = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 1, P.make_params(precision=precision, **C2S))
    clean = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 1, P.make_params(precision=precision, **C2S))
    pi = g.get(1, 1)
    pi[3, 5, 7] = np.nan
    g.set(1, 1, pi)
    g.step(2)
    clean.step(2)
    with pytest.raises(P.ClError) as e:
        g.energies()
    assert e.value.status == P.CL_ENONFINITE
    assert g.energies(allow_nonfinite=True)["nonfinite"] > 0
    assert clean.energies()["nonfinite"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_exact(P, precision, tmp_path):
    """cl_checkpoint_save / cl_checkpoint_load: a run resumed from a checkpoint
    (into a context made with another seed) continues bit for bit like the
    uninterrupted run, self-consistent expansion included; a checkpoint of
    another lattice size is refused."""
    path = str(tmp_path / "lat.ckpt")
    a = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 3, P.make_params(precision=precision, **C2S))
    a.step(7)
    a.save(path)
    a.step(9)
    b = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 99, P.make_params(precision=precision, **C2S))
    b.load(path)
    b.step(9)
    for f in range(2):
        for w in range(2):
            assert np.array_equal(a.get(f, w), b.get(f, w)), (f, w)
    assert a.scalars() == b.scalars()
    assert a.energies()["rho"] == b.energies()["rho"]
    c = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, P.make_params(precision=precision, **C2S))
    with pytest.raises(P.ClError) as e:
        c.load(path)
    assert e.value.status == P.CL_EINVAL
