"""GPU parity of the adjoint sweep (cl_adjoint: reversed DK passes fused with
their transposed Jacobians, checkpoints) against the oracle's discrete
adjoint, and against central finite differences of GPU forward runs in FP64
at 32^3, on fixed backgrounds and with self-consistent expansion.

Tolerances: FP64 storage 1e-9 (normwise) on dJ/d(state), dJ/dq and the
amplitude gradient against the oracle; finite differences 1e-5 relative
(their own truncation error is O(eps^2)); FP32 storage against the FP64
adjoint 2e-3 (rounding of the forward and reversed passes).
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

BASE = dict(dt=0.005, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-2,
            expansion=O.EXP_OFF, fstar_over_mp=0.5)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("N,kw,nsteps,ckpt", [
    (16, BASE, 30, 10),
    (24, dict(BASE, integrator=O.VV2), 40, 7),
    (16, dict(BASE, expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0, H0=0.4), 25, 25),
])
def test_chi_fraction_adjoint_matches_oracle(P, N, kw, nsteps, ckpt):
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 3, P.make_params(**kw))
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 3, O.make_params(**kw))
    s0 = [g.get(f, w) for f in range(2) for w in (0, 1)]
    Jg, qg, lg = g.adjoint(nsteps, ckpt)
    Jo, qo, lo = o.adjoint(nsteps)
    assert abs(Jg - Jo) < 1e-12 * abs(Jo)
    assert abs(qg - qo) < 1e-9 * abs(qo), (qg, qo)
    assert nrel(lg, lo) < 1e-9
    # the state is back at the start, exactly
    for (f, w), x in zip([(f, w) for f in range(2) for w in (0, 1)], s0):
        assert np.array_equal(g.get(f, w), x)
    # and the amplitude gradient chains the same way
    ag, ao = g.ic_amplitude_grad(lg), o.ic_amplitude_grad(lo)
    assert nrel(ag, ao) < 1e-9


@pytest.mark.parametrize("field,what,dk,b", [(1, 0, 1.0, 2), (0, 1, 1.5, 3)])
def test_spectrum_bin_adjoint_matches_oracle(P, field, what, dk, b):
    g = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 4, P.make_params(**BASE))
    o = O.Oracle(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 4, O.make_params(**BASE))
    Jg, qg, lg = g.adjoint(20, 6, P.OBJ_SPECTRUM_BIN, field, what, dk, b)
    Jo, qo, lo = o.adjoint(20, objective=1, field=field, what=what, dk_bin=dk, bin=b)
    assert abs(Jg - Jo) < 1e-10 * abs(Jo)
    assert abs(qg - qo) < 1e-9 * abs(qo) + 1e-18
    assert nrel(lg, lo) < 1e-9


def test_checkpoint_interval_does_not_change_fp64_result(P):
    res = []
    for ck in (3, 50):
        g = P.Lattice(O.MODEL_LPHI4_CHI, 24, 0.5, 1.0, 5, P.make_params(**BASE))
        res.append(g.adjoint(50, ck))
    assert abs(res[0][1] - res[1][1]) < 1e-12 * abs(res[1][1])
    assert nrel(res[0][2], res[1][2]) < 1e-12


def test_central_differences_fp64_32(P):
    """dJ/dq and a state direction against central differences of GPU forward runs (32^3, FP64)."""
    N, kIR, n = 32, 0.5, 200
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 9, P.make_params(**BASE))
    s0 = [[g.get(f, w) for w in (0, 1)] for f in range(2)]
    J, dq, lam = g.adjoint(n, 50)

    def J_of(q, state):
        h = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 9, P.make_params(**dict(BASE, q=q)))
        for f in range(2):
            for w in (0, 1):
                h.set(f, w, state[f][w])
        h.step(n)
        e = h.energies()
        h.close()
        return (e["EK"][1] + e["EG"][1]) / e["rho"]

    assert abs(J_of(BASE["q"], s0) - J) < 1e-12 * J
    eps = 1e-3
    fd = (J_of(BASE["q"] + eps, s0) - J_of(BASE["q"] - eps, s0)) / (2 * eps)
    assert abs(dq - fd) < 1e-5 * abs(fd), (dq, fd)
    rng = np.random.default_rng(3)
    v = [[rng.standard_normal((N, N, N)) * np.abs(s0[f][w]).max() for w in (0, 1)] for f in range(2)]
    e = 1e-7
    sp = [[s0[f][w] + e * v[f][w] for w in (0, 1)] for f in range(2)]
    sm = [[s0[f][w] - e * v[f][w] for w in (0, 1)] for f in range(2)]
    fd = (J_of(BASE["q"], sp) - J_of(BASE["q"], sm)) / (2 * e)
    ad = sum(float(np.sum(lam[f, w] * v[f][w])) for f in range(2) for w in (0, 1))
    assert abs(ad - fd) < 1e-5 * abs(fd), (ad, fd)


def test_fp32_adjoint_close_to_fp64(P):
    kw = BASE
    r = {}
    for prec in (0, 1):
        g = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 2, P.make_params(precision=prec, **kw))
        if prec:   # the same initial state in both precisions
            for f in range(2):
                for w in (0, 1):
                    g.set(f, w, r[0][3][f][w].astype(np.float32).astype(np.float64))
        s = [[g.get(f, w) for w in (0, 1)] for f in range(2)]
        J, dq, lam = g.adjoint(100, 25)
        r[prec] = (J, dq, lam, s)
    assert abs(r[1][0] - r[0][0]) < 1e-5 * abs(r[0][0])
    assert abs(r[1][1] - r[0][1]) < 2e-3 * abs(r[0][1])
    assert nrel(r[1][2], r[0][2]) < 2e-3


def test_autograd_function(P):
    torch = pytest.importorskip("torch")
    from paper_2102_01031_gb300.autograd import RunSpec, evolved_objective
    N = 16
    kw = dict(BASE)
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, P.make_params(**kw))
    s = np.stack([np.stack([g.get(f, w) for w in (0, 1)]) for f in range(2)])
    J0, dq0, lam0 = g.adjoint(20, 10)
    spec = RunSpec.make(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, 20, ckpt_every=10, **kw)
    q = torch.tensor(kw["q"], dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    J = evolved_objective(q, st, spec)
    (3.0 * J).backward()
    assert abs(float(J.detach()) - J0) < 1e-14 * J0
    assert abs(float(q.grad) - 3.0 * dq0) < 1e-12 * abs(3.0 * dq0)
    assert np.abs(st.grad.numpy() - 3.0 * lam0).max() <= 1e-12 * np.abs(3.0 * lam0).max()


def test_autograd_function_device_state(P, monkeypatch):
    """A state held in CUDA tensors goes to the library and its gradient comes
    back without passing through the host: the host transfers are switched off
    for the call, and the result equals the host-array adjoint's."""
    torch = pytest.importorskip("torch")
    from paper_2102_01031_gb300.autograd import RunSpec, evolved_objective
    N = 16
    kw = dict(SELF)
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, P.make_params(**kw))
    s = np.stack([np.stack([g.get(f, w) for w in (0, 1)]) for f in range(2)])
    J0, dq0, lam0, ab0 = g.adjoint(20, 10, scale=True)
    spec = RunSpec.make(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, 20, ckpt_every=10, **kw)
    q = torch.tensor(kw["q"], dtype=torch.float64, device="cuda", requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, device="cuda", requires_grad=True)

    def no_host(*a, **k):
        raise AssertionError("host transfer of the state")
    monkeypatch.setattr(P.Lattice, "set", no_host)
    monkeypatch.setattr(P.Lattice, "get", no_host)
    J = evolved_objective(q, st, spec)
    (0.5 * J).backward()
    monkeypatch.undo()
    assert J.device.type == "cuda" and st.grad.device.type == "cuda"
    assert abs(float(J.detach()) - J0) < 1e-14 * J0
    assert abs(float(q.grad) - 0.5 * dq0) < 1e-12 * abs(0.5 * dq0)
    assert np.abs(st.grad.cpu().numpy() - 0.5 * lam0).max() <= 1e-12 * np.abs(0.5 * lam0).max()


def test_autograd_function_scale(P):
    """Self-consistent expansion: (a, b) at the start as a differentiable input."""
    torch = pytest.importorskip("torch")
    from paper_2102_01031_gb300.autograd import RunSpec, evolved_objective
    N = 16
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, P.make_params(**SELF))
    s = np.stack([np.stack([g.get(f, w) for w in (0, 1)]) for f in range(2)])
    eta0, a0, b0 = g.scalars()
    g.set_scalars(eta0, 1.1 * a0, 0.9 * b0)
    J0, dq0, lam0, ab0 = g.adjoint(20, 10, scale=True)
    spec = RunSpec.make(O.MODEL_LPHI4_CHI, N, 0.5, 1.0, 6, 20, ckpt_every=10, **SELF)
    q = torch.tensor(SELF["q"], dtype=torch.float64, requires_grad=True)
    st = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    sc = torch.tensor([1.1 * a0, 0.9 * b0], dtype=torch.float64, requires_grad=True)
    J = evolved_objective(q, st, spec, scale=sc)
    (2.0 * J).backward()
    assert abs(float(J.detach()) - J0) < 1e-14 * J0
    assert abs(float(q.grad) - 2.0 * dq0) < 1e-12 * abs(2.0 * dq0)
    assert np.abs(st.grad.numpy() - 2.0 * lam0).max() <= 1e-12 * np.abs(2.0 * lam0).max()
    assert np.allclose(sc.grad.numpy(), 2.0 * np.array(ab0), rtol=1e-12, atol=0)


def test_adjoint_128_fp32_checkpoints(P):
    """The C4 shape at reduced length: 128^3, FP32, VV4, 400 steps, checkpoints every 50."""
    g = P.Lattice(O.MODEL_LPHI4_CHI, 128, 0.2, 1.0, 1, P.make_params(precision=1, **dict(BASE, fluct_amp2=1e-4)))
    s0 = [g.get(f, w) for f in range(2) for w in (0, 1)]
    J, dq, lam = g.adjoint(400, 50)
    assert np.isfinite(J) and np.isfinite(dq) and np.all(np.isfinite(lam))
    assert np.abs(lam).max() > 0
    for (f, w), x in zip([(f, w) for f in range(2) for w in (0, 1)], s0):
        assert np.array_equal(g.get(f, w), x)


SELF = dict(BASE, expansion=O.EXP_SELF, fstar_over_mp=2.0)


@pytest.mark.parametrize("N,kw,alpha,nsteps,ckpt,obj", [
    (16, SELF, 1.0, 30, 10, None),
    (16, dict(SELF, integrator=O.VV2), 0.5, 25, 7, None),
    (24, dict(SELF, integrator=O.VV6), 1.0, 8, 3, None),
    (16, SELF, 1.0, 20, 6, (1, 1, 1.0, 2)),
])
def test_self_consistent_adjoint_matches_oracle(P, N, kw, alpha, nsteps, ckpt, obj):
    """Self-consistent expansion: the Friedmann kicks and the drift of a are in
    the reversed passes; dJ/da and dJ/db at the start come out as well."""
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, 0.5, alpha, 3, P.make_params(**kw))
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, 0.5, alpha, 3, O.make_params(**kw))
    s0 = [g.get(f, w) for f in range(2) for w in (0, 1)]
    sc0 = g.scalars()
    if obj is None:
        Jg, qg, lg, ab_g = g.adjoint(nsteps, ckpt, scale=True)
        Jo, qo, lo, ab_o = o.adjoint(nsteps, scale=True)
    else:
        f, w, dk, b = obj
        Jg, qg, lg, ab_g = g.adjoint(nsteps, ckpt, P.OBJ_SPECTRUM_BIN, f, w, dk, b, scale=True)
        Jo, qo, lo, ab_o = o.adjoint(nsteps, objective=1, field=f, what=w, dk_bin=dk, bin=b, scale=True)
    assert abs(Jg - Jo) < 1e-11 * abs(Jo)
    assert abs(qg - qo) < 1e-9 * abs(qo) + 1e-18, (qg, qo)
    assert nrel(lg, lo) < 1e-9
    for x, y in zip(ab_g, ab_o):
        assert abs(x - y) < 1e-9 * abs(y), (ab_g, ab_o)
    assert ab_o[1] != 0.0
    # fields, momenta, a, b and eta are back at the start, exactly
    assert g.scalars() == sc0
    for (f, w), x in zip([(f, w) for f in range(2) for w in (0, 1)], s0):
        assert np.array_equal(g.get(f, w), x)


def test_self_consistent_central_differences_fp64_32(P):
    """dJ/dq, dJ/da, dJ/db and a state direction against central differences
    of GPU forward runs (32^3, FP64, self-consistent expansion)."""
    N, kIR, n = 32, 0.5, 150
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 9, P.make_params(**SELF))
    s0 = [[g.get(f, w) for w in (0, 1)] for f in range(2)]
    sc0 = g.scalars()
    J, dq, lam, (da, db) = g.adjoint(n, 40, scale=True)

    def J_of(q, state, sc):
        h = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 9, P.make_params(**dict(SELF, q=q)))
        for f in range(2):
            for w in (0, 1):
                h.set(f, w, state[f][w])
        h.set_scalars(*sc)
        h.step(n)
        e = h.energies()
        h.close()
        return (e["EK"][1] + e["EG"][1]) / e["rho"]

    q0 = SELF["q"]
    assert abs(J_of(q0, s0, sc0) - J) < 1e-12 * J
    eps = 1e-3
    fd = (J_of(q0 + eps, s0, sc0) - J_of(q0 - eps, s0, sc0)) / (2 * eps)
    assert abs(dq - fd) < 1e-5 * abs(fd), (dq, fd)
    eta0, a0, b0 = sc0
    e = 1e-6
    fd_a = (J_of(q0, s0, (eta0, a0 + e, b0)) - J_of(q0, s0, (eta0, a0 - e, b0))) / (2 * e)
    fd_b = (J_of(q0, s0, (eta0, a0, b0 + e)) - J_of(q0, s0, (eta0, a0, b0 - e))) / (2 * e)
    assert abs(da - fd_a) < 1e-5 * abs(fd_a), (da, fd_a)
    assert abs(db - fd_b) < 1e-5 * abs(fd_b), (db, fd_b)
    rng = np.random.default_rng(4)
    v = [[rng.standard_normal((N, N, N)) * np.abs(s0[f][w]).max() for w in (0, 1)] for f in range(2)]
    e = 1e-7
    sp = [[s0[f][w] + e * v[f][w] for w in (0, 1)] for f in range(2)]
    sm = [[s0[f][w] - e * v[f][w] for w in (0, 1)] for f in range(2)]
    fd = (J_of(q0, sp, sc0) - J_of(q0, sm, sc0)) / (2 * e)
    ad = sum(float(np.sum(lam[f, w] * v[f][w])) for f in range(2) for w in (0, 1))
    assert abs(ad - fd) < 1e-5 * abs(fd), (ad, fd)


def test_self_consistent_fp32_close_to_fp64(P):
    r = {}
    for prec in (0, 1):
        g = P.Lattice(O.MODEL_LPHI4_CHI, 32, 0.5, 1.0, 2, P.make_params(precision=prec, **SELF))
        if prec:
            for f in range(2):
                for w in (0, 1):
                    g.set(f, w, r[0][4][f][w].astype(np.float32).astype(np.float64))
        s = [[g.get(f, w) for w in (0, 1)] for f in range(2)]
        J, dq, lam, ab = g.adjoint(100, 25, scale=True)
        r[prec] = (J, dq, lam, ab, s)
    assert abs(r[1][0] - r[0][0]) < 1e-5 * abs(r[0][0])
    assert abs(r[1][1] - r[0][1]) < 2e-3 * abs(r[0][1])
    assert nrel(r[1][2], r[0][2]) < 2e-3
    for k in range(2):
        assert abs(r[1][3][k] - r[0][3][k]) < 2e-3 * abs(r[0][3][k])


def test_unsupported(P):
    g = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**dict(SELF, b0_mode=1)))
    J, dq, lam = g.adjoint(2, 1)
    with pytest.raises(P.ClError) as e:
        g.ic_amplitude_grad(lam)
    assert e.value.status == P.CL_EUNSUPPORTED
    g1 = P.Lattice(O.MODEL_LPHI4, 16, 0.5, 1.0, 1, P.make_params(**dict(BASE, phi0=[1.0])))
    with pytest.raises(P.ClError) as e:
        g1.adjoint(2, 1)
    assert e.value.status == P.CL_EINVAL
    g2 = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**BASE))
    with pytest.raises(P.ClError):
        g2.adjoint(2, 0)
    gu = P.Lattice(O.MODEL_U1_HIGGS, 16, 0.5, 1.0, 1,
                   P.make_params(dt=0.01, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, phi0=[1.0, 1.0],
                                 fluct_amp2=1e-2, expansion=O.EXP_OFF))
    with pytest.raises(P.ClError) as e:
        gu.adjoint(2, 1)
    assert e.value.status == P.CL_EUNSUPPORTED
