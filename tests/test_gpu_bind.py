"""Caller-owned state memory (cl_bind_buffers, cl_state_buffer): the library
owns the device state unless the caller binds two buffers of its own (torch
CUDA tensors here).  Binding only moves memory, so a bound lattice must evolve
bit for bit like an unbound twin started from the same seed, the bound tensors
must hold exactly what cl_get_state returns, and a binding the call refuses
must change nothing.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALAR = dict(dt=0.005, integrator=4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-2, fstar_over_mp=0.5)
U1 = dict(dt=0.01, integrator=0, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0, phi0=[1.0, 1.0],
          fluct_amp2=1e-2, fstar_over_mp=0.5)
SU2 = dict(dt=0.01, integrator=0, lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
           phi0=[0.5] * 4, dphi0=[0.1] * 4, fluct_amp2=1e-2, fstar_over_mp=0.5)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def arrays(P, g, model):
    """Every state array of lattice g, in storage order, as float64."""
    if model in (P.MODEL_SU2U1_HIGGS, P.MODEL_LPHI4_SU2U1):
        n = {P.MODEL_SU2U1_HIGGS: 35, P.MODEL_LPHI4_SU2U1: 41}[model]
        return [g.get_array(a) for a in range(n)]
    return [g.get(f, w) for f in range(g.nfields()) for w in (0, 1)]


def buffers(P, g, fill=np.nan):
    nb = g.state_bytes()
    dt = torch.float32 if g.params.precision == P.FP32 else torch.float64
    esz = 4 if dt == torch.float32 else 8
    return [torch.full((nb // esz,), fill, dtype=dt, device="cuda") for _ in range(2)]


@pytest.mark.parametrize("model,N,prec,kw,exp", [
    ("MODEL_LPHI4_CHI", 32, "FP32", SCALAR, "EXP_SELF"),
    ("MODEL_LPHI4_CHI", 24, "FP64", SCALAR, "EXP_SELF"),
    ("MODEL_U1_HIGGS", 32, "FP32", U1, "EXP_OFF"),
    ("MODEL_U1_HIGGS", 24, "FP64", U1, "EXP_SELF"),
    ("MODEL_SU2U1_HIGGS", 32, "FP32", SU2, "EXP_OFF"),
])
def test_bound_lattice_evolves_like_its_twin(P, model, N, prec, kw, exp):
    m, pr = getattr(P, model), getattr(P, prec)
    mk = lambda: P.Lattice(m, N, 0.5, 1.0, 7, P.make_params(precision=pr, **dict(kw, expansion=getattr(P, exp))))
    a, b = mk(), mk()
    a.step(3)
    b.step(3)
    t = buffers(P, b)
    b.bind_buffers(t[0], t[1])
    a.step(5)
    b.step(5)
    a.sync()
    b.sync()
    A, B = arrays(P, a, m), arrays(P, b, m)
    for k, (x, y) in enumerate(zip(A, B)):
        assert np.array_equal(x, y), k
    # the bound tensor that holds the state is the state, array a at a N^3 values
    torch.cuda.synchronize()
    view = t[b.state_buffer()][: len(B) * N ** 3].view(len(B), N, N, N).double().cpu().numpy()
    for k, y in enumerate(B):
        assert np.array_equal(view[k], y.reshape(N, N, N)), k
    # the state moves back into the lattice's own memory and stepping goes on alike
    b.bind_buffers(None, None)
    del t
    torch.cuda.synchronize()
    a.step(2)
    b.step(2)
    ea, eb = a.energies(), b.energies()
    assert ea["a"] == eb["a"] and ea["rho"] == eb["rho"]
    for k, (x, y) in enumerate(zip(arrays(P, a, m), arrays(P, b, m))):
        assert np.array_equal(x, y), k
    a.close()
    b.close()


def test_refused_bindings_change_nothing(P):
    g = P.Lattice(P.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, P.make_params(precision=P.FP32, **SCALAR))
    g.step(2)
    g.sync()
    before = arrays(P, g, P.MODEL_LPHI4_CHI)
    t = buffers(P, g)
    nb = g.state_bytes()
    wide = torch.zeros(nb // 4 + 64, dtype=torch.float32, device="cuda")
    bad = [
        (wide[1: 1 + nb // 4], t[1]),                       # 4 bytes off the alignment
        (t[0], t[0]),                                       # the two overlap
        (t[0][: nb // 4 - 64], t[1][: nb // 4 - 64]),       # too small
        (torch.zeros(nb // 4, dtype=torch.float32), t[1]),  # host memory
    ]
    for x, y in bad:
        with pytest.raises(P.ClError) as e:
            g.bind_buffers(x, y)
        assert e.value.status == 1  # CL_EINVAL
    with pytest.raises(P.ClError) as e:
        g.bind_buffers(t[0], t[1], lat=1)  # no lattice 1
    assert e.value.status == 1
    after = arrays(P, g, P.MODEL_LPHI4_CHI)
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    # unbinding a lattice that is not bound is a no-op
    g.bind_buffers(None, None)
    g.step(1)
    assert np.isfinite(g.energies()["rho"])
    g.close()


def test_bound_ensemble_member_and_adjoint(P):
    mk = lambda: P.Ensemble(P.MODEL_LPHI4_CHI, [16, 24], [0.5, 0.5], 1.0, [3, 4],
                            P.make_params(precision=P.FP32, **dict(SCALAR, expansion=P.EXP_SELF)))
    a, b = mk(), mk()
    a.step(2)
    b.step(2)
    nb = 4 * 24 ** 3 * 4
    t = [torch.zeros(nb // 4, dtype=torch.float32, device="cuda") for _ in range(2)]
    b.bind_buffers(t[0], t[1], lat=1)
    a.step(4)
    b.step(4)
    for f in range(2):
        for w in (0, 1):
            assert np.array_equal(a.get(1, f, w), b.get(1, f, w))
            assert np.array_equal(a.get(0, f, w), b.get(0, f, w))
    a.close()
    b.close()
    # the adjoint sweep reads the state through its own copy of the addresses
    kw = dict(SCALAR, expansion=P.EXP_OFF)
    g = P.Lattice(P.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, P.make_params(precision=P.FP64, **kw))
    h = P.Lattice(P.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, P.make_params(precision=P.FP64, **kw))
    g.step(2)
    h.step(2)
    Jg0 = g.adjoint(8, 4)[0]
    Jh0 = h.adjoint(8, 4)[0]
    assert Jg0 == Jh0
    t = buffers(P, h)
    h.bind_buffers(t[0], t[1])
    g.step(3)
    h.step(3)
    Jg, qg, lg = g.adjoint(10, 4)
    Jh, qh, lh = h.adjoint(10, 4)
    assert Jg == Jh and qg == qh and np.array_equal(lg, lh)
    g.close()
    h.close()
