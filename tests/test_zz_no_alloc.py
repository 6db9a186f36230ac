"""cl_volume_averages_noalloc: volume averages for callers that cannot
allocate device memory (fixed device budgets, foreign memory pools, loops that
must not synchronise).  Its partial sums live in a static device array instead
of context scratch.  Checked through the C ABI against cl_energies on the same
state, on calls in a row: a 96^3 call (more blocks than the array has rows, so
the grid-stride loop runs) followed by a 16^3 call, which writes fewer rows than
the first left behind; the one-field model; and a NaN planted on the host."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}   # FP64 / FP32 storage, as in the other parity tests


def device_state(P, torch, lat, nf, precision):
    dt = torch.float32 if precision == P.FP32 else torch.float64
    return [torch.from_numpy(lat.get(f, w).reshape(-1)).to("cuda", dt).contiguous()
            for f in range(nf) for w in range(2)]


def run_noalloc(P, torch, dev, model, N, kIR, a, q, precision):
    ptrs = (ctypes.c_void_p * len(dev))(*[t.data_ptr() for t in dev])
    out = torch.full((16,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = P.lib().cl_volume_averages_noalloc(model, N, kIR, a, q, precision, ptrs,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == P.CL_OK
    torch.cuda.synchronize()
    return out.cpu().numpy()


def compare(o, e, nf, tol):
    pairs = [(o[0:2], e["EK"][:2]), (o[2:4], e["EG"][:2]), (o[4:6], e["EV"][:2]),
             (o[6:8], e["mean_phi"][:2]), (o[8:10], e["mean_phi2"][:2]),
             (o[10:12], e["mean_pi"][:2]), (o[12:14], e["mean_pi2"][:2])]
    for got, ref in pairs:
        for g, r in zip(got[:nf], ref[:nf]):
            # <pi> is a mean of values of either sign: compared against the scale of <pi^2>^(1/2)
            scale = max(abs(r), 1e-300)
            assert abs(g - r) <= tol * scale or abs(g - r) <= tol * np.sqrt(max(e["mean_pi2"])), (g, r)
        for g in got[nf:]:
            assert g == 0.0
    assert abs(o[14] - e["rho"]) <= tol * abs(e["rho"])
    assert o[15] == 0.0


def lattice(P, model, N, kIR, q, precision, seed):
    kw = dict(dt=0.005, integrator=P.VV4, q=q, phi0=[1.0, 0.0], fluct_amp2=1e-2,
              expansion=P.EXP_SELF, fstar_over_mp=0.5, precision=precision)
    return P.Lattice(model, N, kIR, 1.0, seed, P.make_params(**kw))


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_cl_energies_twice(precision):
    torch = pytest.importorskip("torch")
    import paper_2102_01031_gb300 as P
    P.build()
    model, kIR, q = P.MODEL_LPHI4_CHI, 0.5, 100.0
    for call, (N, steps) in enumerate(((96, 20), (16, 30))):
        lat = lattice(P, model, N, kIR, q, precision, 5 + call)
        lat.step(steps)
        e = lat.energies()
        _, a, _ = lat.scalars()
        dev = device_state(P, torch, lat, 2, precision)
        o = run_noalloc(P, torch, dev, model, N, kIR, a, q, precision)
        compare(o, e, 2, TOL[precision])
        lat.close()


def test_noalloc_one_field_model_and_nonfinite_count():
    torch = pytest.importorskip("torch")
    import paper_2102_01031_gb300 as P
    P.build()
    N, kIR = 32, 0.5
    lat = lattice(P, P.MODEL_LPHI4, N, kIR, 0.0, P.FP64, 3)
    lat.step(15)
    e = lat.energies()
    _, a, _ = lat.scalars()
    dev = device_state(P, torch, lat, 1, P.FP64)
    o = run_noalloc(P, torch, dev, P.MODEL_LPHI4, N, kIR, a, 0.0, P.FP64)
    compare(o, e, 1, TOL[0])
    dev[1][1234] = float("nan")      # one non-finite momentum, planted on the host side of the call
    o = run_noalloc(P, torch, dev, P.MODEL_LPHI4, N, kIR, a, 0.0, P.FP64)
    assert o[15] == 1.0
    lat.close()


def test_noalloc_rejects_sizes_beyond_limit():
    import paper_2102_01031_gb300 as P
    P.build()
    ptrs = (ctypes.c_void_p * 4)(1, 1, 1, 1)
    rc = P.lib().cl_volume_averages_noalloc(P.MODEL_LPHI4_CHI, 1024, 0.5, 1.0, 1.0, P.FP32, ptrs,
                                            ctypes.c_void_p(1), None)
    assert rc == P.CL_EINVAL
