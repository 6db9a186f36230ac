"""The 27- and 81-stage compositions (VV8, VV10) on the GPU against the oracle:
the same DK pass, more passes per step (the pass plan itself is checked on the
CPU in test_pass_weights_cpu.py, the compositions' orders in the oracle pins)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

C2S = dict(dt=0.005, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4, expansion=O.EXP_SELF, fstar_over_mp=0.5)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def nrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("integ", [O.VV8, O.VV10])
def test_high_order_compositions_match_oracle(P, integ):
    kw = dict(C2S, integrator=integ)
    g = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, P.make_params(**kw))
    o = O.Oracle(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 3, O.make_params(**kw))
    g.step(10)
    o.step(10)
    for f in range(2):
        for w in (0, 1):
            e = nrel(g.get(f, w), o.get(f, w))
            assert e < 1e-10, (f, w, e)
    eg, eo = g.energies(), o.energies()
    for k in ("a", "b", "eta", "rho"):
        assert abs(eg[k] - eo[k]) <= 1e-10 * max(abs(eo[k]), 1e-300), (k, eg[k], eo[k])
    assert abs(eg["eta"] - 10 * 0.005) < 1e-12
