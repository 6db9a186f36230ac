"""The bounded device waits of the persistent passes run out and report
CL_ETIMEOUT without a GPU fault: one thread waits, with a 0.2 s limit, on a
counter that nothing sets and on an mbarrier that gets no arrival
(cl_selftest_wait); the same waits return at once when satisfied, and the
device stays usable afterwards (a lattice steps and matches the oracle)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

LIMIT_NS = 200_000_000


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_runs_out_and_reports(P, kind):
    st, ns = P.selftest_wait(kind, satisfied=False, limit_ns=LIMIT_NS)
    assert st == P.CL_ETIMEOUT
    assert LIMIT_NS <= ns < 10 * LIMIT_NS, ns
    st, ns = P.selftest_wait(kind, satisfied=True, limit_ns=LIMIT_NS)
    assert st == P.CL_OK and ns < LIMIT_NS // 2, ns


def test_wait_arguments_and_device_afterwards(P):
    for kind, limit in ((2, LIMIT_NS), (0, 0), (1, 20_000_000_000)):
        with pytest.raises(P.ClError) as e:
            P.selftest_wait(kind, satisfied=False, limit_ns=limit)
        assert e.value.status == P.CL_EINVAL
    kw = dict(dt=0.01, integrator=O.VV2, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4)
    g = P.Lattice(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, P.make_params(**kw))
    o = O.Oracle(O.MODEL_LPHI4_CHI, 16, 0.5, 1.0, 1, O.make_params(**kw))
    g.step(5)
    o.step(5)
    for f in range(2):
        d = np.abs(g.get(f, 0) - o.get(f, 0)).max() / np.abs(o.get(f, 0)).max()
        assert d < 1e-10, (f, d)
