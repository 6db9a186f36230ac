"""CPU check of the library's pass plan (cl_pass_weights: host arithmetic, no GPU):
the fused kick-drift passes that cl_step_h launches are the oracle's unfused
step -- kick d/2, drift d, kick d/2 for every substep d of the integrator's
composition (pinned in test_oracle_pins.py) -- with adjacent half kicks merged
("first same as last", Sec. 5.1), the stream carried across calls, and one
closing half kick."""
import os
import shutil

import numpy as np
import pytest

import oracle as O


@pytest.fixture(scope="module")
def P():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


INTEGRATORS = [O.LF, O.VV2, O.VV4, O.VV6, O.VV8, O.VV10]


@pytest.mark.parametrize("integ", INTEGRATORS)
def test_passes_are_the_merged_unfused_step(P, oracle_mod, integ):
    h, n = 0.013, 3
    W = P.pass_weights(integ, h, [n])
    d = np.tile(O.schedule(integ, h), n)          # the oracle's drifts, step after step
    assert W.shape == (len(d) + 1, 4)
    ck, wout, win, dnext = W.T
    # one drift per pass, the oracle's, bit for bit; the closing pass drifts 0
    assert np.array_equal(dnext[:-1], d) and dnext[-1] == 0.0
    # every kick is the kick-out of the previous drift plus the kick-in of the next
    assert np.array_equal(win[:-1], 0.5 * d) and win[-1] == 0.0
    assert wout[0] == 0.0 and np.array_equal(wout[1:], 0.5 * d)
    assert np.array_equal(ck, wout + win)
    # the kicks and the drifts each add up to the n steps' time
    assert abs(ck.sum() - n * h) < 1e-15 and abs(dnext.sum() - n * h) < 1e-15


@pytest.mark.parametrize("integ", [O.VV4, O.LF])
def test_stream_carries_across_calls(P, oracle_mod, integ):
    h = 0.02
    one = P.pass_weights(integ, h, [5])
    split = P.pass_weights(integ, h, [2, 0, 3])
    assert np.array_equal(one, split)
    # a negative step runs the same plan backwards in time
    back = P.pass_weights(integ, -h, [5])
    assert np.array_equal(back, -one)


def test_pass_weights_arguments(P):
    assert P.pass_weights(O.VV2, 0.1, []).shape == (0, 4)        # nothing launched, nothing to close
    assert P.pass_weights(O.VV2, 0.1, [0, 0]).shape == (0, 4)
    assert P.pass_weights(O.VV10, 0.1, [2]).shape == (163, 4)    # 2 x 81 substeps + the closing kick
    for bad in ((3, 0.1, [1]), (O.VV2, float("nan"), [1]), (O.VV2, 0.1, [-1])):
        with pytest.raises(P.ClError) as e:
            P.pass_weights(*bad)
        assert e.value.status == P.CL_EINVAL
