"""The device generator of the initial conditions, bit for bit.

The vacuum fluctuations of Sec. 3.5.1 (eqs. fpr_influct, QuantumFlucts2) are
drawn from Philox4x32-10 (Salmon et al., SC'11) keyed by the seed.  Generator
output is integer work, so the GPU's words and the 53-bit deviates made from
them must equal the oracle's exactly: checked through cl_philox_draws (the same
device code cl_init uses) on the published known answers, on 10^4 random
counters and keys, and on 10^4 sampled draw pairs of the initial conditions
(Fourier index, component, draw, seed) against the oracle's own draw pairs.
"""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(w, 16) for w in line.split()])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_device_philox_known_answers(P):
    r = kat_rows()
    assert len(r) == 3
    words, u = P.philox_draws(0, r[:, 0:4], r[:, 4:6])
    assert np.array_equal(words, r[:, 6:10])
    for i in range(len(r)):
        assert u[i, 0] == O.u01(int(words[i, 0]), int(words[i, 1]))
        assert u[i, 1] == O.u01(int(words[i, 2]), int(words[i, 3]))


def test_device_philox_random_counters_match_oracle(P):
    rng = np.random.default_rng(2021)
    n = 10000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # edge words: all zero, all one, single high bits
    ctr[:4] = [[0, 0, 0, 0], [0xffffffff] * 4, [0x80000000, 0, 0, 1], [1, 0x80000000, 0xffffffff, 0]]
    key[:4] = [[0, 0], [0xffffffff, 0xffffffff], [0x80000000, 1], [0, 0x80000000]]
    words, u = P.philox_draws(0, ctr, key)
    ref = np.array([O.philox4x32_10([int(x) for x in ctr[i]], [int(x) for x in key[i]]) for i in range(n)],
                   dtype=np.uint64).astype(np.uint32)
    assert np.array_equal(words, ref)
    uref = np.array([[O.u01(int(w[0]), int(w[1])), O.u01(int(w[2]), int(w[3]))] for w in ref])
    assert np.array_equal(u, uref)
    assert u.min() > 0.0 and u.max() <= 1.0


def test_device_ic_draw_pairs_match_oracle(P):
    rng = np.random.default_rng(7)
    n = 10000
    seeds = [1, 2, 7, 0xdeadbeefcafef00d, 2 ** 64 - 1]
    idx = rng.integers(0, 512 ** 3, size=n, dtype=np.int64)
    idx[:3] = [0, 1, 512 ** 3 - 1]
    f = rng.integers(0, 4, size=n).astype(np.int32)
    j = rng.integers(0, 2, size=n).astype(np.int32)
    for seed in seeds:
        ctr = np.zeros((n, 4), dtype=np.uint32)
        ctr[:, 0] = idx.astype(np.uint32)
        ctr[:, 1] = f.astype(np.uint32)
        ctr[:, 2] = j.astype(np.uint32)
        key = np.zeros((n, 2), dtype=np.uint32)
        key[:, 0] = seed & 0xffffffff
        key[:, 1] = seed >> 32
        words, u = P.philox_draws(1, ctr, key)
        assert not words.any()
        assert np.array_equal(u, O.draw_pairs(seed, idx, f, j)), hex(seed)


def test_device_philox_rejects_bad_arguments(P):
    with pytest.raises(P.ClError) as e:
        P.philox_draws(2, np.zeros((1, 4)), np.zeros((1, 2)))
    assert e.value.status == P.CL_EINVAL
    w, u = P.philox_draws(0, np.zeros((0, 4)), np.zeros((0, 2)))
    assert w.shape == (0, 4) and u.shape == (0, 2)
