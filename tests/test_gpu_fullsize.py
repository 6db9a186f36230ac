"""Parity against the oracle at the sizes the benchmark rows run, not only by
properties:

  * U(1) Abelian-Higgs at 256^3 (Sec. 4.4.1 initial conditions): sampled
    Fourier modes of the charged field and its momentum against the oracle's
    one-by-one values, and of the link momenta against the oracle's Gauss-law
    inversion of the same charged field (eq. GaugeCurrentFluc on the lattice);
    then two leapfrog steps of the FP32 pass from the GPU's FP32 state against
    the oracle started from the same values (normwise 1e-5 per array, the FP32
    tolerance of the other parity tests; averages 1e-6).
  * The SU(2) x U(1) doublet at 256^3, and the lphi4SU2U1 model (with the
    singlet and the U(1)-charged scalar): one leapfrog step of the FP32 pass
    against the oracle from the same state (normwise 1e-5 per array).
  * The adjoint at 128^3 in FP32 with checkpoints every 50 of 400 VV4 steps,
    against the FP64 GPU adjoint (itself held to the oracle's discrete adjoint
    at 1e-9) from the same FP32-rounded start: J within 1e-5, dJ/dq and
    dJ/d(state) within 2e-3 (normwise), the bound the 32^3 FP32 adjoint test
    states for the rounding of the forward and the reversed passes.
"""
import numpy as np
import pytest

import oracle as O
from tests.parity import nrel

pytestmark = pytest.mark.gpu

C3 = dict(dt=0.01, integrator=O.LF, lam=1.0, v=1.0, gQ=0.5, fstar_over_omegastar=1.0,
          phi0=[1.0, 1.0], fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5)
SU2 = dict(dt=0.01, integrator=O.LF, lam=1.0, v=0.5, gQ=0.6, gQB=0.8, fstar_over_omegastar=1.3,
           phi0=[0.5] * 4, dphi0=[0.1] * 4, fluct_amp2=1e-2, expansion=O.EXP_OFF, fstar_over_mp=0.5)
BASE = dict(dt=0.005, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4,
            expansion=O.EXP_OFF, fstar_over_mp=0.5)


@pytest.fixture(scope="module")
def P():
    import paper_2102_01031_gb300 as P
    P.build()
    P.lib()
    return P


def sampled_indices(N, n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.integers(0, N ** 3, n), [1, N - 1, N * N, N ** 3 - 1, N // 2, 5 * N * N + 3]])


def test_u1_256_initial_conditions_sampled_modes(P):
    N, kIR = 256, 0.1
    g = P.Lattice(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, P.make_params(precision=P.FP64, **C3))
    idx = sampled_indices(N, 400, 3)
    f, gg = O.ic_sample(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, O.make_params(**C3), idx)
    for c in (0, 1):
        F = np.fft.fftn(g.get(c, 0) - C3["phi0"][c]).reshape(-1)[idx]
        G = np.fft.fftn(g.get(c, 1)).reshape(-1)[idx]
        assert np.abs(F - f[:, c]).max() < 1e-9 * np.abs(f[:, c]).max(), c
        assert np.abs(G - gg[:, c]).max() < 1e-9 * np.abs(gg[:, c]).max(), c
    # link momenta: the oracle's Gauss-law inversion of the GPU's charged field
    o = O.Oracle(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, O.make_params(**dict(C3, fluct_amp2=0.0)))
    for c in (0, 1):
        for w in (0, 1):
            o.set(c, w, g.get(c, w))
    ref = o.gauss_modes(idx)
    del o
    for d in range(3):
        E = np.fft.fftn(g.get(2 + d, 1)).reshape(-1)[idx]
        assert np.abs(E - ref[:, d]).max() < 1e-9 * np.abs(ref[:, d]).max(), d
        assert np.abs(g.get(2 + d, 0)).max() == 0.0   # the links start at zero
    g.close()


def test_u1_256_fp32_leapfrog_matches_oracle(P):
    N, kIR = 256, 0.1
    g = P.Lattice(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, P.make_params(precision=P.FP32, **C3))
    o = O.Oracle(O.MODEL_U1_HIGGS, N, kIR, 1.0, 1, O.make_params(**dict(C3, fluct_amp2=0.0)))
    for f in range(5):
        for w in (0, 1):
            o.set(f, w, g.get(f, w))
    o.set_scalars(*g.scalars())
    g.step(2)
    o.step(2)
    for f in range(5):
        for w in (0, 1):
            ref = o.get(f, w)
            e = nrel(g.get(f, w), ref)
            print("U(1) 256^3 FP32, 2 LF steps: array (%d, %d) normwise %.3g" % (f, w, e))
            assert e < 1e-5, (f, w, e)
    eg, eo = g.energies(), o.energies()
    for k in ("EKA", "EGA", "rho"):
        assert abs(eg[k] - eo[k]) <= 1e-6 * abs(eo[k]), (k, eg[k], eo[k])
    for k in ("EK", "EG", "EV"):
        assert abs(eg[k][0] - eo[k][0]) <= 1e-6 * abs(eo[k][0]), (k, eg[k][0], eo[k][0])
    g.close()


def test_doublet_256_fp32_leapfrog_matches_oracle(P):
    N, kIR, NA = 256, 0.1, 35
    g = P.Lattice(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 1, P.make_params(precision=P.FP32, **SU2))
    o = O.Oracle(O.MODEL_SU2U1_HIGGS, N, kIR, 1.0, 1, O.make_params(**dict(SU2, fluct_amp2=0.0)))
    for a in range(NA):
        o.set_array(a, g.get_array(a))
    o.set_scalars(*g.scalars())
    g.step(1)
    o.step(1)
    worst = 0.0
    for a in range(NA):
        ref = o.get_array(a)
        got = g.get_array(a)
        if np.abs(ref).max() == 0.0:
            assert np.abs(got).max() == 0.0, a
            continue
        e = nrel(got, ref)
        worst = max(worst, e)
        assert e < 1e-5, (a, e)
    print("doublet 256^3 FP32, 1 LF step: worst array normwise %.3g" % worst)
    eg, eo = g.energies(), o.energies()
    for k in ("EKA", "EGA", "EKB", "EGB", "rho"):
        assert abs(eg[k] - eo[k]) <= 1e-5 * abs(eo[k]), (k, eg[k], eo[k])
    g.close()


def test_lphi4su2u1_256_fp32_leapfrog_matches_oracle(P):
    """The lphi4SU2U1 model at 256^3 (singlet, charged scalar and doublet, both
    gauge fields): one leapfrog step of the FP32 pass against the oracle from
    the same state (normwise 1e-5 per array)."""
    N, kIR, NA = 256, 0.1, 41
    kw = dict(SU2, v=0.0, qG=1.5, qH=0.8, Qc=0.7)
    g = P.Lattice(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 1, P.make_params(precision=P.FP32, **kw))
    o = O.Oracle(O.MODEL_LPHI4_SU2U1, N, kIR, 1.0, 1, O.make_params(**dict(kw, fluct_amp2=0.0)))
    for a in range(NA):
        o.set_array(a, g.get_array(a))
    o.set_scalars(*g.scalars())
    g.step(1)
    o.step(1)
    worst = 0.0
    for a in range(NA):
        ref = o.get_array(a)
        got = g.get_array(a)
        if np.abs(ref).max() == 0.0:
            assert np.abs(got).max() == 0.0, a
            continue
        e = nrel(got, ref)
        worst = max(worst, e)
        assert e < 1e-5, (a, e)
    print("lphi4SU2U1 256^3 FP32, 1 LF step: worst array normwise %.3g" % worst)
    eg, eo = g.energies(), o.energies()
    for k in ("EK", "EG", "EV"):
        for i in range(3):
            assert abs(eg[k][i] - eo[k][i]) <= 1e-5 * abs(eo[k][i]), (k, i, eg[k][i], eo[k][i])
    g.close()


@pytest.mark.parametrize("expansion", [O.EXP_OFF, O.EXP_SELF])
def test_adjoint_128_fp32_against_fp64(P, expansion):
    kw = dict(BASE, expansion=expansion, fstar_over_mp=0.5 if expansion == O.EXP_OFF else 2.0)
    r = {}
    for prec in (P.FP32, P.FP64):
        g = P.Lattice(O.MODEL_LPHI4_CHI, 128, 0.2, 1.0, 1, P.make_params(precision=prec, **kw))
        if prec == P.FP64:   # the FP32 run's start, FP32-rounded, and its scalars
            for f in range(2):
                for w in (0, 1):
                    g.set(f, w, r[P.FP32][3][f][w])
            g.set_scalars(*r[P.FP32][4])
        s = [[g.get(f, w) for w in (0, 1)] for f in range(2)]
        sc = g.scalars()
        J, dq, lam = g.adjoint(400, 50)
        r[prec] = (J, dq, lam, s, sc)
        g.close()
    J32, dq32, l32 = r[P.FP32][:3]
    J64, dq64, l64 = r[P.FP64][:3]
    eJ, eq, el = abs(J32 - J64) / abs(J64), abs(dq32 - dq64) / abs(dq64), nrel(l32, l64)
    print("adjoint 128^3 400 steps, expansion %d: J %.3g, dJ/dq %.3g, dJ/dstate %.3g" % (expansion, eJ, eq, el))
    assert eJ < 1e-5
    assert eq < 2e-3
    assert el < 2e-3


C2S = dict(dt=0.005, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-4,
           expansion=O.EXP_SELF, fstar_over_mp=0.5)


def test_c2_512_initial_conditions_sampled_modes(P):
    """C2 at its larger size, 512^3 (two fields, kIR = 0.1): Fourier modes of the
    GPU's FP64 initial fields and momenta against the oracle's one-by-one values."""
    N, kIR = 512, 0.1
    g = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, P.make_params(precision=P.FP64, **C2S))
    idx = sampled_indices(N, 300, 11)
    f, gg = O.ic_sample(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, O.make_params(**C2S), idx)
    for fld, off in ((0, 1.0), (1, 0.0)):
        F = np.fft.fftn(g.get(fld, 0) - off).reshape(-1)[idx]
        assert np.abs(F - f[:, fld]).max() < 1e-9 * np.abs(f[:, fld]).max(), fld
        G = np.fft.fftn(g.get(fld, 1)).reshape(-1)[idx]
        assert np.abs(G - gg[:, fld]).max() < 1e-9 * np.abs(gg[:, fld]).max(), fld
    g.close()


def test_c2_512_fp32_against_fp64(P):
    """C2 at 512^3 in the benchmark's launch configuration (FP32 storage, VV4,
    self-consistent expansion) against the FP64 path (the same kernels, held to the
    oracle at smaller sizes) from the same FP32-rounded start: four steps, every
    array within 1e-5 normwise, the energies within 1e-6, the Hubble violation no
    larger than 1.05 x the FP64 run's plus the FP32 rounding of the constraint."""
    N, kIR = 512, 0.1
    g64 = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, P.make_params(precision=P.FP64, **C2S))
    g32 = P.Lattice(O.MODEL_LPHI4_CHI, N, kIR, 1.0, 1, P.make_params(precision=P.FP32, **C2S))
    for f in range(2):
        for w in (0, 1):
            x = g64.get(f, w).astype(np.float32).astype(np.float64)
            g64.set(f, w, x)
            g32.set(f, w, x)
    sc = g64.scalars()
    g32.set_scalars(*sc)
    g64.set_scalars(*sc)
    for g in (g64, g32):
        g.step(4)
    for f in range(2):
        for w in (0, 1):
            e = nrel(g32.get(f, w), g64.get(f, w))
            print("C2 512^3 FP32 vs FP64, 4 VV4 steps: field %d %s normwise %.3g" % (f, "pi" if w else "phi", e))
            assert e < 1e-5, (f, w, e)
    e32, e64 = g32.energies(), g64.energies()
    for k in ("EK", "EG", "EV"):
        for i in range(2):
            if e64[k][i] != 0.0:
                assert abs(e32[k][i] - e64[k][i]) <= 1e-6 * abs(e64[k][i]), (k, i, e32[k][i], e64[k][i])
    for k in ("a", "b", "rho"):
        assert abs(e32[k] - e64[k]) <= 1e-6 * abs(e64[k]), (k, e32[k], e64[k])
    assert abs(e32["hubble_viol"]) <= 1.05 * abs(e64["hubble_viol"]) + 1e-6, (e32["hubble_viol"], e64["hubble_viol"])
    g32.close()
    g64.close()
