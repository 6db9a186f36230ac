"""Pins of the oracle's discrete adjoint (gradient of a final observable with
respect to the coupling q, the initial state and the initial mode
amplitudes), against central finite differences of the oracle's own forward
run.  The objective is evaluated from the forward energies / spectrum, not
from the adjoint's seed, so a wrong seed, a dropped term, a wrong sign or a
transposed Hessian fails here.
"""
import numpy as np
import pytest

import oracle as O

BASE = dict(dt=0.01, integrator=O.VV4, q=100.0, phi0=[1.0, 0.0], fluct_amp2=1e-2,
            expansion=O.EXP_OFF, fstar_over_mp=0.5)


def chi_fraction(o):
    e = o.energies()
    return (e["EK"][1] + e["EG"][1]) / e["rho"]


def run_J(model, N, kIR, seed, kw, state, nsteps, objective=0, spec=None):
    o = O.Oracle(model, N, kIR, 1.0, seed, O.make_params(**kw))
    for f in range(len(state)):
        for w in (0, 1):
            o.set(f, w, state[f][w])
    o.step(nsteps)
    if objective == 0:
        return chi_fraction(o)
    field, what, dk, b = spec
    return o.spectrum(field, what, dk)[1][b]


def state_of(o, nf):
    return [[o.get(f, w).copy() for w in (0, 1)] for f in range(nf)]


@pytest.mark.parametrize("kw", [BASE, dict(BASE, integrator=O.VV2),
                                dict(BASE, expansion=O.EXP_FIXED, omega_eos=1.0 / 3.0, H0=0.4)])
def test_dJ_dq_matches_central_difference(oracle_mod, kw):
    N, kIR, seed, n = 8, 1.0, 3, 15
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, O.make_params(**kw))
    s0 = state_of(o, 2)
    J, dq, lam = o.adjoint(n)
    assert abs(J - run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, kw, s0, n)) < 1e-14
    eps = 1e-3
    Jp = run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, dict(kw, q=kw["q"] + eps), s0, n)
    Jm = run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, dict(kw, q=kw["q"] - eps), s0, n)
    fd = (Jp - Jm) / (2 * eps)
    assert abs(dq - fd) < 1e-6 * abs(fd) + 1e-12, (dq, fd)


@pytest.mark.parametrize("objective,spec", [(0, None), (1, (1, 0, 1.0, 2)), (1, (0, 1, 1.0, 3))])
def test_state_gradient_matches_directional_difference(oracle_mod, objective, spec):
    N, kIR, seed, n = 8, 1.0, 4, 12
    kw = BASE
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, O.make_params(**kw))
    s0 = state_of(o, 2)
    if objective == 0:
        J, dq, lam = o.adjoint(n)
    else:
        J, dq, lam = o.adjoint(n, objective=1, field=spec[0], what=spec[1], dk_bin=spec[2], bin=spec[3])
    # the state is left as it was
    for f in range(2):
        for w in (0, 1):
            assert np.array_equal(o.get(f, w), s0[f][w])
    rng = np.random.default_rng(5)
    for trial in range(3):
        v = [[rng.standard_normal((N, N, N)) for w in (0, 1)] for f in range(2)]
        if trial == 1:   # momenta only
            v = [[0 * v[f][0], v[f][1]] for f in range(2)]
        eps = 1e-6
        sp = [[s0[f][w] + eps * v[f][w] for w in (0, 1)] for f in range(2)]
        sm = [[s0[f][w] - eps * v[f][w] for w in (0, 1)] for f in range(2)]
        fd = (run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, kw, sp, n, objective, spec) -
              run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, kw, sm, n, objective, spec)) / (2 * eps)
        ad = sum(float(np.sum(lam[f, w] * v[f][w])) for f in range(2) for w in (0, 1))
        assert abs(ad - fd) < 1e-6 * max(abs(fd), 1e-30) + 1e-13, (trial, ad, fd)


def test_explicit_q_term_of_the_objective(oracle_mod):
    """Zero steps: dJ/dq is the explicit dependence of the final energy fraction on q."""
    N, kIR, seed = 8, 1.0, 6
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, O.make_params(**BASE))
    s0 = state_of(o, 2)
    J, dq, lam = o.adjoint(0)
    eps = 1e-4
    fd = (run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, dict(BASE, q=BASE["q"] + eps), s0, 0) -
          run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, dict(BASE, q=BASE["q"] - eps), s0, 0)) / (2 * eps)
    assert abs(dq - fd) < 1e-8 * abs(fd)
    # and the momentum seed is the closed form (delta_{f,chi} - J) pi_f / (a^6 V rho)
    e = o.energies()
    V = N ** 3
    for f in range(2):
        ref = ((1.0 if f == 1 else 0.0) - J) * s0[f][1] / (V * e["rho"])
        assert np.abs(lam[f, 1] - ref).max() < 1e-15 * max(np.abs(ref).max(), 1e-300) + 1e-20


def mode_direction(N, idx, theta, omega, j, H, alpha=1.0, a=1.0):
    """d(phi, pi)/d|z_j| of canonical mode idx (its conjugate partner included)."""
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    kx, ky, kz = idx % N, (idx // N) % N, idx // (N * N)
    ph = np.exp(2j * np.pi * (kx * x + ky * y + kz * z) / N)
    partner = ((-kx) % N) + N * (((-ky) % N) + N * ((-kz) % N))
    e = np.exp(1j * theta) / np.sqrt(2)
    sg = 1.0 if j == 0 else -1.0
    dF = e
    dG = a ** (alpha - 1) * 1j * omega * sg * e - H * e
    V = N ** 3
    if partner == idx:   # self-conjugate: the real part is kept
        dphi = dF.real * ph.real / V
        dpi = a ** (3 - alpha) * dG.real * ph.real / V
    else:
        dphi = 2 * (dF * ph).real / V
        dpi = a ** (3 - alpha) * 2 * (dG * ph).real / V
    return dphi, dpi


def test_mode_amplitude_gradient_matches_difference(oracle_mod):
    N, kIR, seed, n = 8, 1.0, 7, 10
    kw = BASE
    p = O.make_params(**kw)
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p)
    s0 = state_of(o, 2)
    J, dq, lam = o.adjoint(n)
    g = o.ic_amplitude_grad(lam)
    V = N ** 3
    # canonical sites: a generic one, one on an axis, a self-conjugate one
    sites = [1 + N * 2 + N * N * 3, 3, N // 2 + N * (N // 2)]
    dr = O.ic_draws(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p, sites)
    for i, idx in enumerate(sites):
        for f in range(2):
            for j in range(2):
                r, th, om = dr[i, f, 2 * j], dr[i, f, 2 * j + 1], dr[i, f, 4]
                assert r > 0
                dphi, dpi = mode_direction(N, idx, th, om, j, H=0.0)
                eps = 1e-3 * r
                sp = [[s0[k][w].copy() for w in (0, 1)] for k in range(2)]
                sm = [[s0[k][w].copy() for w in (0, 1)] for k in range(2)]
                sp[f][0] += eps * dphi
                sp[f][1] += eps * dpi
                sm[f][0] -= eps * dphi
                sm[f][1] -= eps * dpi
                fd = (run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, kw, sp, n) -
                      run_J(O.MODEL_LPHI4_CHI, N, kIR, seed, kw, sm, n)) / (2 * eps)
                kz_, ky_, kx_ = idx // (N * N), (idx // N) % N, idx % N
                got = g[f, j, kz_, ky_, kx_]
                assert abs(got - fd) < 1e-6 * abs(fd) + 1e-14, (idx, f, j, got, fd)
    # zero at non-canonical sites and at the zero mode
    assert g[:, :, 0, 0, 0].max() == 0.0
    partner = (N - 1) + N * (N - 2) + N * N * (N - 3)
    assert np.all(g.reshape(2, 2, V)[:, :, partner] == 0.0)


def test_all_amplitudes_scaled_together(oracle_mod):
    """Scaling every amplitude by (1 + e) is fluct_amp2 -> fluct_amp2 (1 + e)^2:
    dJ/de = sum over modes of |z| dJ/d|z|."""
    N, kIR, seed, n = 8, 1.0, 8, 10
    kw = BASE
    p = O.make_params(**kw)
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p)
    J, dq, lam = o.adjoint(n)
    g = o.ic_amplitude_grad(lam).reshape(2, 2, -1)
    idx = np.arange(N ** 3)
    dr = O.ic_draws(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p, idx)
    pred = sum(float(np.sum(dr[:, f, 2 * j] * g[f, j])) for f in range(2) for j in range(2))
    eps = 1e-4

    def J_at(e):
        q = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed,
                     O.make_params(**dict(kw, fluct_amp2=kw["fluct_amp2"] * (1 + e) ** 2)))
        q.step(n)
        return chi_fraction(q)

    fd = (J_at(eps) - J_at(-eps)) / (2 * eps)
    assert abs(pred - fd) < 1e-6 * abs(fd), (pred, fd)


SELF = dict(BASE, expansion=O.EXP_SELF, fstar_over_mp=2.0, dt=0.02)


def run_J_self(alpha, kw, state, scal, nsteps, objective=0, spec=None, N=8, kIR=1.0, seed=3):
    """J after nsteps from (state, (eta, a, b)) with self-consistent expansion."""
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, alpha, seed, O.make_params(**kw))
    for f in range(len(state)):
        for w in (0, 1):
            o.set(f, w, state[f][w])
    o.set_scalars(*scal)
    o.step(nsteps)
    if objective == 0:
        return chi_fraction(o)
    field, what, dk, b = spec
    return o.spectrum(field, what, dk)[1][b]


@pytest.mark.parametrize("alpha", [1.0, 0.5])
@pytest.mark.parametrize("objective,spec", [(0, None), (1, (1, 1, 1.0, 2))])
def test_self_consistent_expansion_gradients(oracle_mod, alpha, objective, spec):
    """With a' = b evolving by the Friedmann kicks, dJ/dq, dJ/d(phi, pi) and
    dJ/d(a, b) at the start against central differences of forward runs."""
    N, kIR, seed, n = 8, 1.0, 3, 15
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, alpha, seed, O.make_params(**SELF))
    s0 = state_of(o, 2)
    sc0 = o.scalars()
    kw = dict(objective=1, field=spec[0], what=spec[1], dk_bin=spec[2], bin=spec[3]) if objective else {}
    J, dq, lam, (da, db) = o.adjoint(n, scale=True, **kw)
    assert o.scalars() == sc0
    assert abs(J - run_J_self(alpha, SELF, s0, sc0, n, objective, spec)) < 1e-14 * abs(J)
    # the expansion matters here: a grows by several per cent
    o.step(n)
    assert o.scalars()[1] > 1.05
    eps = 1e-3
    fd = (run_J_self(alpha, dict(SELF, q=SELF["q"] + eps), s0, sc0, n, objective, spec) -
          run_J_self(alpha, dict(SELF, q=SELF["q"] - eps), s0, sc0, n, objective, spec)) / (2 * eps)
    assert abs(dq - fd) < 1e-6 * abs(fd) + 1e-14, (dq, fd)
    e = 1e-6
    eta0, a0, b0 = sc0
    fd_a = (run_J_self(alpha, SELF, s0, (eta0, a0 + e, b0), n, objective, spec) -
            run_J_self(alpha, SELF, s0, (eta0, a0 - e, b0), n, objective, spec)) / (2 * e)
    fd_b = (run_J_self(alpha, SELF, s0, (eta0, a0, b0 + e), n, objective, spec) -
            run_J_self(alpha, SELF, s0, (eta0, a0, b0 - e), n, objective, spec)) / (2 * e)
    assert abs(da - fd_a) < 1e-6 * abs(fd_a) + 1e-13, (da, fd_a)
    assert abs(db - fd_b) < 1e-6 * abs(fd_b) + 1e-13, (db, fd_b)
    rng = np.random.default_rng(11)
    v = [[rng.standard_normal((N, N, N)) for w in (0, 1)] for f in range(2)]
    sp = [[s0[f][w] + e * v[f][w] for w in (0, 1)] for f in range(2)]
    sm = [[s0[f][w] - e * v[f][w] for w in (0, 1)] for f in range(2)]
    fd = (run_J_self(alpha, SELF, sp, sc0, n, objective, spec) -
          run_J_self(alpha, SELF, sm, sc0, n, objective, spec)) / (2 * e)
    ad = sum(float(np.sum(lam[f, w] * v[f][w])) for f in range(2) for w in (0, 1))
    assert abs(ad - fd) < 1e-6 * abs(fd) + 1e-13, (ad, fd)


def test_self_consistent_seed_in_a(oracle_mod):
    """Zero steps: dJ/da is the explicit a-dependence of the energy fraction, dJ/db = 0."""
    o = O.Oracle(O.MODEL_LPHI4_CHI, 8, 1.0, 1.0, 5, O.make_params(**SELF))
    s0 = state_of(o, 2)
    eta0, a0, b0 = o.scalars()
    J, dq, lam, (da, db) = o.adjoint(0, scale=True)
    e = 1e-6
    fd = (run_J_self(1.0, SELF, s0, (eta0, a0 + e, b0), 0, seed=5) -
          run_J_self(1.0, SELF, s0, (eta0, a0 - e, b0), 0, seed=5)) / (2 * e)
    assert abs(da - fd) < 1e-8 * abs(fd)
    assert db == 0.0


def test_self_consistent_amplitude_gradient(oracle_mod):
    """Self-consistent expansion with a' from the homogeneous values (b0_mode 0):
    the ICs are drawn with H = b0/a0 != 0 and b0 does not move with the
    amplitudes, so scaling all of them by (1 + e) is differentiated exactly by
    the chain of lam."""
    N, kIR, seed, n = 8, 1.0, 8, 10
    p = O.make_params(**SELF)
    o = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p)
    assert o.scalars()[2] > 0.5
    J, dq, lam = o.adjoint(n)
    g = o.ic_amplitude_grad(lam).reshape(2, 2, -1)
    dr = O.ic_draws(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, p, np.arange(N ** 3))
    pred = sum(float(np.sum(dr[:, f, 2 * j] * g[f, j])) for f in range(2) for j in range(2))
    eps = 1e-4

    def J_at(e):
        q = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed,
                     O.make_params(**dict(SELF, fluct_amp2=SELF["fluct_amp2"] * (1 + e) ** 2)))
        q.step(n)
        return chi_fraction(q)

    fd = (J_at(eps) - J_at(-eps)) / (2 * eps)
    assert abs(pred - fd) < 1e-6 * abs(fd), (pred, fd)
    # a' from the lattice averages would move b0 with the amplitudes: refused
    o1 = O.Oracle(O.MODEL_LPHI4_CHI, N, kIR, 1.0, seed, O.make_params(**dict(SELF, b0_mode=1)))
    with pytest.raises(ValueError):
        o1.ic_amplitude_grad(lam)


def test_unsupported_cases(oracle_mod):
    o = O.Oracle(O.MODEL_U1_HIGGS, 8, 1.0, 1.0, 1, O.make_params(**dict(BASE, gQ=0.5)))
    with pytest.raises(ValueError):
        o.adjoint(2)
    o1 = O.Oracle(O.MODEL_LPHI4, 8, 1.0, 1.0, 1, O.make_params(**dict(BASE, phi0=[1.0])))
    with pytest.raises(ValueError):
        o1.adjoint(2, objective=0)      # no chi field
