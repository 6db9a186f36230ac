"""Seeded synthetic lattice states shared by the oracle and the CUDA path.

This module holds no arithmetic of the method: it only draws reproducible
arrays (sums of random plane waves with numpy's PCG64 generator) that the
parity tests load into both sides with set_state.
"""
import numpy as np


def smooth_field(N, seed, n_waves=6, amp=0.3, offset=0.0, kmax=4):
    """offset + sum of n_waves random plane waves with integer wave numbers <= kmax."""
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    f = np.full((N, N, N), float(offset))
    for _ in range(n_waves):
        m = rng.integers(-kmax, kmax + 1, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        a = amp * rng.uniform(0.2, 1.0) / n_waves
        f += a * np.cos(2 * np.pi * (m[0] * x + m[1] * y + m[2] * z) / N + ph)
    return f


def random_field(N, seed, scale=1.0, offset=0.0):
    rng = np.random.default_rng(seed)
    return offset + scale * rng.standard_normal((N, N, N))


def scalar_state(N, seed, nf=2, rough=False):
    """[(phi_f, pi_f) for f < nf]: phi ~ 1 + waves for f = 0, small waves otherwise."""
    out = []
    for f in range(nf):
        gen = random_field if rough else smooth_field
        if rough:
            phi = gen(N, seed * 101 + f, scale=0.05, offset=1.0 if f == 0 else 0.0)
            pi = gen(N, seed * 103 + f, scale=0.05)
        else:
            phi = gen(N, seed * 101 + f, amp=0.3 if f == 0 else 0.05, offset=1.0 if f == 0 else 0.0)
            pi = gen(N, seed * 103 + f, amp=0.2 if f == 0 else 0.05)
        out.append((phi, pi))
    return out


def su2_doublet_state(N, seed, link_spread=0.4, mom=0.3, phi_offset=0.6, u1=True):
    """Arrays of the SU(2) x U(1) doublet model in its array order (35 arrays,
    each [z][y][x]): doublet components near phi_offset, random unit
    quaternions spread about the identity for the SU(2) links, and random
    momenta; with u1=False the U(1) link fields and momenta are zero."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(4):
        out.append(phi_offset + 0.2 * rng.standard_normal((N, N, N)))
    for c in range(4):
        out.append(mom * rng.standard_normal((N, N, N)))
    for i in range(6):
        out.append((0.2 * rng.standard_normal((N, N, N))) if u1 else np.zeros((N, N, N)))
    for i in range(3):
        q = link_spread * rng.standard_normal((4, N, N, N))
        q[0] += 1.0
        q /= np.sqrt((q ** 2).sum(axis=0))
        out.extend(list(q))
    for i in range(9):
        out.append(mom * rng.standard_normal((N, N, N)))
    return out
