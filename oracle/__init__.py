"""FP64 CPU oracle of the lattice kick-drift method (CosmoLattice manual,
arXiv:2102.01031) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its
``cpu_baseline`` leg and ``--impl reference`` arm) may import this package.
It shares no code with the CUDA library in ``paper_2102_01031_gb300``; the
product path never falls back to it.

The oracle itself is plain C++ (``clo.cpp``), compiled here with g++ and
loaded through ctypes.  See ``clo.h`` for the conventions.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODEL_LPHI4, MODEL_LPHI4_CHI, MODEL_U1_HIGGS, MODEL_SU2U1_HIGGS, MODEL_LPHI4_SU2U1 = 1, 2, 3, 4, 5
LF, VV2, VV4, VV6, VV8, VV10 = 0, 2, 4, 6, 8, 10
EXP_OFF, EXP_SELF, EXP_FIXED = 0, 1, 2


class Params(ctypes.Structure):
    _fields_ = [
        ("dt", ctypes.c_double),
        ("q", ctypes.c_double),
        ("fluct_amp2", ctypes.c_double),
        ("fstar_over_mp", ctypes.c_double),
        ("phi0", ctypes.c_double * 4),
        ("dphi0", ctypes.c_double * 4),
        ("lam", ctypes.c_double),
        ("v", ctypes.c_double),
        ("gQ", ctypes.c_double),
        ("fstar_over_omegastar", ctypes.c_double),
        ("kcut", ctypes.c_double),
        ("omega_eos", ctypes.c_double),
        ("H0", ctypes.c_double),
        ("integrator", ctypes.c_int),
        ("expansion", ctypes.c_int),
        ("b0_mode", ctypes.c_int),
        ("pad_", ctypes.c_int),
        ("gQB", ctypes.c_double),
        ("qG", ctypes.c_double),
        ("qH", ctypes.c_double),
        ("Qc", ctypes.c_double),
    ]


class Energies(ctypes.Structure):
    _fields_ = [
        ("eta", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double),
        ("EK", ctypes.c_double * 4), ("EG", ctypes.c_double * 4), ("EV", ctypes.c_double * 4),
        ("EKA", ctypes.c_double), ("EGA", ctypes.c_double),
        ("rho", ctypes.c_double),
        ("hubble_lhs", ctypes.c_double), ("hubble_rhs", ctypes.c_double),
        ("hubble_viol", ctypes.c_double), ("energy_cons", ctypes.c_double),
        ("mean_phi", ctypes.c_double * 4), ("mean_phi2", ctypes.c_double * 4),
        ("mean_pi", ctypes.c_double * 4), ("mean_pi2", ctypes.c_double * 4),
        ("EKB", ctypes.c_double), ("EGB", ctypes.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else float(v)
        return d


def build(force=False):
    """Compile clo.cpp into _build/liboracle.so (g++, -O2, no -march flags)."""
    src = os.path.join(_HERE, "clo.cpp")
    hdr = os.path.join(_HERE, "clo.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            c_p = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            L.clo_init.argtypes = [ctypes.POINTER(c_p), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(Params)]
            L.clo_free.argtypes = [c_p]
            L.clo_step.argtypes = [c_p, ctypes.c_int]
            L.clo_step_h.argtypes = [c_p, ctypes.c_int, ctypes.c_double]
            L.clo_energies.argtypes = [c_p, ctypes.POINTER(Energies)]
            L.clo_get_state.argtypes = [c_p, ctypes.c_int, ctypes.c_int, dp]
            L.clo_set_state.argtypes = [c_p, ctypes.c_int, ctypes.c_int, dp]
            L.clo_get_scalars.argtypes = [c_p, dp, dp, dp]
            L.clo_set_scalars.argtypes = [c_p, ctypes.c_double, ctypes.c_double, ctypes.c_double]
            L.clo_nfields.argtypes = [c_p]
            L.clo_gauss_constraint.argtypes = [c_p, dp, dp, dp, dp]
            L.clo_get_array.argtypes = [c_p, ctypes.c_int, dp]
            L.clo_set_array.argtypes = [c_p, ctypes.c_int, dp]
            L.clo_gauss_residual.argtypes = [c_p, ctypes.c_int, dp]
            L.clo_su2_exp.argtypes = [dp, dp]
            L.clo_su2_exp.restype = None
            L.clo_spectrum.argtypes = [c_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
            L.clo_em_spectrum.argtypes = [c_p, ctypes.c_int, ctypes.c_double, dp, dp,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int)]
            L.clo_occupation.argtypes = [c_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp,
                                         ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]
            L.clo_norm_spectrum.argtypes = [c_p, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
            L.clo_norm_spectrum_of.argtypes = [c_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]
            L.clo_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
            L.clo_philox4x32_10.restype = None
            L.clo_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
            L.clo_u01.restype = ctypes.c_double
            L.clo_kernel.argtypes = [c_p, ctypes.c_int, dp]
            L.clo_gauss_modes.argtypes = [c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), dp]
            L.clo_draw_pairs.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), dp]
            L.clo_fft3d.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int]
            L.clo_dft3d_naive.argtypes = [dp, dp, dp, dp, ctypes.c_int, ctypes.c_int]
            L.clo_schedule.argtypes = [ctypes.c_int, ctypes.c_double, dp, ctypes.c_int]
            L.clo_ic_sample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_uint64, ctypes.POINTER(Params), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int64), dp]
            L.clo_adjoint.argtypes = [c_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, dp, dp, dp, dp]
            L.clo_ic_amplitude_grad.argtypes = [c_p, dp, dp]
            L.clo_ic_draws.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.POINTER(Params), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int64), dp]
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(**kw):
    """Params with the defaults used throughout the tests; keywords override."""
    p = Params()
    p.dt = kw.pop("dt", 0.01)
    p.q = kw.pop("q", 100.0)
    p.fluct_amp2 = kw.pop("fluct_amp2", 0.0)
    p.fstar_over_mp = kw.pop("fstar_over_mp", 0.0)
    for name in ("phi0", "dphi0"):
        vals = list(kw.pop(name, [0.0] * 4)) + [0.0] * 4
        arr = getattr(p, name)
        for i in range(4):
            arr[i] = vals[i]
    p.lam = kw.pop("lam", 1.0)
    p.v = kw.pop("v", 1.0)
    p.gQ = kw.pop("gQ", 0.5)
    p.fstar_over_omegastar = kw.pop("fstar_over_omegastar", 1.0)
    p.kcut = kw.pop("kcut", -1.0)
    p.omega_eos = kw.pop("omega_eos", 0.0)
    p.H0 = kw.pop("H0", 0.0)
    p.integrator = kw.pop("integrator", VV2)
    p.expansion = kw.pop("expansion", EXP_OFF)
    p.b0_mode = kw.pop("b0_mode", 0)
    p.gQB = kw.pop("gQB", 0.5)
    p.qG = kw.pop("qG", 0.0)
    p.qH = kw.pop("qH", 0.0)
    p.Qc = kw.pop("Qc", 1.0)
    if kw:
        raise TypeError("unknown params: %s" % sorted(kw))
    return p


class Oracle:
    """One oracle lattice (context)."""

    def __init__(self, model, N, kIR, alpha, seed, params):
        self.L = lib()
        self.N = N
        self.V = N ** 3
        self.params = params
        h = ctypes.c_void_p()
        rc = self.L.clo_init(ctypes.byref(h), model, N, kIR, alpha, seed, ctypes.byref(params))
        if rc != 0:
            raise ValueError("clo_init failed (%d)" % rc)
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            self.L.clo_free(self.h)
            self.h = None

    def nfields(self):
        return self.L.clo_nfields(self.h)

    def step(self, n, h=None):
        rc = self.L.clo_step(self.h, n) if h is None else self.L.clo_step_h(self.h, n, h)
        if rc != 0:
            raise RuntimeError("clo_step failed (%d)" % rc)

    def energies(self):
        e = Energies()
        self.L.clo_energies(self.h, ctypes.byref(e))
        return e.as_dict()

    def kernel(self, a):
        """Doublet models: the kernel K (pi' = K) of momentum array a, [z][y][x]."""
        out = np.empty(self.V, dtype=np.float64)
        if self.L.clo_kernel(self.h, a, _dp(out)) != 0:
            raise IndexError(a)
        return out.reshape(self.N, self.N, self.N)

    def gauss_modes(self, idx):
        """U(1) model: Fourier values (unnormalised forward transform) of the
        Gauss-law link momenta of the current charged field at Fourier sites idx:
        complex array (len(idx), 3)."""
        idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
        out = np.zeros(idx.size * 6)
        rc = self.L.clo_gauss_modes(self.h, idx.size, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    _dp(out))
        if rc != 0:
            raise ValueError("clo_gauss_modes")
        out = out.reshape(-1, 3, 2)
        return out[:, :, 0] + 1j * out[:, :, 1]

    def get(self, field, what=0):
        out = np.empty(self.V, dtype=np.float64)
        if self.L.clo_get_state(self.h, field, what, _dp(out)) != 0:
            raise IndexError((field, what))
        return out.reshape(self.N, self.N, self.N)  # [z][y][x]

    def set(self, field, what, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        if a.size != self.V or self.L.clo_set_state(self.h, field, what, _dp(a)) != 0:
            raise IndexError((field, what))

    def get_array(self, a):
        """Doublet model: array `a` in the order of clo_get_array, as [z][y][x]."""
        out = np.empty(self.V, dtype=np.float64)
        if self.L.clo_get_array(self.h, a, _dp(out)) != 0:
            raise IndexError(a)
        return out.reshape(self.N, self.N, self.N)

    def set_array(self, a, arr):
        x = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        if x.size != self.V or self.L.clo_set_array(self.h, a, _dp(x)) != 0:
            raise IndexError(a)

    def gauss_residual(self, g=0):
        """Per-site Gauss residual of generator g (0: U(1); 1..3: SU(2) colours)."""
        out = np.empty(self.V, dtype=np.float64)
        if self.L.clo_gauss_residual(self.h, g, _dp(out)) != 0:
            raise ValueError("no such Gauss law")
        return out.reshape(self.N, self.N, self.N)

    def scalars(self):
        e, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        self.L.clo_get_scalars(self.h, ctypes.byref(e), ctypes.byref(a), ctypes.byref(b))
        return e.value, a.value, b.value

    def set_scalars(self, eta, a, b):
        self.L.clo_set_scalars(self.h, eta, a, b)

    def gauss(self):
        r, l, s, m = (ctypes.c_double() for _ in range(4))
        if self.L.clo_gauss_constraint(self.h, ctypes.byref(r), ctypes.byref(l), ctypes.byref(s),
                                       ctypes.byref(m)) != 0:
            raise ValueError("no gauge field")
        return r.value, l.value, s.value, m.value

    def spectrum(self, field, what=0, dk_bin=1.0):
        cap = 4096
        k = np.zeros(cap)
        d = np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.clo_spectrum(self.h, field, what, dk_bin, _dp(k), _dp(d),
                                 m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap,
                                 ctypes.byref(nb))
        if rc != 0:
            raise ValueError("clo_spectrum failed (%d)" % rc)
        n = nb.value
        return k[:n].copy(), d[:n].copy(), m[:n].copy()


    def em_spectrum(self, which, dk_bin=1.0):
        """(k, delta, multiplicity) of the U(1) electric (which=0) or magnetic (1) field."""
        cap = 4096
        k, d = np.zeros(cap), np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.clo_em_spectrum(self.h, which, dk_bin, _dp(k), _dp(d),
                                    m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        if rc != 0:
            raise ValueError("clo_em_spectrum failed (%d)" % rc)
        n = nb.value
        return k[:n].copy(), d[:n].copy(), m[:n].copy()

    def occupation(self, field, dk_bin=1.0, fo2=None):
        """(k, n_k, multiplicity) per bin: lattice occupation number of scalar field
        `field`; fo2 = (f*/omega*)^2, by default 1/fluct_amp2."""
        if fo2 is None:
            fo2 = 1.0 / self.params.fluct_amp2
        cap = 4096
        k, nk = np.zeros(cap), np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.clo_occupation(self.h, field, dk_bin, fo2, _dp(k), _dp(nk),
                                   m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        if rc != 0:
            raise ValueError("clo_occupation failed (%d)" % rc)
        n = nb.value
        return k[:n].copy(), nk[:n].copy(), m[:n].copy()

    def norm_spectrum(self, dk_bin=1.0, fo2=None, which=0):
        """(k, Delta_r, Delta_r', n, multiplicity) of the charged field's modulus r = |phi|
        (gauge models; n is that of the canonical modulus sqrt2 r); fo2 = (f*/omega*)^2,
        default 1/fluct_amp2.  which = 1: lphi4SU2U1's U(1)-charged scalar."""
        if fo2 is None:
            fo2 = 1.0 / self.params.fluct_amp2
        cap = 4096
        k, d1, d2, n = (np.zeros(cap) for _ in range(4))
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.clo_norm_spectrum_of(self.h, which, dk_bin, fo2, _dp(k), _dp(d1), _dp(d2), _dp(n),
                                      m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        if rc != 0:
            raise ValueError("clo_norm_spectrum failed (%d)" % rc)
        b = nb.value
        return k[:b].copy(), d1[:b].copy(), d2[:b].copy(), n[:b].copy(), m[:b].copy()

    def adjoint(self, nsteps, objective=0, field=1, what=0, dk_bin=1.0, bin=1, scale=False):
        """Discrete adjoint: (J, dJ/dq, lam) with lam[f][w] = dJ/d(field f, what w) at
        the current state (arrays [z][y][x]); with scale=True a fourth entry
        (dJ/da, dJ/db) at the current state.  The state is left unchanged."""
        nf = 1 if self.nfields() == 1 else 2
        lam = np.zeros(2 * nf * self.V)
        ab = np.zeros(2)
        J, dq = ctypes.c_double(), ctypes.c_double()
        rc = self.L.clo_adjoint(self.h, nsteps, objective, field, what, dk_bin, bin, ctypes.byref(J),
                                ctypes.byref(dq), _dp(lam), _dp(ab))
        if rc != 0:
            raise ValueError("clo_adjoint failed (%d)" % rc)
        lam = lam.reshape(nf, 2, self.N, self.N, self.N)
        if scale:
            return J.value, dq.value, lam, (float(ab[0]), float(ab[1]))
        return J.value, dq.value, lam

    def ic_amplitude_grad(self, lam):
        """dJ/d|z_j| of every canonical mode from lam (as returned by adjoint at the ICs):
        array [field][j][z][y][x], zero at non-canonical sites."""
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(-1))
        out = np.zeros_like(lam)
        if self.L.clo_ic_amplitude_grad(self.h, _dp(lam), _dp(out)) != 0:
            raise ValueError("clo_ic_amplitude_grad")
        nf = lam.size // (2 * self.V)
        return out.reshape(nf, 2, self.N, self.N, self.N)


def ic_draws(model, N, kIR, alpha, seed, params, idx):
    """(|z1|, arg z1, |z2|, arg z2, omega) per field at canonical site indices."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    nf = 1 if model == MODEL_LPHI4 else 2
    out = np.zeros(idx.size * nf * 5)
    rc = lib().clo_ic_draws(model, N, kIR, alpha, seed, ctypes.byref(params), idx.size,
                            idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    if rc != 0:
        raise ValueError("clo_ic_draws")
    return out.reshape(idx.size, nf, 5)


def su2_exp(theta):
    """exp(-i theta.sigma/2) as (u0, u1, u2, u3), U = u0 - i u.sigma."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(3))
    u = np.zeros(4)
    lib().clo_su2_exp(_dp(th), _dp(u))
    return u


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().clo_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def u01(hi, lo):
    return lib().clo_u01(hi, lo)


def draw_pairs(seed, idx, f, j):
    """The oracle's IC draw pairs (u1, u2) at Fourier indices idx, components f,
    draws j (0 amplitudes, 1 phases): shape (n, 2)."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64).reshape(-1))
    f = np.ascontiguousarray(np.asarray(f, dtype=np.int32).reshape(-1))
    j = np.ascontiguousarray(np.asarray(j, dtype=np.int32).reshape(-1))
    out = np.zeros((idx.size, 2))
    ip = ctypes.POINTER(ctypes.c_int)
    rc = lib().clo_draw_pairs(int(seed), idx.size, idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              f.ctypes.data_as(ip), j.ctypes.data_as(ip), _dp(out))
    if rc != 0:
        raise ValueError("clo_draw_pairs")
    return out


def fft3d(x, sign):
    """Unnormalised 3-D DFT of a complex N^3 array with the oracle's own FFT."""
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[0]
    re = np.ascontiguousarray(x.real.reshape(-1))
    im = np.ascontiguousarray(x.imag.reshape(-1))
    if lib().clo_fft3d(_dp(re), _dp(im), N, sign) != 0:
        raise ValueError("fft3d")
    return (re + 1j * im).reshape(x.shape)


def dft3d_naive(x, sign):
    x = np.asarray(x, dtype=np.complex128)
    N = x.shape[0]
    re = np.ascontiguousarray(x.real.reshape(-1))
    im = np.ascontiguousarray(x.imag.reshape(-1))
    ore = np.empty_like(re)
    oim = np.empty_like(im)
    if lib().clo_dft3d_naive(_dp(re), _dp(im), _dp(ore), _dp(oim), N, sign) != 0:
        raise ValueError("dft3d_naive")
    return (ore + 1j * oim).reshape(x.shape)


def ic_sample(model, N, kIR, alpha, seed, params, idx):
    """Initial Fourier values (F, G) per field at the given linear site indices."""
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    nf = {MODEL_LPHI4: 1, MODEL_SU2U1_HIGGS: 4, MODEL_LPHI4_SU2U1: 7}.get(model, 2)
    out = np.zeros(idx.size * nf * 4)
    rc = lib().clo_ic_sample(model, N, kIR, alpha, seed, ctypes.byref(params), idx.size,
                             idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    if rc != 0:
        raise ValueError("clo_ic_sample")
    o = out.reshape(idx.size, nf, 4)
    return o[..., 0] + 1j * o[..., 1], o[..., 2] + 1j * o[..., 3]


def schedule(integrator, h):
    out = np.zeros(256)
    n = lib().clo_schedule(integrator, h, _dp(out), 256)
    if n < 0:
        raise ValueError("schedule")
    return out[:n].copy()
