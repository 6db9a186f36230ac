"""GB300 (sm_103a) lattice kick-drift library: Python binding of ``include/cl.h``.

The library evolves scalar fields (and U(1) gauge links) on a periodic N^3
lattice in an expanding universe with the velocity-Verlet / leapfrog
kick-drift integrators of the CosmoLattice manual (arXiv:2102.01031).  Every
step of the method runs in the CUDA kernels of ``libclgb300.so``; this module
only marshals arguments through ctypes.  There is no CPU fallback: importing
works without a GPU, but creating a lattice fails loudly when the library or
the GPU is missing.

Functions carry the names of the C ABI (``cl_init``, ``cl_step``,
``cl_energies``, ``cl_gauss_constraint``, ``cl_spectrum``, ...); ``Lattice``
wraps one context.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libclgb300.so")

CL_OK, CL_EINVAL, CL_ENOMEM, CL_ECUDA, CL_ESTATE, CL_ETIMEOUT, CL_ENONFINITE, CL_EUNSUPPORTED = range(8)
MODEL_LPHI4, MODEL_LPHI4_CHI, MODEL_U1_HIGGS, MODEL_SU2U1_HIGGS, MODEL_LPHI4_SU2U1 = 1, 2, 3, 4, 5
LF, VV2, VV4, VV6, VV8, VV10 = 0, 2, 4, 6, 8, 10
FP64, FP32 = 0, 1
EXP_OFF, EXP_SELF, EXP_FIXED = 0, 1, 2

# every entry point declared in include/cl.h
EXPORTS = (
    "cl_init", "cl_free", "cl_step", "cl_step_h", "cl_sync", "cl_energies", "cl_gauss_constraint",
    "cl_spectrum", "cl_get_state", "cl_set_state", "cl_get_scalars", "cl_set_scalars",
    "cl_state_bytes", "cl_upload_state", "cl_download_state", "cl_nfields", "cl_kernel_launches",
    "cl_last_error", "cl_enable_pass_timing", "cl_pass_timing", "cl_volume_averages_noalloc",
    "cl_ensemble_init", "cl_ensemble_size", "cl_lattice_energies", "cl_lattice_get_state",
    "cl_lattice_set_state", "cl_lattice_scalars", "cl_lattice_tile", "cl_ensemble_spectrum",
    "cl_adjoint", "cl_ic_amplitude_grad", "cl_occupation", "cl_measure_fp64_rate", "cl_em_spectrum",
    "cl_get_array", "cl_set_array", "cl_norm_spectrum", "cl_checkpoint_save", "cl_checkpoint_load",
    "cl_set_tune_cache", "cl_selftest_wait", "cl_pass_weights", "cl_philox_draws",
    "cl_adjoint_pass_timing", "cl_bind_buffers", "cl_state_buffer", "cl_norm_spectrum_of",
)
OBJ_CHI_FRACTION, OBJ_SPECTRUM_BIN = 0, 1


class ClError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("cl status %d: %s" % (status, msg))
        self.status = status


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
        ("precision", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("autotune", ctypes.c_int),
        ("tile_by", ctypes.c_int),
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
        ("nonfinite", ctypes.c_int64),
        ("EKB", ctypes.c_double), ("EGB", ctypes.c_double),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else (int(v) if name == "nonfinite" else float(v))
        return d


_lib = None


def build(force=False):
    """Compile csrc/*.cu for sm_103a into _build/libclgb300.so (see builder.py)."""
    from . import builder
    return builder.build(force=force)


def lib():
    """Load libclgb300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("CUDA library not built: %s (run __graft_entry__.build())" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    L.cl_init.argtypes = [ctypes.POINTER(vp), ip, ip, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                          ctypes.POINTER(Params)]
    L.cl_free.argtypes = [vp]
    L.cl_step.argtypes = [vp, ip]
    L.cl_step_h.argtypes = [vp, ip, ctypes.c_double]
    L.cl_sync.argtypes = [vp]
    L.cl_energies.argtypes = [vp, ctypes.POINTER(Energies)]
    L.cl_gauss_constraint.argtypes = [vp, dp, dp, dp, dp]
    L.cl_spectrum.argtypes = [vp, ip, ip, ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_int64), ip,
                              ctypes.POINTER(ctypes.c_int)]
    L.cl_get_state.argtypes = [vp, ip, ip, dp]
    L.cl_set_state.argtypes = [vp, ip, ip, dp]
    L.cl_get_array.argtypes = [vp, ip, dp]
    L.cl_checkpoint_save.argtypes = [vp, ctypes.c_char_p]
    L.cl_set_tune_cache.argtypes = [ctypes.c_char_p]
    L.cl_checkpoint_load.argtypes = [vp, ctypes.c_char_p]
    L.cl_norm_spectrum.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                   ctypes.POINTER(ctypes.c_int64), ip, ctypes.POINTER(ctypes.c_int)]
    L.cl_norm_spectrum_of.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double, dp, dp, dp, dp,
                                   ctypes.POINTER(ctypes.c_int64), ip, ctypes.POINTER(ctypes.c_int)]
    L.cl_set_array.argtypes = [vp, ip, dp]
    L.cl_get_scalars.argtypes = [vp, dp, dp, dp]
    L.cl_set_scalars.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.cl_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.cl_upload_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.cl_download_state.argtypes = [vp, vp, ctypes.c_size_t]
    L.cl_bind_buffers.argtypes = [vp, ip, vp, vp, ctypes.c_size_t]
    L.cl_state_buffer.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.cl_nfields.argtypes = [vp]
    L.cl_kernel_launches.argtypes = [vp]
    L.cl_kernel_launches.restype = ctypes.c_int64
    L.cl_last_error.argtypes = [vp]
    L.cl_last_error.restype = ctypes.c_char_p
    L.cl_enable_pass_timing.argtypes = [vp, ip]
    L.cl_pass_timing.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64), ip]
    L.cl_adjoint_pass_timing.argtypes = [vp, dp, ctypes.POINTER(ctypes.c_int64), ip]
    L.cl_volume_averages_noalloc.argtypes = [ip, ip, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ip, ctypes.POINTER(vp), vp, vp]
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.cl_ensemble_init.argtypes = [ctypes.POINTER(vp), ip, ip, ctypes.POINTER(ctypes.c_int), dp,
                                   ctypes.c_double, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Params)]
    L.cl_ensemble_size.argtypes = [vp]
    L.cl_lattice_energies.argtypes = [vp, ip, ctypes.POINTER(Energies)]
    L.cl_lattice_get_state.argtypes = [vp, ip, ip, ip, dp]
    L.cl_lattice_set_state.argtypes = [vp, ip, ip, ip, dp]
    L.cl_lattice_scalars.argtypes = [vp, ip, dp, dp, dp]
    L.cl_lattice_tile.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_int)]
    L.cl_ensemble_spectrum.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ip, ip, ip, ctypes.c_double, dp, dp,
                                       i64p, ip, ctypes.POINTER(ctypes.c_int)]
    L.cl_adjoint.argtypes = [vp, ip, ip, ip, ip, ip, ctypes.c_double, ip, dp, dp, dp, dp]
    L.cl_ic_amplitude_grad.argtypes = [vp, dp, dp]
    L.cl_measure_fp64_rate.argtypes = [vp, dp]
    L.cl_pass_weights.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), dp,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.cl_selftest_wait.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.cl_em_spectrum.argtypes = [vp, ip, ctypes.c_double, dp, dp, ctypes.POINTER(ctypes.c_int64), ip,
                                 ctypes.POINTER(ctypes.c_int)]
    u32p = ctypes.POINTER(ctypes.c_uint32)
    L.cl_philox_draws.argtypes = [vp, ip, ip, u32p, u32p, u32p, dp]
    L.cl_occupation.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double, dp, dp,
                                ctypes.POINTER(ctypes.c_int64), ip, ctypes.POINTER(ctypes.c_int)]
    _lib = L
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(**kw):
    """cl_params with defaults; keywords override (stream: int handle or None)."""
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
    p.precision = kw.pop("precision", FP64)
    p.autotune = int(kw.pop("autotune", 0))
    p.tile_by = int(kw.pop("tile_by", 0))
    p.gQB = kw.pop("gQB", 0.5)
    p.qG = kw.pop("qG", 0.0)
    p.qH = kw.pop("qH", 0.0)
    p.Qc = kw.pop("Qc", 1.0)
    st = kw.pop("stream", None)
    p.stream = ctypes.c_void_p(int(st) if st else 0)
    if kw:
        raise TypeError("unknown params: %s" % sorted(kw))
    return p


def set_tune_cache(path):
    """cl_set_tune_cache: keep autotuned tile heights in `path` (None: off)."""
    L = lib()
    rc = L.cl_set_tune_cache(os.fsencode(path) if path else None)
    if rc != CL_OK:
        raise ClError(rc, "cl_set_tune_cache")


def measure_fp64_rate(stream=None):
    """cl_measure_fp64_rate: measured FP64 operations per second of the current
    device (FMA = 2), the roof of the FP64 plain pass."""
    L = lib()
    r = ctypes.c_double()
    rc = L.cl_measure_fp64_rate(stream, ctypes.byref(r))
    if rc != 0:
        raise ClError(rc, "cl_measure_fp64_rate failed")
    return r.value


def pass_weights(integrator, h, steps_per_call):
    """cl_pass_weights: (npass, 4) array of (ck, wout, win, dnext) of the passes that
    successive cl_step_h calls of these step counts launch, with the closing half kick."""
    L = lib()
    calls = (ctypes.c_int * max(1, len(steps_per_call)))(*steps_per_call)
    n = ctypes.c_int()
    cap = 16
    while True:
        out = np.zeros(4 * cap)
        rc = L.cl_pass_weights(int(integrator), float(h), len(steps_per_call), calls, _dp(out), cap,
                               ctypes.byref(n))
        if rc == CL_OK:
            return out[:4 * n.value].reshape(-1, 4)
        if rc != CL_EINVAL or n.value <= cap:
            raise ClError(rc, "cl_pass_weights")
        cap = n.value


def philox_draws(mode, ctr, key, stream=None):
    """cl_philox_draws: the initial conditions' generator on the GPU.  ctr is (n, 4)
    and key (n, 2) uint32; returns (words (n, 4) uint32, deviates (n, 2) float64):
    mode 0 the raw Philox4x32-10 words and their two 53-bit deviates, mode 1 the
    draw pair of the initial conditions (ctr rows = Fourier index, component,
    draw, unused; key rows = the seed's low and high words)."""
    L = lib()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(-1, 2))
    if len(c) != len(k):
        raise ValueError("ctr and key lengths differ")
    n = len(c)
    out = np.zeros((n, 4), dtype=np.uint32)
    u = np.zeros((n, 2))
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = L.cl_philox_draws(stream, int(mode), n, c.ctypes.data_as(u32p), k.ctypes.data_as(u32p),
                           out.ctypes.data_as(u32p), _dp(u))
    if rc != CL_OK:
        raise ClError(rc, "cl_philox_draws")
    return out, u


def selftest_wait(kind, satisfied, limit_ns, stream=None):
    """cl_selftest_wait: run one of the passes' bounded device waits (kind 0 the
    counter wait, 1 the mbarrier wait) that is satisfied or never is; returns
    (status, device nanoseconds the wait took), status CL_OK or CL_ETIMEOUT."""
    L = lib()
    ns = ctypes.c_uint64()
    rc = L.cl_selftest_wait(stream, int(kind), 1 if satisfied else 0, int(limit_ns), ctypes.byref(ns))
    if rc not in (CL_OK, CL_ETIMEOUT):
        raise ClError(rc, "cl_selftest_wait")
    return rc, ns.value


def torch_stream():
    """Handle of torch's current CUDA stream (PyTorch supplies streams only)."""
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(L, h, rc, what):
    if rc != CL_OK:
        msg = L.cl_last_error(h).decode(errors="replace")
        raise ClError(rc, "%s: %s" % (what, msg))


class Lattice:
    """One lattice context of the CUDA library (cl_init ... cl_free)."""

    def __init__(self, model, N, kIR, alpha, seed, params):
        self.L = lib()
        self.N = N
        self.V = N ** 3
        self.params = params
        h = ctypes.c_void_p()
        rc = self.L.cl_init(ctypes.byref(h), model, N, kIR, alpha, seed, ctypes.byref(params))
        if rc != CL_OK:
            raise ClError(rc, "cl_init: " + self.L.cl_last_error(None).decode(errors="replace"))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.cl_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def nfields(self):
        return self.L.cl_nfields(self.h)

    def step(self, n, h=None):
        rc = self.L.cl_step(self.h, n) if h is None else self.L.cl_step_h(self.h, n, h)
        _check(self.L, self.h, rc, "cl_step")

    def sync(self):
        _check(self.L, self.h, self.L.cl_sync(self.h), "cl_sync")

    def energies(self, allow_nonfinite=False):
        e = Energies()
        rc = self.L.cl_energies(self.h, ctypes.byref(e))
        if not (allow_nonfinite and rc == CL_ENONFINITE):
            _check(self.L, self.h, rc, "cl_energies")
        return e.as_dict()

    def get(self, field, what=0):
        out = np.empty(self.V, dtype=np.float64)
        _check(self.L, self.h, self.L.cl_get_state(self.h, field, what, _dp(out)), "cl_get_state")
        return out.reshape(self.N, self.N, self.N)  # [z][y][x]

    def set(self, field, what, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        if a.size != self.V:
            raise ValueError("need %d values" % self.V)
        _check(self.L, self.h, self.L.cl_set_state(self.h, field, what, _dp(a)), "cl_set_state")

    def get_device(self, field, what, ptr):
        """cl_get_state into device memory: `ptr` is the address of N^3 doubles on
        the GPU (e.g. a CUDA tensor's data_ptr()); the copy stays on the device."""
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self.L, self.h, self.L.cl_get_state(self.h, field, what, ctypes.cast(ctypes.c_void_p(ptr), dp)),
               "cl_get_state")

    def set_device(self, field, what, ptr):
        """cl_set_state from device memory (N^3 doubles at `ptr`, x fastest)."""
        dp = ctypes.POINTER(ctypes.c_double)
        _check(self.L, self.h, self.L.cl_set_state(self.h, field, what, ctypes.cast(ctypes.c_void_p(ptr), dp)),
               "cl_set_state")

    def save(self, path):
        """cl_checkpoint_save: state and scalars to `path` (written atomically)."""
        _check(self.L, self.h, self.L.cl_checkpoint_save(self.h, os.fsencode(path)), "cl_checkpoint_save")

    def load(self, path):
        """cl_checkpoint_load: resume from a checkpoint of a matching lattice."""
        _check(self.L, self.h, self.L.cl_checkpoint_load(self.h, os.fsencode(path)), "cl_checkpoint_load")

    def get_array(self, a):
        """cl_get_array (doublet model): array `a` of the state as [z][y][x]."""
        out = np.empty(self.V, dtype=np.float64)
        _check(self.L, self.h, self.L.cl_get_array(self.h, a, _dp(out)), "cl_get_array")
        return out.reshape(self.N, self.N, self.N)

    def set_array(self, a, arr):
        x = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        if x.size != self.V:
            raise ValueError("need %d values" % self.V)
        _check(self.L, self.h, self.L.cl_set_array(self.h, a, _dp(x)), "cl_set_array")

    def scalars(self):
        e, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.L, self.h, self.L.cl_get_scalars(self.h, ctypes.byref(e), ctypes.byref(a),
                                                     ctypes.byref(b)), "cl_get_scalars")
        return e.value, a.value, b.value

    def set_scalars(self, eta, a, b):
        _check(self.L, self.h, self.L.cl_set_scalars(self.h, eta, a, b), "cl_set_scalars")

    def gauss(self):
        r, l, s, m = (ctypes.c_double() for _ in range(4))
        _check(self.L, self.h, self.L.cl_gauss_constraint(self.h, ctypes.byref(r), ctypes.byref(l),
                                                          ctypes.byref(s), ctypes.byref(m)),
               "cl_gauss_constraint")
        return r.value, l.value, s.value, m.value

    def spectrum(self, field, what=0, dk_bin=1.0):
        cap = 4096
        k = np.zeros(cap)
        d = np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.cl_spectrum(self.h, field, what, dk_bin, _dp(k), _dp(d),
                                m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        _check(self.L, self.h, rc, "cl_spectrum")
        n = nb.value
        return k[:n].copy(), d[:n].copy(), m[:n].copy()

    def norm_spectrum(self, dk_bin=1.0, fo2=0.0, which=0):
        """cl_norm_spectrum_of (gauge models): (k, Delta_r, Delta_r', n, multiplicity) of
        the charged field's modulus r = |phi| (n: that of the canonical modulus sqrt2 r);
        fo2 = (f*/omega*)^2 (<= 0: 1/fluct_amp2); which = 1: lphi4SU2U1's vphi."""
        cap = 4096
        k, d1, d2, n = (np.zeros(cap) for _ in range(4))
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.cl_norm_spectrum_of(self.h, which, dk_bin, fo2, _dp(k), _dp(d1), _dp(d2), _dp(n),
                                        m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        _check(self.L, self.h, rc, "cl_norm_spectrum_of")
        b = nb.value
        return k[:b].copy(), d1[:b].copy(), d2[:b].copy(), n[:b].copy(), m[:b].copy()

    def em_spectrum(self, which, dk_bin=1.0):
        """cl_em_spectrum: (k, delta, multiplicity) of the U(1) electric (which=0) or
        magnetic (which=1) field; doublet model also the SU(2) electric (2) and
        magnetic (3) fields, summed over colour."""
        cap = 4096
        k, d = np.zeros(cap), np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.cl_em_spectrum(self.h, which, dk_bin, _dp(k), _dp(d),
                                   m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        _check(self.L, self.h, rc, "cl_em_spectrum")
        n = nb.value
        return k[:n].copy(), d[:n].copy(), m[:n].copy()

    def occupation(self, field, dk_bin=1.0, fo2=0.0):
        """cl_occupation: (k, n_k, multiplicity) per bin, lattice occupation number of
        scalar field `field`; fo2 = (f*/omega*)^2 (<= 0: 1/fluct_amp2)."""
        cap = 4096
        k, nk = np.zeros(cap), np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        rc = self.L.cl_occupation(self.h, field, dk_bin, fo2, _dp(k), _dp(nk),
                                  m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap, ctypes.byref(nb))
        _check(self.L, self.h, rc, "cl_occupation")
        n = nb.value
        return k[:n].copy(), nk[:n].copy(), m[:n].copy()

    def state_bytes(self):
        n = ctypes.c_size_t()
        _check(self.L, self.h, self.L.cl_state_bytes(self.h, ctypes.byref(n)), "cl_state_bytes")
        return n.value

    def bind_buffers(self, buf0, buf1, lat=0):
        """cl_bind_buffers: two caller-owned CUDA tensors (contiguous, on the
        context's device, 256-byte aligned, each at least the lattice's state
        size) become the lattice's two state buffers, the state copied into
        them.  They stay referenced here while bound.  bind_buffers(None, None)
        moves the state back into memory of the lattice's own."""
        bound = self.__dict__.setdefault("_bound", {})
        if buf0 is None and buf1 is None:
            _check(self.L, self.h, self.L.cl_bind_buffers(self.h, lat, None, None, 0), "cl_bind_buffers")
            bound.pop(lat, None)
            return
        for t in (buf0, buf1):
            if not t.is_contiguous():
                raise ValueError("bound buffers must be contiguous")
        nbytes = min(buf0.numel() * buf0.element_size(), buf1.numel() * buf1.element_size())
        _check(self.L, self.h, self.L.cl_bind_buffers(self.h, lat, ctypes.c_void_p(buf0.data_ptr()),
                                                      ctypes.c_void_p(buf1.data_ptr()), nbytes),
               "cl_bind_buffers")
        bound[lat] = (buf0, buf1)

    def state_buffer(self):
        """cl_state_buffer: 0 or 1, the buffer that holds the state once the
        passes enqueued so far have run."""
        w = ctypes.c_int()
        _check(self.L, self.h, self.L.cl_state_buffer(self.h, ctypes.byref(w)), "cl_state_buffer")
        return w.value

    def upload(self, host_ptr, nbytes):
        _check(self.L, self.h, self.L.cl_upload_state(self.h, ctypes.c_void_p(host_ptr), nbytes),
               "cl_upload_state")

    def download(self, host_ptr, nbytes):
        _check(self.L, self.h, self.L.cl_download_state(self.h, ctypes.c_void_p(host_ptr), nbytes),
               "cl_download_state")

    def launches(self):
        return int(self.L.cl_kernel_launches(self.h))

    def enable_pass_timing(self, on=True):
        _check(self.L, self.h, self.L.cl_enable_pass_timing(self.h, 1 if on else 0), "timing")

    def pass_timing(self, reset=False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self.L, self.h, self.L.cl_pass_timing(self.h, ctypes.byref(ms), ctypes.byref(n),
                                                     1 if reset else 0), "timing")
        return ms.value, n.value

    def adjoint_pass_timing(self, reset=False):
        """cl_adjoint_pass_timing: (ms, passes) of the reversed passes timed so far."""
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self.L, self.h, self.L.cl_adjoint_pass_timing(self.h, ctypes.byref(ms), ctypes.byref(n),
                                                             1 if reset else 0), "timing")
        return ms.value, n.value

    def adjoint(self, nsteps, ckpt_every=500, objective=OBJ_CHI_FRACTION, field=1, what=0, dk_bin=1.0,
                bin=1, scale=False, lam_ptr=None):
        """cl_adjoint: (J, dJ/dq, lam), lam[f][w] = dJ/d(field f, what w) at the current
        state ([z][y][x] arrays); with scale=True a fourth entry (dJ/da, dJ/db).
        With lam_ptr (the device address of 2 nf N^3 doubles, e.g. a CUDA tensor's
        data_ptr()) dJ/d(state) is written there on the GPU and lam is None.
        The state is left unchanged."""
        nf = self.nfields()
        ab = np.zeros(2)
        J, dq = ctypes.c_double(), ctypes.c_double()
        if lam_ptr is None:
            lam = np.zeros(2 * nf * self.V)
            lp = _dp(lam)
        else:
            lam = None
            lp = ctypes.cast(ctypes.c_void_p(lam_ptr), ctypes.POINTER(ctypes.c_double))
        rc = self.L.cl_adjoint(self.h, nsteps, ckpt_every, objective, field, what, dk_bin, bin,
                               ctypes.byref(J), ctypes.byref(dq), lp, _dp(ab))
        _check(self.L, self.h, rc, "cl_adjoint")
        if lam is not None:
            lam = lam.reshape(nf, 2, self.N, self.N, self.N)
        if scale:
            return J.value, dq.value, lam, (float(ab[0]), float(ab[1]))
        return J.value, dq.value, lam

    def ic_amplitude_grad(self, lam):
        """cl_ic_amplitude_grad: dJ/d|z_j| per field and draw, [f][j][z][y][x]."""
        lam = np.ascontiguousarray(np.asarray(lam, dtype=np.float64).reshape(-1))
        out = np.zeros_like(lam)
        _check(self.L, self.h, self.L.cl_ic_amplitude_grad(self.h, _dp(lam), _dp(out)), "cl_ic_amplitude_grad")
        return out.reshape(-1, 2, self.N, self.N, self.N)


class Ensemble:
    """An ensemble context (cl_ensemble_init ... cl_free): lattices of sizes
    Ns[l], kIRs[l] and seeds[l] advanced together by one launch per call."""

    def __init__(self, model, Ns, kIRs, alpha, seeds, params):
        self.L = lib()
        self.Ns = [int(n) for n in Ns]
        n = len(self.Ns)
        if len(kIRs) != n or len(seeds) != n:
            raise ValueError("Ns, kIRs and seeds need one entry per lattice")
        self.params = params
        ns = (ctypes.c_int * n)(*self.Ns)
        ks = (ctypes.c_double * n)(*[float(k) for k in kIRs])
        ss = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
        h = ctypes.c_void_p()
        rc = self.L.cl_ensemble_init(ctypes.byref(h), model, n, ns, ks, alpha, ss, ctypes.byref(params))
        if rc != CL_OK:
            raise ClError(rc, "cl_ensemble_init: " + self.L.cl_last_error(None).decode(errors="replace"))
        self.h = h

    # caller-owned state buffers of lattice `lat` (cl_bind_buffers, cl_state_buffer)
    bind_buffers = Lattice.bind_buffers
    state_buffer = Lattice.state_buffer

    def close(self):
        if getattr(self, "h", None):
            self.L.cl_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def size(self):
        return self.L.cl_ensemble_size(self.h)

    def step(self, n, h=None):
        rc = self.L.cl_step(self.h, n) if h is None else self.L.cl_step_h(self.h, n, h)
        _check(self.L, self.h, rc, "cl_step")

    def sync(self):
        _check(self.L, self.h, self.L.cl_sync(self.h), "cl_sync")

    def energies(self, lat, allow_nonfinite=False):
        e = Energies()
        rc = self.L.cl_lattice_energies(self.h, lat, ctypes.byref(e))
        if not (allow_nonfinite and rc == CL_ENONFINITE):
            _check(self.L, self.h, rc, "cl_lattice_energies")
        return e.as_dict()

    def get(self, lat, field, what=0):
        N = self.Ns[lat]
        out = np.empty(N ** 3, dtype=np.float64)
        _check(self.L, self.h, self.L.cl_lattice_get_state(self.h, lat, field, what, _dp(out)),
               "cl_lattice_get_state")
        return out.reshape(N, N, N)  # [z][y][x]

    def set(self, lat, field, what, arr):
        N = self.Ns[lat]
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        if a.size != N ** 3:
            raise ValueError("need %d values" % N ** 3)
        _check(self.L, self.h, self.L.cl_lattice_set_state(self.h, lat, field, what, _dp(a)),
               "cl_lattice_set_state")

    def scalars(self, lat):
        e, a, b = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.L, self.h, self.L.cl_lattice_scalars(self.h, lat, ctypes.byref(e), ctypes.byref(a),
                                                         ctypes.byref(b)), "cl_lattice_scalars")
        return e.value, a.value, b.value

    def tile(self, lat):
        n, by, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.L, self.h, self.L.cl_lattice_tile(self.h, lat, ctypes.byref(n), ctypes.byref(by),
                                                      ctypes.byref(st)), "cl_lattice_tile")
        return n.value, by.value, st.value

    def spectrum_mean(self, lats, field, what=0, dk_bin=1.0):
        cap = 4096
        k = np.zeros(cap)
        d = np.zeros(cap)
        m = np.zeros(cap, dtype=np.int64)
        nb = ctypes.c_int()
        ls = (ctypes.c_int * len(lats))(*[int(x) for x in lats])
        rc = self.L.cl_ensemble_spectrum(self.h, ls, len(lats), field, what, dk_bin, _dp(k), _dp(d),
                                         m.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), cap,
                                         ctypes.byref(nb))
        _check(self.L, self.h, rc, "cl_ensemble_spectrum")
        n = nb.value
        return k[:n].copy(), d[:n].copy(), m[:n].copy()

    def launches(self):
        return int(self.L.cl_kernel_launches(self.h))

    def enable_pass_timing(self, on=True):
        _check(self.L, self.h, self.L.cl_enable_pass_timing(self.h, 1 if on else 0), "timing")

    def pass_timing(self, reset=False):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        _check(self.L, self.h, self.L.cl_pass_timing(self.h, ctypes.byref(ms), ctypes.byref(n),
                                                     1 if reset else 0), "timing")
        return ms.value, n.value
