"""CPU-only checks of the C ABI library: it builds for sm_103a, loads, and
exports every entry point that include/cl.h declares.  No compute call is
made (there is no GPU here)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "cl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(cl_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built_lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    import paper_2102_01031_gb300 as P
    return P.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("cl_init", "cl_step", "cl_energies", "cl_gauss_constraint", "cl_spectrum", "cl_free",
              "cl_get_state", "cl_set_state", "cl_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    import paper_2102_01031_gb300 as P
    assert sorted(P.EXPORTS) == sorted(n for n in declared_symbols())


def test_build_targets_sm_103a_only():
    from paper_2102_01031_gb300 import builder
    assert builder.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_init_without_gpu_fails_loudly(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2102_01031_gb300 as P
    with pytest.raises(P.ClError):
        P.Lattice(P.MODEL_LPHI4, 32, 0.5, 1.0, 1, P.make_params())


@pytest.mark.parametrize("model,N,kIR,kw,status", [
    (7, 16, 0.5, {}, 1),                              # unknown model
    (1, 20, 0.5, {}, 1),                              # N not a multiple of 8
    (1, 1024, 0.5, {}, 1),                            # N above 512
    (1, 16, 0.0, {}, 1),                              # kIR must be positive
    (1, 16, 0.5, dict(precision=5), 1),
    (1, 16, 0.5, dict(integrator=3), 1),
    (3, 16, 0.5, dict(gQ=0.0), 1),                    # U(1) needs a coupling
    (4, 16, 0.5, dict(gQB=0.0), 1),                   # the doublet needs an SU(2) coupling
    (4, 24, 0.5, {}, 7),                              # doublet tiles need N % 16 == 0
    (1, 16, 0.5, dict(tile_by=-1), 1),
])
def test_init_refuses_bad_arguments_before_the_device(built_lib, model, N, kIR, kw, status):
    """cl_init checks its arguments before any CUDA call, so these are refused
    here without a GPU (CL_EINVAL = 1, CL_EUNSUPPORTED = 7), with a message."""
    import paper_2102_01031_gb300 as P
    with pytest.raises(P.ClError) as e:
        P.Lattice(model, N, kIR, 1.0, 1, P.make_params(**kw))
    assert e.value.status == status
    assert "cl_init" in str(e.value) and len(str(e.value)) > 20


def test_init_without_a_gpu_fails_loudly(built_lib):
    """A valid request on a machine without a GPU ends in CL_ECUDA (3), not in a
    CPU fallback."""
    import paper_2102_01031_gb300 as P
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(P.ClError) as e:
        P.Lattice(1, 16, 0.5, 1.0, 1, P.make_params())
    assert e.value.status == P.CL_ECUDA
