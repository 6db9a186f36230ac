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
