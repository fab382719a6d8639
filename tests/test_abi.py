"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/srbe.h declares; the binding wraps exactly those.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2509_24742_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "srbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(srbe_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for required in ["srbe_create", "srbe_set_positions", "srbe_sample_k", "srbe_forces",
                     "srbe_solve_electrode_charges", "srbe_step", "srbe_set_electrode", "srbe_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2509_24742_gb300 import srbe
    assert sorted(srbe.EXPORTS) == declared()


def test_library_is_built_for_sm_103a():
    # every object was compiled with the sm_103a gencode only
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    for src in B.SOURCES:
        assert os.path.exists(os.path.join(B.OUT, src.replace(".cu", ".o")))


def test_create_rejects_bad_arguments(lib):
    """Argument checks run before any device work."""
    from paper_2509_24742_gb300 import srbe
    L = srbe.load()
    h = ctypes.c_void_p()
    box = (ctypes.c_double * 3)(2.0, 2.0, -1.0)
    assert L.srbe_create(box, 3.5, 0.05, 1.2, 10, 2, 0.0, 1.0, ctypes.byref(h)) == srbe.SRBE_EINVAL
    box = (ctypes.c_double * 3)(2.0, 2.0, 12.0)
    assert L.srbe_create(box, 3.5, 0.05, 1.2, -1, 2, 0.0, 1.0, ctypes.byref(h)) == srbe.SRBE_EINVAL
    assert L.srbe_create(box, 0.0, 0.05, 1.2, 10, 2, 0.0, 1.0, ctypes.byref(h)) == srbe.SRBE_EINVAL
    assert L.srbe_destroy(None) == srbe.SRBE_OK


def test_no_silent_cpu_path_without_gpu():
    """Without a GPU the library reports a CUDA error instead of computing anything."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_24742_gb300 import srbe
    with pytest.raises(srbe.SrbeError) as e:
        srbe.Context((2.0, 2.0, 12.0), 3.5, 0.05, 1.2, 10, 2)
    assert e.value.code == srbe.SRBE_ECUDA
