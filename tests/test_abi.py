"""The C ABI without a GPU: the library loads and exports every function
that include/treepm.h declares; the binding fails cleanly without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tpm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g

    g.build()
    import paper_1909_04667_gb300 as tpm

    return ctypes.CDLL(tpm.lib_path())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tpm_build_tree", "tpm_compute_forces", "tpm_pm_long_range", "tpm_create", "tpm_release"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_clean_failure_without_device(lib):
    import paper_1909_04667_gb300 as tpm

    assert tpm.version() == 2
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(tpm.TreePMError):
        tpm.Context(0)


def test_every_declared_function_has_a_binding_signature(lib):
    # without argtypes ctypes passes Python ints as 32-bit C ints: a device
    # pointer would arrive truncated
    import paper_1909_04667_gb300 as tpm

    missing = [n for n in declared_functions() if getattr(tpm._lib, n).argtypes is None]
    assert not missing, missing
