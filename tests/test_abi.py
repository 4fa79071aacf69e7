"""The C-ABI library loads and exports every entry point include/lhf.h declares (no GPU
needed: nothing is called), and the binding fails loudly without the library."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lhf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lhf_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1408_3839_gb300 import build

    return build.build()


def test_header_declares_the_path_calls():
    names = declared_functions()
    for required in ["lhf_create", "lhf_lattice_setup", "lhf_basis_setup", "lhf_grid_setup",
                     "lhf_assemble_core_hamiltonian", "lhf_circulant_fft", "lhf_k_point_eigensolve",
                     "lhf_bloch_spectra", "lhf_dense_eigensolve"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib_path):
    import paper_1408_3839_gb300.lhf as B

    lib = B.load()
    for n in declared_functions():
        assert getattr(lib, n).argtypes is not None, n


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    import paper_1408_3839_gb300.lhf as B

    monkeypatch.setattr(B, "_lib", None)
    monkeypatch.setattr(B, "HERE", str(tmp_path))
    with pytest.raises(RuntimeError, match="no CPU path"):
        B.load()
