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


def test_batched_descriptors_match_single_descriptors():
    """The vectorised descriptor array (binding) carries the same values as the per-system ctypes
    descriptors: scalar fields byte for byte, and the pointed-to host arrays element for element."""
    import numpy as np

    import lhf_workloads as W
    import paper_1408_3839_gb300.lhf as B

    cfgs = [W.tube_256(3000), W.box_64(L=4, n_perp=64), W.cubic_32(seed=15, L=3, n_c=10), W.periodic_8()]
    batch = B._Batch(cfgs)
    arr = ctypes.cast(batch.ptr(), ctypes.POINTER(B.lhf_system_desc * len(cfgs))).contents
    for cfg, got in zip(cfgs, arr):
        ref = B._Desc(cfg).system
        assert bytes(got.grid) == bytes(ref.grid)
        for f in ("L", "b", "periodic", "K_sum"):
            assert list(getattr(got.lattice, f)) == list(getattr(ref.lattice, f))
        assert got.lattice.M0 == ref.lattice.M0 and got.basis.m0 == ref.basis.m0 and got.basis.rho == ref.basis.rho
        M0, m0 = ref.lattice.M0, ref.basis.m0
        for name, n in (("Z", M0), ("a", 3 * M0)):
            assert [getattr(got.lattice, name)[i] for i in range(n)] == [getattr(ref.lattice, name)[i] for i in range(n)]
        for name, n in (("kind", m0), ("alpha", m0), ("centre", 3 * m0)):
            assert [getattr(got.basis, name)[i] for i in range(n)] == [getattr(ref.basis, name)[i] for i in range(n)]
        if cfg.get("Z_cell") is None:
            assert not bool(got.lattice.Z_cell)
        else:
            n = len(cfg["Z_cell"]) * M0
            assert [got.lattice.Z_cell[i] for i in range(n)] == list(np.ravel(cfg["Z_cell"]))


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every descriptor struct of the binding has the size and field offsets of include/lhf.h
    (compiled here by the host C compiler): a field added on one side only fails on the CPU."""
    import shutil
    import subprocess

    import paper_1408_3839_gb300.lhf as B

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = ["lhf_lattice_desc", "lhf_basis_desc", "lhf_grid_desc", "lhf_system_desc", "lhf_sizes"]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "lhf.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for name, _ in getattr(B, st)._fields_:
            lines.append(f'  printf("{st} {name} %zu\\n", offsetof({st}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    for row in filter(None, out):
        st, field, value = row.split()
        cls = getattr(B, st)
        got = ctypes.sizeof(cls) if field == "size" else getattr(cls, field).offset
        assert got == int(value), (st, field, got, value)
