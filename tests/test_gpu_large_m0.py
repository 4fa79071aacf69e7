"""Orders above 16 functions per cell: the k-point solves take a whole warp per k-point there
(half a warp up to 16).  End-to-end spectra on both Gram routes, the k-point eigensolve on the
oracle's blocks, Bloch eigenvectors and the allocation-free entry point, for m0 = 20 and 32."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import check_eigenvalues

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3839_gb300 import build, lhf as B

    build.build()
    return B


@pytest.fixture(scope="module")
def ctx(lhf):
    c = lhf.Context(0)
    yield c
    c.close()


CASES = {
    "m0_20": lambda: W.tube(8, seed=21, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=5, m0_pshell=5, lo=0.3, hi=8.0),
    "m0_32": lambda: W.tube(6, seed=22, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=2, m0_pshell=10, lo=0.4, hi=8.0),
}


def to_dev(Z):
    return torch.from_numpy(np.ascontiguousarray(np.stack([Z.real, Z.imag], -1))).cuda()


@pytest.mark.parametrize("name", sorted(CASES))
def test_large_m0_spectra_both_routes(ctx, oracle_mod, lhf, name):
    cfg = CASES[name]()
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    Hr, Sr = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hr), oracle_mod.block_dft(Sr)
    ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
    for prec in (lhf.FP64, lhf.MIXED):
        eig = torch.empty((sz["n_kpoints"], sz["m0"]), dtype=torch.float64, device="cuda")
        ks = torch.empty((sz["n_kpoints"],), dtype=torch.int32, device="cuda")
        ctx.bloch_spectra([cfg], eig, ks, prec)
        ctx.sync()
        assert np.array_equal(ks.cpu().numpy(), st)
        worst, ratio = check_eigenvalues(eig.cpu().numpy(), ref, Hb, Sb, Hr, Sr, status=st)
        assert ratio <= 1.0, (prec, worst, ratio)


@pytest.mark.parametrize("name", sorted(CASES))
def test_large_m0_eigensolve_vectors_and_noalloc(ctx, oracle_mod, lhf, name):
    cfg = CASES[name]()
    ctx.setup(cfg)
    Hr, Sr = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hr), oracle_mod.block_dft(Sr)
    K, m0 = int(np.prod(cfg["L"])), Hb.shape[-1]
    ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
    hb, sb = to_dev(Hb), to_dev(Sb)
    eig = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    ctx.k_point_eigensolve(hb, sb, eig)
    vecs = torch.empty((K, m0, m0, 2), dtype=torch.float64, device="cuda")
    eig2 = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    ctx.k_point_eigenvectors(hb, sb, eig2, vecs)
    ctx.sync()
    for e in (eig, eig2):
        worst, ratio = check_eigenvalues(e.cpu().numpy(), ref, Hb, Sb, status=st)
        assert ratio <= 1.0, (worst, ratio)
    v = vecs.cpu().numpy()
    v = v[..., 0] + 1j * v[..., 1]
    Sk = Sb.reshape(-1, m0, m0)
    Sk = 0.5 * (Sk + np.conj(np.transpose(Sk, (0, 2, 1))))
    for k in range(K):
        n = m0 - st[k]
        U = v[k, :n].T
        assert np.abs(U.conj().T @ Sk[k] @ U - np.eye(n)).max() < 1e-8
    e3 = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    lhf.k_point_eigensolve_noalloc(cfg["L"], m0, hb, sb, e3)
    torch.cuda.synchronize()
    worst, ratio = check_eigenvalues(e3.cpu().numpy(), ref, Hb, Sb, status=st)
    assert ratio <= 1.0, (worst, ratio)
