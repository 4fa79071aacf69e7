"""The lowest eigenvalues of open (L,1,1) boxes without the dense eigensolve
(lhf_box_lowest_eigenvalues: block LOBPCG on the banded box matrices, block-circulant
preconditioner): against the oracle's dense generalized eigenvalues of the same box (small L), the
GPU dense solver (L = 64 and 256) to 1e-10 of the spectrum's scale, and, beyond the dense limit
(L = 2048, N_b = 16384), convergence, tolerance consistency and determinism."""

import numpy as np
import pytest

import lhf_workloads as W

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


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


def _lobpcg(ctx, cfg, n_ev, tol=1e-8):
    eig = torch.empty(n_ev, dtype=torch.float64, device="cuda")
    st, it, res = ctx.box_lowest_eigenvalues(cfg, n_ev, eig, tol=tol, max_iter=300)
    return eig.cpu().numpy(), it, res


@pytest.mark.parametrize("L,n_perp,n_ev", [(8, 48, 6), (16, 64, 12)])
def test_lowest_box_eigenvalues_match_the_oracle(ctx, oracle_mod, L, n_perp, n_ev):
    cfg = W.box_64(seed=30 + L, L=L, n_perp=n_perp)
    got, it, res = _lobpcg(ctx, cfg, n_ev)
    H, S = oracle_mod.core_dense(cfg)
    ref = oracle_mod.dense_gen_eigenvalues(H, S)[:n_ev]
    assert res <= 1e-8 and it >= 1
    assert np.all(np.diff(got) >= 0)
    assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (got - ref, it)


@pytest.mark.parametrize("L", [64, 256])
def test_lowest_box_eigenvalues_match_the_dense_solver(ctx, L):
    cfg = W.box_64(seed=40 + L, L=L, n_perp=64)
    n_ev = 16
    got, it, res = _lobpcg(ctx, cfg, n_ev)
    N = len(cfg["alpha"]) * L
    full = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.bloch_spectra([cfg], full)
    ctx.sync()
    ref = full.cpu().numpy()[:n_ev]
    assert res <= 1e-8
    assert np.abs(got - ref).max() <= 1e-10 * max(1.0, np.abs(ref).max()), (got - ref, it)


def test_box_beyond_the_dense_limit(ctx, lhf):
    # N_b = 8 x 2048 = 16384 (the dense solver stops at 8192): converges; the Ritz values are
    # reproducible and do not depend on the tolerance beyond its own size
    cfg = W.box_64(seed=7, L=2048, n_perp=48)
    with pytest.raises(lhf.LhfError):
        ctx.bloch_spectra([cfg], torch.empty(8 * 2048, dtype=torch.float64, device="cuda"))
    a, it_a, res_a = _lobpcg(ctx, cfg, 8, tol=1e-6)
    b, it_b, res_b = _lobpcg(ctx, cfg, 8, tol=1e-8)
    assert res_a <= 1e-6 and res_b <= 1e-8 and it_b >= it_a
    assert np.all(np.diff(b) >= 0)
    assert np.abs(a - b).max() <= 1e-8 * max(1.0, np.abs(b).max())
    c, _, _ = _lobpcg(ctx, cfg, 8, tol=1e-8)
    assert np.array_equal(b, c)  # deterministic


def test_invalid_requests_are_refused(ctx, lhf):
    eig = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(lhf.LhfError) as ei:
        ctx.box_lowest_eigenvalues(W.periodic_8(), 4, eig)
    assert ei.value.status == lhf.LHF_ERR_ARG
    with pytest.raises(lhf.LhfError) as ei:
        ctx.box_lowest_eigenvalues(W.box_64(seed=1, L=8, n_perp=48), 0, eig)
    assert ei.value.status == lhf.LHF_ERR_ARG
