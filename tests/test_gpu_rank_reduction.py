"""Rank reduction of the lattice-summed potential (lhf_set_rank_reduction, FP64 route, (L,1,1)
lattices): the reduced blocks against the oracle's unreduced blocks within the stated per-entry
bound rho ||Q_j,mu,nu||_2 R_tot (rho the largest residual row norm the pivoted Gram-Schmidt
leaves out, Q the cell fold of the product row, computed here from the oracle's basis samples)
plus FP64 rounding; overlap
blocks unchanged; the reduced rank reported; spectra of the full-size tube; the mixed route and
graphs unaffected."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import block_rel_err, check_eigenvalues

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
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


CASES = {
    "periodic_8": W.periodic_8,
    "tube_16_m16": lambda: W.tube(16, seed=11, n_c=32, n_perp=64, half_width=8.0),
    "chain_64": lambda: W.chain(64),
}


def _blocks(ctx, cfg):
    ctx.setup(cfg)
    L, m0 = cfg["L"][0], len(cfg["alpha"])
    H = torch.empty((L, 1, 1, m0, m0), dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    ctx.assemble_core_hamiltonian(H, S)
    ctx.sync()
    return H.cpu().numpy()[:, 0, 0], S.cpu().numpy()[:, 0, 0]


def _fold_norms(oracle_mod, cfg):
    """||Q_j,mu,nu||_2 for every block j and entry: Q(c) = sum_p g_mu,j g_nu,0 at node c + p n_c."""
    L, nc = cfg["L"][0], cfg["n_cell"][0]
    g0 = oracle_mod.basis_samples(cfg, 0, 0)
    m0 = g0.shape[0]
    out = np.empty((L, m0, m0))
    for j in range(L):
        gj = oracle_mod.basis_samples(cfg, 0, j)
        P = gj[:, None, :] * g0[None, :, :]
        Q = P.reshape(m0, m0, L, nc).sum(axis=2)
        out[j] = np.sqrt((Q ** 2).sum(axis=2))
    return out


@pytest.mark.parametrize("eps", [1e-12, 1e-7])
@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_blocks_within_the_stated_bound(lhf, oracle_mod, name, eps):
    cfg = CASES[name]()
    ctx = lhf.Context(0)
    try:
        ctx.set_rank_reduction(eps)
        ctx.setup(cfg)
        info = ctx.rank_reduction_info()
        H, S = _blocks(ctx, cfg)
    finally:
        ctx.close()
    Hr, Sr = oracle_mod.core_blocks(cfg)
    Hr, Sr = Hr[:, 0, 0], Sr[:, 0, 0]
    m0 = H.shape[-1]
    assert info["rank_in"] == len(cfg["Z"]) * cfg["R"]
    assert 1 <= info["rank_out"] < info["rank_in"]
    assert info["dropped"] <= eps * info["largest"]
    assert block_rel_err(S, Sr, m0) <= 1e-12  # the overlap does not involve the potential
    bound = info["dropped"] * _fold_norms(oracle_mod, cfg) * info["rank_in"]
    noise = 1e-12 * np.abs(Hr).reshape(len(Hr), -1).max(axis=1)[:, None, None]
    err = np.abs(H - Hr)
    assert np.all(err <= bound + noise), float((err - bound - noise).max())


def test_full_size_tube_rank_and_spectrum(lhf, oracle_mod):
    cfg = W.tube_256()
    ctx = lhf.Context(0)
    try:
        eig0 = torch.empty((256, 16), dtype=torch.float64, device="cuda")
        ctx.setup(cfg)
        ctx.bloch_spectra([cfg], eig0, None, lhf.FP64)
        ctx.set_rank_reduction(1e-12)
        ctx.setup(cfg)
        info = ctx.rank_reduction_info()
        eig1 = torch.empty_like(eig0)
        ks = torch.empty((256,), dtype=torch.int32, device="cuda")
        ctx.bloch_spectra([cfg], eig1, ks, lhf.FP64)
        ctx.sync()
        # the mixed route ignores the setting: bitwise equal to a context without it
        em = torch.empty_like(eig0)
        ctx.bloch_spectra([cfg], em, None, lhf.MIXED)
        ctx.sync()
    finally:
        ctx.close()
    ref_ctx = lhf.Context(0)
    try:
        em0 = torch.empty_like(eig0)
        ref_ctx.bloch_spectra([cfg], em0, None, lhf.MIXED)
        ref_ctx.sync()
    finally:
        ref_ctx.close()
    assert info["rank_in"] == 64 and info["rank_out"] <= 40, info
    Hr, Sr = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hr), oracle_mod.block_dft(Sr)
    ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
    assert np.array_equal(ks.cpu().numpy(), st)
    worst, ratio = check_eigenvalues(eig1.cpu().numpy(), ref, Hb, Sb, Hr, Sr, status=st)
    assert ratio <= 1.0, (worst, ratio)
    assert torch.equal(em, em0)
