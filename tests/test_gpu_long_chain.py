"""Long (L,1,1) chains, L > 4096 (the lattice sizes of the paper's Table 4.1 reach 2^15 cells with
m0 = 4): the block DFT runs as a four-step transform (L = A B, two passes of lengths A and B with
twiddles between them).  Checked: sampled first-column blocks against the oracle's per-entry 1D
factors, the GPU DFT against numpy's FFT of the GPU's own blocks (powers of two and a composite
length with direct sums inside), and the k-point spectra against the oracle's eigensolver on
those transformed blocks."""

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
def ctx(lhf):
    c = lhf.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


def _blocks_and_dft(ctx, cfg):
    ctx.setup(cfg)
    L, m0 = cfg["L"][0], len(cfg["alpha"])
    H = torch.empty((L, 1, 1, m0, m0), dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    ctx.assemble_core_hamiltonian(H, S)
    Hb = torch.empty(H.shape + (2,), dtype=torch.float64, device="cuda")
    Sb = torch.empty_like(Hb)
    ctx.circulant_fft(H, S, Hb, Sb)
    ctx.sync()
    to_c = lambda X: (lambda a: a[..., 0] + 1j * a[..., 1])(X.cpu().numpy())
    return H.cpu().numpy(), S.cpu().numpy(), to_c(Hb), to_c(Sb)


@pytest.mark.parametrize("L", [8192, 6000, 32768])
def test_four_step_dft_of_long_chains(ctx, L):
    H, S, Hb, Sb = _blocks_and_dft(ctx, W.chain(L))
    for X, Xb in ((H, Hb), (S, Sb)):
        ref = np.fft.fft(X, axis=0)  # sum_j X_j exp(-2 pi i j kappa / L)
        scale = np.abs(X).sum(axis=0).max()
        assert np.abs(Xb - ref).max() <= 1e-13 * scale, np.abs(Xb - ref).max() / scale


def test_long_chain_blocks_against_oracle_samples(ctx, oracle_mod):
    L = 8192
    cfg = W.chain(L)
    H, S, _, _ = _blocks_and_dft(ctx, cfg)
    c = oracle_mod.rank_coefficients(cfg)
    V = [oracle_mod.potential_factors(cfg, l) for l in range(3)]
    t1 = oracle_mod.gram_1d(cfg, 1, 0, 0, V[1])
    t2 = oracle_mod.gram_1d(cfg, 2, 0, 0, V[2])
    for j in (0, 1, 3, L - 1):
        C0, K0, M0 = oracle_mod.gram_1d(cfg, 0, j, 0, V[0])
        C1, K1, M1 = t1
        C2, K2, M2 = t2
        Sj = M0 * M1 * M2
        Hj = 0.5 * (K0 * M1 * M2 + M0 * K1 * M2 + M0 * M1 * K2) - np.einsum("r,rij,rij,rij->ij", c, C0, C1, C2)
        assert block_rel_err(H[j, 0, 0], Hj, 4) <= 1e-12, j
        assert block_rel_err(S[j, 0, 0], Sj, 4) <= 1e-12, j


@pytest.mark.parametrize("L", [8192, 32768])
def test_long_chain_spectra(ctx, oracle_mod, L):
    cfg = W.chain(L)
    H, S, _, _ = _blocks_and_dft(ctx, cfg)
    Hb, Sb = np.fft.fft(H, axis=0), np.fft.fft(S, axis=0)
    ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
    ctx.setup(cfg)
    eig = torch.empty((L, 4), dtype=torch.float64, device="cuda")
    ks = torch.empty((L,), dtype=torch.int32, device="cuda")
    ctx.bloch_spectra([cfg], eig, ks)
    ctx.sync()
    assert np.array_equal(ks.cpu().numpy(), st)
    worst, ratio = check_eigenvalues(eig.cpu().numpy(), ref, Hb, Sb, H, S, status=st)
    assert ratio <= 1.0, (worst, ratio)
