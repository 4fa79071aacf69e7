"""The separable k-space route on the GPU (lhf_kspace_blocks; Theorem 2.5, Prop. 4.2) against the
oracle's direct DFT of its assembled blocks, and against the GPU's own real-space route
(assembly + block DFT) on both Gram precisions; then the k-point spectrum from its blocks."""

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


def small_tube(L, seed, **kw):
    base = dict(n_c=32, n_perp=64, half_width=8.0, M0=2, m0_s=4, m0_pshell=4, lo=0.04, hi=30.0)
    base.update(kw)
    return W.tube(L, seed=seed, **base)


CASES = {
    "periodic_8": lambda: W.periodic_8(),
    "tube_16_m16": lambda: small_tube(16, seed=11),
    "tube_12_odd_window": lambda: small_tube(12, seed=12, lo=0.3, K_sum=7),
    "tube_24_windowed": lambda: small_tube(24, seed=13, lo=0.5, hi=20.0, n_c=24),
    "tube_9_m5_odd": lambda: W.tube(9, seed=14, n_c=20, n_perp=48, half_width=6.0, M0=1, m0_s=2,
                                    m0_pshell=1, lo=0.2, hi=9.0),
    "cubic_3": lambda: W.cubic_32(seed=15, L=3, n_c=10),
    "slab_4x3": lambda: W.make_system(
        L=[4, 3, 1], b=[2.0, 2.0, 8.0], periodic=[1, 1, 0], n_cell=[16, 16, 64], h=[0.125] * 3,
        x0=[0.0, 0.0, -4.0], cell0=[0.0, 0.0, -4.0], Z=[1.0], a=[[1.1, 0.9, 0.2]], kind=[0, 1, 3],
        alpha=[0.7, 1.5, 0.9], centre=[[1.1, 0.9, 0.2]] * 3, R=20, u0=-6.8657, du=0.557),
}


def kspace(ctx, cfg, precision=0):
    ctx.setup(cfg)
    L, m0 = cfg["L"], ctx.query_sizes()["m0"]
    Hb = torch.empty((L[0], L[1], L[2], m0, m0, 2), dtype=torch.float64, device="cuda")
    Sb = torch.empty_like(Hb)
    ctx.kspace_blocks(Hb, Sb, precision)
    return Hb, Sb


def real_space(ctx, cfg, precision=0):
    ctx.setup(cfg)
    L, m0 = cfg["L"], ctx.query_sizes()["m0"]
    H = torch.empty((L[0], L[1], L[2], m0, m0), dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    ctx.assemble_core_hamiltonian(H, S, precision)
    Hb = torch.empty(H.shape + (2,), dtype=torch.float64, device="cuda")
    Sb = torch.empty_like(Hb)
    ctx.circulant_fft(H, S, Hb, Sb)
    return H, S, Hb, Sb


def cplx(X):
    x = X.cpu().numpy()
    return x[..., 0] + 1j * x[..., 1]


@pytest.mark.parametrize("name", sorted(CASES))
def test_kspace_blocks_match_oracle_and_real_space_route(ctx, oracle_mod, lhf, name):
    cfg = CASES[name]()
    Hk, Sk = kspace(ctx, cfg)
    ctx.sync()
    H, S = oracle_mod.core_blocks(cfg)
    nblk = H.shape[0] * H.shape[1] * H.shape[2]
    sh, ss = np.abs(H).max(), np.abs(S).max()
    Hb_ref, Sb_ref = oracle_mod.block_dft(H), oracle_mod.block_dft(S)
    assert np.abs(cplx(Hk) - Hb_ref).max() <= 1e-12 * sh * np.sqrt(nblk) * 4
    assert np.abs(cplx(Sk) - Sb_ref).max() <= 1e-12 * ss * np.sqrt(nblk) * 4
    for prec in (lhf.FP64, lhf.MIXED):
        Hg, Sg, Hbg, Sbg = real_space(ctx, cfg, prec)
        Hk2, Sk2 = kspace(ctx, cfg, prec)
        ctx.sync()
        assert np.abs(cplx(Hk2) - cplx(Hbg)).max() <= 1e-12 * sh * np.sqrt(nblk) * 4, prec
        assert np.abs(cplx(Sk2) - cplx(Sbg)).max() <= 1e-12 * ss * np.sqrt(nblk) * 4, prec


@pytest.mark.parametrize("name", ["tube_16_m16", "cubic_3", "slab_4x3"])
def test_spectrum_from_kspace_blocks(ctx, oracle_mod, name):
    cfg = CASES[name]()
    Hk, Sk = kspace(ctx, cfg)
    K, m0 = int(np.prod(cfg["L"])), Hk.shape[-2]
    eig = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    ks = torch.empty((K,), dtype=torch.int32, device="cuda")
    ctx.k_point_eigensolve(Hk, Sk, eig, ks)
    ctx.sync()
    H, S = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(H), oracle_mod.block_dft(S)
    ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
    assert np.array_equal(ks.cpu().numpy(), st)
    worst, ratio = check_eigenvalues(eig.cpu().numpy(), ref, Hb, Sb, H, S, status=st)
    assert ratio <= 1.0, (worst, ratio)


def test_kspace_rejects_open_box(ctx, lhf):
    ctx.setup(W.box_64(L=4, n_perp=64))
    Hb = torch.empty((4, 1, 1, 8, 8, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lhf.LhfError) as ei:
        ctx.kspace_blocks(Hb, Hb)
    assert ei.value.status == lhf.LHF_ERR_UNSUPPORTED
