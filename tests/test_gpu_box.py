"""Parity of the open-box route (dense matrices of an (L,1,1) lattice with open ends, the
paper's box case of Sec. 3 and Table 4.1's full eigensolver) with the FP64 oracle: direction-0
factors between cell pairs, the dense H and S, and the dense generalized eigensolve.

Tolerances: matrix entries 1e-12 of the (cell, cell) block max (as for the periodic blocks);
eigenvalues by the first-order perturbation bound of tests/_numerics.py."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import check_dense_eigenvalues

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


def dev(shape, dtype=torch.float64):
    return torch.empty(shape, dtype=dtype, device="cuda")


BOXES = {
    "box_4": lambda: W.box_64(seed=21, L=4, n_perp=64),
    "box_7": lambda: W.box_64(seed=22, L=7, n_perp=48),
    "box_2": lambda: W.box_64(seed=23, L=2, n_perp=40),
}


def dense_blocks_err(X, Xref, m0):
    """max over (cell, cell) blocks of max|X - Xref| / max|Xref| (0/0 counts as 0)."""
    N = X.shape[0]
    L = N // m0
    Xb = X.reshape(L, m0, L, m0).transpose(0, 2, 1, 3).reshape(L * L, -1)
    Rb = Xref.reshape(L, m0, L, m0).transpose(0, 2, 1, 3).reshape(L * L, -1)
    num = np.abs(Xb - Rb).max(axis=1)
    den = np.abs(Rb).max(axis=1)
    return float(np.where(den == 0, num, num / np.where(den == 0, 1.0, den)).max())


def gpu_dense(ctx, cfg):
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    assert sz["periodic"] == 0
    N = sz["n_basis"]
    H, S = dev((N, N)), dev((N, N))
    ctx.assemble_core_hamiltonian(H, S)
    ctx.sync()
    return H.cpu().numpy(), S.cpu().numpy()


@pytest.mark.parametrize("name", ["box_4", "box_2"])
def test_box_basis_and_potential_factors(ctx, oracle_mod, name):
    cfg = BOXES[name]()
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    for l in range(3):
        G = dev((sz["m0"], cfg["n"][l]))
        ctx.basis_factors(l, G)
        ref = oracle_mod.basis_samples(cfg, l, 0)
        assert np.abs(G.cpu().numpy() - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())
        nv = sz["n_potential"][l]
        V = dev((sz["rank"], nv))
        ctx.potential_factors(l, V)
        vref = oracle_mod.potential_factors(cfg, l)[:, :nv]
        rel = np.abs(V.cpu().numpy() - vref).max(axis=1) / np.abs(vref).max(axis=1)
        assert rel.max() <= 1e-13, (l, rel.max())


@pytest.mark.parametrize("name", ["box_4", "box_7"])
def test_box_direction0_factors(ctx, oracle_mod, name):
    cfg = BOXES[name]()
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    m0, Rt, L0 = sz["m0"], sz["rank"], cfg["L"][0]
    J = sz["window"][0]
    C = dev((L0, J, Rt + 2, m0, m0))
    dlo = ctx.gram_factors(0, C)
    C = C.cpu().numpy()
    V = oracle_mod.potential_factors(cfg, 0)
    checked = 0
    for p in range(L0):
        for dd in range(J):
            q = p + dlo + dd
            if not 0 <= q < L0:
                continue
            Cr, K, M = oracle_mod.gram_1d(cfg, 0, p, q, V)
            big = np.abs(Cr).max()
            for r in range(Rt):
                den = np.abs(Cr[r]).max()
                assert np.abs(C[p, dd, r] - Cr[r]).max() <= 1e-12 * den + 1e-40 * big, (p, dd, r)
            assert np.abs(C[p, dd, Rt] - K).max() <= 1e-12 * max(np.abs(K).max(), 1e-300)
            assert np.abs(C[p, dd, Rt + 1] - M).max() <= 1e-12 * max(np.abs(M).max(), 1e-300)
            checked += 1
    assert checked >= L0
    # pairs outside the window are exact zeros in the oracle
    for p in range(L0):
        for q in range(L0):
            if not dlo <= q - p < dlo + J:
                Cr, K, M = oracle_mod.gram_1d(cfg, 0, p, q, V)
                assert np.all(Cr == 0) and np.all(K == 0) and np.all(M == 0)


@pytest.mark.parametrize("name", sorted(BOXES))
def test_box_dense_matrices(ctx, oracle_mod, name):
    cfg = BOXES[name]()
    H, S = gpu_dense(ctx, cfg)
    Hr, Sr = oracle_mod.core_dense(cfg)
    m0 = len(cfg["alpha"])
    assert dense_blocks_err(H, Hr, m0) <= 1e-12
    assert dense_blocks_err(S, Sr, m0) <= 1e-12
    # (cell, cell) blocks without overlapping supports are exact zeros on both sides
    L = H.shape[0] // m0
    Hb = np.abs(H).reshape(L, m0, L, m0).max(axis=(1, 3))
    Rb = np.abs(Hr).reshape(L, m0, L, m0).max(axis=(1, 3))
    assert np.all(Hb[Rb == 0] == 0)


@pytest.mark.parametrize("name", sorted(BOXES))
def test_box_dense_eigensolve_same_input(ctx, oracle_mod, name):
    cfg = BOXES[name]()
    H, S = gpu_dense(ctx, cfg)
    N = H.shape[0]
    eig = dev((N,))
    Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
    ctx.dense_eigensolve(Hd, Sd, N, eig)
    ctx.sync()
    ref = oracle_mod.dense_gen_eigenvalues(H, S)
    worst, ratio = check_dense_eigenvalues(eig.cpu().numpy(), ref, H, S)
    assert ratio <= 1.0, (worst, ratio)


@pytest.mark.parametrize("name", sorted(BOXES))
def test_box_spectrum_end_to_end(ctx, oracle_mod, name):
    cfg = BOXES[name]()
    N = len(cfg["alpha"]) * cfg["L"][0]
    eig = dev((N,))
    ks = dev((cfg["L"][0],), torch.int32)
    ctx.bloch_spectra([cfg], eig, ks)
    ctx.sync()
    Hr, Sr = oracle_mod.core_dense(cfg)
    ref = oracle_mod.dense_gen_eigenvalues(Hr, Sr)
    H, S = gpu_dense(ctx, cfg)
    worst, ratio = check_dense_eigenvalues(eig.cpu().numpy(), ref, Hr, Sr, dH=H - Hr, dS=S - Sr)
    assert ratio <= 1.0, (worst, ratio)
    assert np.all(ks.cpu().numpy() == 0)


def test_box_and_periodic_in_one_batch(ctx, oracle_mod):
    box = BOXES["box_4"]()
    per = W.periodic_8()
    n_box = len(box["alpha"]) * box["L"][0]
    n_per = len(per["alpha"]) * per["L"][0]
    eig = dev((n_per + n_box,))
    ctx.bloch_spectra([per, box], eig)
    ctx.sync()
    got = eig.cpu().numpy()
    e1 = dev((n_per,))
    ctx.bloch_spectra([per], e1)
    e2 = dev((n_box,))
    ctx.bloch_spectra([box], e2)
    ctx.sync()
    assert np.array_equal(got[:n_per], e1.cpu().numpy())
    assert np.array_equal(got[n_per:], e2.cpu().numpy())


@pytest.mark.parametrize("N", [1, 2, 3, 37, 300])
def test_dense_eigensolve_random_pencils(ctx, oracle_mod, N):
    rng = np.random.default_rng(100 + N)
    A = rng.standard_normal((N, N))
    S = A @ A.T / N + np.eye(N) * 0.5
    B = rng.standard_normal((N, N))
    H = (B + B.T) * 3.0
    eig = dev((N,))
    Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
    ctx.dense_eigensolve(Hd, Sd, N, eig)
    ctx.sync()
    ref = oracle_mod.dense_gen_eigenvalues(H, S)
    worst, ratio = check_dense_eigenvalues(eig.cpu().numpy(), ref, H, S)
    assert ratio <= 1.0, (worst, ratio)
    assert np.all(np.diff(eig.cpu().numpy()) >= 0)


def test_dense_eigensolve_not_positive_definite(ctx, lhf):
    N = 16
    S = np.eye(N)
    S[5, 5] = -1.0
    H = np.eye(N)
    eig = dev((N,))
    Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
    ctx.dense_eigensolve(Hd, Sd, N, eig)
    with pytest.raises(lhf.LhfError) as ei:
        ctx.sync()
    assert ei.value.status == lhf.LHF_ERR_NOT_SPD
    assert np.all(np.isnan(eig.cpu().numpy()))
    # the context stays usable
    S[5, 5] = 1.0
    Sd = torch.from_numpy(S).cuda()
    ctx.dense_eigensolve(Hd, Sd, N, eig)
    ctx.sync()
    assert np.allclose(eig.cpu().numpy(), 1.0, atol=1e-14)


@pytest.mark.slow
def test_box_64_full_size(ctx, oracle_mod):
    """The (64,1,1) box at full size: N_b = 512, n1 = 3712 (padded), n2 = n3 = 320, R = 32."""
    cfg = W.box_64()
    H, S = gpu_dense(ctx, cfg)
    Hr, Sr = oracle_mod.core_dense(cfg)
    assert dense_blocks_err(H, Hr, 8) <= 1e-12
    assert dense_blocks_err(S, Sr, 8) <= 1e-12
    N = H.shape[0]
    eig = dev((N,))
    ctx.bloch_spectra([cfg], eig)
    ctx.sync()
    ref = oracle_mod.dense_gen_eigenvalues(Hr, Sr)
    worst, ratio = check_dense_eigenvalues(eig.cpu().numpy(), ref, Hr, Sr, dH=H - Hr, dS=S - Sr)
    assert ratio <= 1.0, (worst, ratio)
