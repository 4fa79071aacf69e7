"""Bloch eigenvectors on the GPU (lhf_k_point_eigenvectors, Prop. 6.1 eq. (6.8)) against the
FP64 oracle, through the C ABI.

Both sides read the same blocks (the oracle's Hbar, Sbar), so differences are the solvers'.
Checked per k-point: k_status and eigenvalues as for lhf_k_point_eigensolve (perturbation
tolerance), S-orthonormality of the kept eigenvectors, the residual of the pencil, agreement
with the oracle's eigenvectors (the S-inner product of each GPU vector with the oracle's
eigenspace of its eigenvalue: 1 for a simple eigenvalue, the projection for a cluster; equal
vectors where the phase convention is well posed), the conjugate relation between kappa and
-kappa, and, for a small lattice, the eigenvector of the whole lattice matrix built by eq. (6.8)
against the oracle's dense matrices."""

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
    "tube_9_m5_odd": lambda: W.tube(9, seed=14, n_c=20, n_perp=48, half_width=6.0, M0=1, m0_s=2,
                                    m0_pshell=1, lo=0.2, hi=9.0),
    "cubic_3": lambda: W.cubic_32(seed=15, L=3, n_c=10),
}


def to_dev(Z):
    return torch.from_numpy(np.ascontiguousarray(np.stack([Z.real, Z.imag], -1))).cuda()


def gpu_vectors(ctx, Hb, Sb):
    K, m0 = int(np.prod(Hb.shape[:3])), Hb.shape[-1]
    eig = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    vecs = torch.empty((K, m0, m0, 2), dtype=torch.float64, device="cuda")
    ks = torch.empty((K,), dtype=torch.int32, device="cuda")
    ctx.k_point_eigenvectors(to_dev(Hb), to_dev(Sb), eig, vecs, ks)
    ctx.sync()
    v = vecs.cpu().numpy()
    return eig.cpu().numpy(), v[..., 0] + 1j * v[..., 1], ks.cpu().numpy()


def compare_with_oracle(eig, vecs, ks, oracle_mod, Hb, Sb, H=None, S=None):
    """Asserts the checks of the module docstring; returns the worst ratios to tolerance.

    Tolerances per k-point follow the conditioning of the reduced pencil: with S~ the kept
    overlap scaled to unit diagonal and kappa_S = 1 / (its smallest kept eigenvalue), the
    back-transformed vectors are S-orthonormal and satisfy U^H H U = diag(lambda) to
    c m eps kappa_S (c = 64); an eigenvector separated by gap from the rest of the spectrum moves
    by c m eps kappa_S ||H~|| / gap (S-norm), and its S-projection on the oracle's eigenspace
    differs from 1 by the square of that plus the normalisation error."""
    m0 = Hb.shape[-1]
    eps = np.finfo(float).eps
    ref, vref, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    assert np.array_equal(ks, st)
    worst, ratio = check_eigenvalues(eig, ref, Hb, Sb, H, S, status=st)
    assert ratio <= 1.0, (worst, ratio)
    # both solvers take the Hermitian parts of the blocks (they are Hermitian up to the rounding
    # of the transform); the checks use the same matrices
    Hk = Hb.reshape(-1, m0, m0)
    Sk = Sb.reshape(-1, m0, m0)
    Hk = 0.5 * (Hk + np.conj(np.transpose(Hk, (0, 2, 1))))
    Sk = 0.5 * (Sk + np.conj(np.transpose(Sk, (0, 2, 1))))
    K = Hk.shape[0]
    Lt = Hb.shape[:3]
    s0 = np.mean(np.real(np.einsum("kii->ki", Sk)), axis=0)
    rat = {"orth": 0.0, "ritz": 0.0, "space": 0.0, "vec": 0.0}
    for k in range(K):
        n = m0 - st[k]
        assert np.all(vecs[k, n:] == 0)
        # kappa and -kappa: the solver takes one k-point of each conjugate pair (the lower
        # index) and writes the complex conjugate to the other, which is checked by that relation
        k0, k1, k2 = np.unravel_index(k, Lt)
        mk = np.ravel_multi_index(((-k0) % Lt[0], (-k1) % Lt[1], (-k2) % Lt[2]), Lt)
        if mk != k:
            assert np.array_equal(vecs[mk], np.conj(vecs[k]))
        else:  # a self-conjugate k-point has real blocks: real eigenvectors up to rounding
            assert np.abs(vecs[k].imag).max() <= 1e-8 * max(1.0, np.abs(vecs[k]).max())
        if mk < k:
            continue
        U = vecs[k, :n].T
        d = np.real(np.diag(Sk[k]))
        kept = np.nonzero(d > oracle_mod.DROP_TOL * s0)[0]
        assert np.all(vecs[k][:, np.setdiff1d(np.arange(m0), kept)] == 0)
        Dk = 1.0 / np.sqrt(d[kept])
        Ss = Sk[k][np.ix_(kept, kept)] * np.outer(Dk, Dk)
        Hs = Hk[k][np.ix_(kept, kept)] * np.outer(Dk, Dk)
        sig = np.linalg.eigvalsh(0.5 * (Ss + Ss.conj().T))
        kap_s = 1.0 / sig[sig >= oracle_mod.LINDEP_TOL].min()
        base = 64.0 * m0 * eps * kap_s
        nH = np.linalg.norm(Hs, 2)
        # S-orthonormality and the Rayleigh-Ritz conditions, in the scaled coordinates
        Us = U[kept] / Dk[:, None]
        rat["orth"] = max(rat["orth"], np.abs(Us.conj().T @ Ss @ Us - np.eye(n)).max() / base)
        rat["ritz"] = max(rat["ritz"], np.abs(Us.conj().T @ Hs @ Us - np.diag(eig[k, :n])).max() / (base * nH))
        # eigenspaces: clusters of eigenvalues closer than 1e-6 of the scale
        lam = ref[k, :n]
        Uo = vref[k, :n].T
        i = 0
        while i < n:
            j = i + 1
            while j < n and lam[j] - lam[j - 1] < 1e-6 * nH:
                j += 1
            gap = min(lam[i] - lam[i - 1] if i > 0 else np.inf, lam[j] - lam[j - 1] if j < n else np.inf)
            tv = base * nH / gap
            P = Uo[:, i:j]
            for r in range(i, j):
                c = P.conj().T @ (Sk[k] @ U[:, r])  # coordinates in the oracle's eigenspace
                rat["space"] = max(rat["space"], abs(np.linalg.norm(c) - 1.0) / (tv * tv + base))
                if j == i + 1:
                    mags = np.sort(np.abs(Uo[kept, r] / Dk))[::-1]
                    if len(mags) == 1 or mags[0] - mags[1] > 1e-3 * mags[0]:  # phase well posed
                        dv = np.abs((U[kept, r] - Uo[kept, r]) / Dk).max()
                        rat["vec"] = max(rat["vec"], dv / (tv * (1.0 + 2.0 / (1e-3 * mags[0]))))
            i = j
    print("eigenvector deviations / tolerance:", {a: f"{b:.2e}" for a, b in rat.items()})
    assert max(rat.values()) <= 1.0, rat
    return rat


@pytest.mark.parametrize("name", sorted(CASES))
def test_bloch_eigenvectors_match_oracle(ctx, oracle_mod, name):
    cfg = CASES[name]()
    ctx.setup(cfg)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, ks = gpu_vectors(ctx, Hb, Sb)
    compare_with_oracle(eig, vecs, ks, oracle_mod, Hb, Sb, Hj, Sj)
    # the eigenvalues equal those of the tridiagonal route within the same tolerance
    K, m0 = eig.shape
    e2 = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    ctx.k_point_eigensolve(to_dev(Hb), to_dev(Sb), e2)
    ctx.sync()
    worst, ratio = check_eigenvalues(eig, e2.cpu().numpy(), Hb, Sb, Hj, Sj, status=ks)
    assert ratio <= 1.0, (worst, ratio)


def test_lattice_eigenvectors_of_the_dense_matrix(ctx, oracle_mod):
    # eq. (6.8): x_p = exp(2 pi i kappa p / L) u / sqrt(L) from the GPU's Bloch vectors is an
    # eigenvector of the oracle's dense lattice pencil
    cfg = CASES["periodic_8"]()
    ctx.setup(cfg)
    H, S = oracle_mod.core_dense(cfg)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, ks = gpu_vectors(ctx, Hb, Sb)
    L = cfg["L"]
    scale = np.abs(H).max() + np.abs(eig).max() * np.abs(S).max()
    for k in range(L[0]):
        for r in range(Hb.shape[-1] - ks[k]):
            x = oracle_mod.lattice_eigenvector(vecs[k, r], (k, 0, 0), L)
            assert np.abs(H @ x - eig[k, r] * (S @ x)).max() <= 1e-9 * scale, (k, r)


def test_removed_functions_and_canonical_route(ctx, oracle_mod):
    # a cancelled Bloch function (removed) and an indefinite scaled overlap (canonical route)
    cfg = CASES["tube_9_m5_odd"]()
    ctx.setup(cfg)
    m0, K = 5, 9
    rng = np.random.default_rng(1)
    X = rng.standard_normal((K, m0, m0)) + 1j * rng.standard_normal((K, m0, m0))
    Hh = X + np.conj(np.transpose(X, (0, 2, 1)))
    B = rng.standard_normal((K, m0, m0)) + 1j * rng.standard_normal((K, m0, m0))
    Sh = B @ np.conj(np.transpose(B, (0, 2, 1))) + m0 * np.eye(m0)
    Sh[2, 3, :] *= 1e-5  # function 3 nearly cancelled at kappa = 2 (and 7)
    Sh[2, :, 3] *= 1e-5
    Sh[4, 0, 1] = 0.999 * np.sqrt(Sh[4, 0, 0].real * Sh[4, 1, 1].real) * 3.0  # indefinite at kappa = 4 (and 5)
    Sh[4, 1, 0] = np.conj(Sh[4, 0, 1])
    Hh[0], Sh[0] = Hh[0].real, Sh[0].real  # blocks of a real lattice matrix: real at kappa = 0,
    for k in range(5, 9):  # conjugate at -kappa
        Hh[k] = np.conj(Hh[9 - k])
        Sh[k] = np.conj(Sh[9 - k])
    Hb, Sb = Hh.reshape(K, 1, 1, m0, m0), Sh.reshape(K, 1, 1, m0, m0)
    eig, vecs, ks = gpu_vectors(ctx, Hb, Sb)
    assert ks[2] == 1 and ks[7] == 1 and ks[4] >= 1 and ks[5] >= 1
    assert np.all(vecs[2, :, 3] == 0)
    compare_with_oracle(eig, vecs, ks, oracle_mod, Hb, Sb)


def test_full_size_tube_256_eigenvectors(ctx, oracle_mod, lhf):
    # the bench system: GPU blocks (mixed route) through the GPU DFT, then the eigenvectors
    cfg = W.tube_256(3000)
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    m0, K = sz["m0"], sz["n_kpoints"]
    H = torch.empty((256, 1, 1, m0, m0), dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    ctx.assemble_core_hamiltonian(H, S, lhf.MIXED)
    Hb = torch.empty((256, 1, 1, m0, m0, 2), dtype=torch.float64, device="cuda")
    Sb = torch.empty_like(Hb)
    ctx.circulant_fft(H, S, Hb, Sb)
    eig = torch.empty((K, m0), dtype=torch.float64, device="cuda")
    vecs = torch.empty((K, m0, m0, 2), dtype=torch.float64, device="cuda")
    ks = torch.empty((K,), dtype=torch.int32, device="cuda")
    ctx.k_point_eigenvectors(Hb, Sb, eig, vecs, ks)
    ctx.sync()
    hb = Hb.cpu().numpy()
    sb = Sb.cpu().numpy()
    v = vecs.cpu().numpy()
    compare_with_oracle(eig.cpu().numpy(), v[..., 0] + 1j * v[..., 1], ks.cpu().numpy(), oracle_mod,
                        hb[..., 0] + 1j * hb[..., 1], sb[..., 0] + 1j * sb[..., 1])


@pytest.mark.parametrize("name,kappas,lo,cnt", [
    ("tube_9_m5_odd", [(0, 0, 0), (2, 0, 0), (4, 0, 0)], (0, 0, 0), None),
    ("cubic_3", [(1, 0, 2), (0, 0, 0)], (3, 5, 7), (20, 9, 11)),
    ("tube_256", [(5, 0, 0), (128, 0, 0)], (1000, 100, 120), (200, 8, 8)),
])
def test_bloch_orbitals_on_the_grid(ctx, oracle_mod, name, kappas, lo, cnt):
    cfg = W.tube_256(3000) if name == "tube_256" else CASES[name]()
    ctx.setup(cfg)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, ks = gpu_vectors(ctx, Hb, Sb)
    cnt = tuple(cfg["n"]) if cnt is None else cnt
    Lt = cfg["L"]
    for kap in kappas:
        k = np.ravel_multi_index(kap, Lt)
        rows = vecs[k, :3]
        coef = torch.from_numpy(np.ascontiguousarray(np.stack([rows.real, rows.imag], -1))).cuda()
        out = torch.empty((3,) + tuple(cnt) + (2,), dtype=torch.float64, device="cuda")
        ctx.bloch_orbitals(kap, coef, lo, cnt, out)
        ctx.sync()
        got = out.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
        for r in range(3):
            ref = oracle_mod.bloch_orbital(cfg, kap, rows[r], lo, cnt)
            assert np.abs(got[r] - ref).max() <= 1e-12 * np.abs(ref).max(), (kap, r)


def test_bloch_orbitals_reject_bad_windows(ctx, lhf):
    cfg = CASES["tube_9_m5_odd"]()
    ctx.setup(cfg)
    coef = torch.zeros((1, 5, 2), dtype=torch.float64, device="cuda")
    out = torch.empty((1, 4, 4, 4, 2), dtype=torch.float64, device="cuda")
    for kap, lo, cnt in [((9, 0, 0), (0, 0, 0), (4, 4, 4)), ((0, 0, 0), (178, 0, 0), (4, 4, 4)),
                         ((0, 0, 0), (0, 0, 0), (0, 4, 4))]:
        with pytest.raises(lhf.LhfError) as ei:
            ctx.bloch_orbitals(kap, coef, lo, cnt, out)
        assert ei.value.status == lhf.LHF_ERR_ARG
