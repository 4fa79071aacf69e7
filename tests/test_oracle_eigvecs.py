"""Pins of the oracle's Bloch eigenvectors (Prop. 6.1, eq. (6.8)) against facts other than
itself: the eigenvector of the whole lattice matrix, assembled entry by entry by the oracle's
dense route, is the Bloch vector spread over the cells with the phase exp(2 pi i kappa p / L);
the eigenvalues agree with the oracle's own Jacobi eigenvalues (a different algorithm); m0 = 1
has the closed form u = Sbar^-1/2; and the pairs satisfy the pencil and S-orthonormality."""

import numpy as np
import pytest

import lhf_workloads as W


def small_tube(L=6, seed=21):
    return W.tube(L, seed=seed, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=2, m0_pshell=1,
                  lo=0.3, hi=8.0)


def test_lattice_eigenvectors_from_bloch_vectors(oracle_mod):
    # eq. (6.8): x_p = exp(2 pi i kappa p / L) u / sqrt(L) solves the dense pencil H x = lambda S x
    cfg = small_tube(L=6, seed=8)
    H, S = oracle_mod.core_dense(cfg)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    assert np.all(st == 0)
    L = cfg["L"]
    m0 = Hb.shape[-1]
    scale = np.abs(H).max() + np.abs(eig).max() * np.abs(S).max()
    for k in range(L[0]):
        for r in range(m0):
            x = oracle_mod.lattice_eigenvector(vecs[k, r], (k, 0, 0), L)
            res = H @ x - eig[k, r] * (S @ x)
            assert np.abs(res).max() <= 1e-10 * scale, (k, r)
            assert abs(np.vdot(x, S @ x) - 1.0) < 1e-10  # S-normalised on the lattice too
    # the opposite phase convention is not an eigenvector (kappa != 0, L/2)
    x = oracle_mod.lattice_eigenvector(vecs[1, 0], (-1, 0, 0), L)
    assert np.abs(H @ x - eig[1, 0] * (S @ x)).max() > 1e-4 * scale


def test_3d_lattice_eigenvector(oracle_mod):
    cfg = W.cubic_32(seed=15, L=3, n_c=10)
    H, S = oracle_mod.core_dense(cfg)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    L = cfg["L"]
    scale = np.abs(H).max() + np.nanmax(np.abs(eig[np.isfinite(eig)])) * np.abs(S).max()
    K = np.arange(L[0] * L[1] * L[2]).reshape(L)
    for kap in [(0, 0, 0), (1, 0, 2), (2, 1, 1)]:
        k = K[kap]
        for r in range(Hb.shape[-1] - st[k]):
            x = oracle_mod.lattice_eigenvector(vecs[k, r], kap, L)
            assert np.abs(H @ x - eig[k, r] * (S @ x)).max() <= 1e-9 * scale, (kap, r)


def test_eigenvectors_satisfy_the_pencil_and_match_jacobi_eigenvalues(oracle_mod):
    cfg = small_tube(L=8, seed=3)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    ref, st_ref = oracle_mod.k_point_eigenvalues(Hb, Sb)
    assert np.array_equal(st, st_ref)
    fin = np.isfinite(ref)
    assert np.abs(eig[fin] - ref[fin]).max() < 1e-10 * max(1.0, np.abs(ref[fin]).max())
    Hb = Hb.reshape(-1, *Hb.shape[-2:])
    Sb = Sb.reshape(-1, *Sb.shape[-2:])
    for k in range(Hb.shape[0]):
        U = vecs[k].T  # columns
        G = U.conj().T @ Sb[k] @ U
        assert np.abs(G - np.eye(G.shape[0])).max() < 1e-10
        R = Hb[k] @ U - Sb[k] @ U * eig[k][None, :]
        assert np.abs(R).max() < 1e-10 * (np.abs(Hb[k]).max() + np.abs(eig[k]).max() * np.abs(Sb[k]).max())


def test_m0_one_and_phase_convention(oracle_mod):
    rng = np.random.default_rng(5)
    Hb = (rng.standard_normal((4, 1, 1)) + 0j)
    Sb = (rng.uniform(0.5, 2.0, (4, 1, 1)) + 0j)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    assert np.allclose(vecs[:, 0, 0], 1.0 / np.sqrt(Sb[:, 0, 0].real), rtol=1e-14, atol=0)
    assert np.allclose(eig[:, 0], (Hb / Sb).real.ravel(), rtol=1e-14)
    # phase: the first component of largest magnitude is real and positive
    m = 5
    X = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Y = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    Hh, Sh = X + X.conj().T, Y @ Y.conj().T + m * np.eye(m)
    _, v, _ = oracle_mod.k_point_eigenvectors(Hh[None], Sh[None])
    for r in range(m):
        big = np.argmax(np.abs(v[0, r]) ** 2)
        assert v[0, r, big].imag == 0.0 and v[0, r, big].real > 0


def test_removed_functions_have_zero_components(oracle_mod):
    # a Bloch function that cancels at one k-point is removed there (same rule as the eigenvalues)
    rng = np.random.default_rng(9)
    m, K = 4, 3
    B = rng.standard_normal((K, m, m)) + 1j * rng.standard_normal((K, m, m))
    Sb = B @ B.conj().transpose(0, 2, 1) + m * np.eye(m)
    Sb[1, 2, :] *= 1e-5
    Sb[1, :, 2] *= 1e-5
    Hb = Sb * 0.5 + np.eye(m)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    _, st_ref = oracle_mod.k_point_eigenvalues(Hb, Sb)
    assert st[1] == 1 and np.array_equal(st, st_ref)
    assert np.all(vecs[1, :, 2] == 0) and np.all(vecs[1, 3] == 0) and np.isinf(eig[1, 3])


def test_bloch_orbital_is_normalised_and_bloch_periodic(oracle_mod):
    # the orbital of an S-normalised Bloch vector has unit norm in the P1 mass inner product of the
    # whole grid (the Galerkin overlap that Sbar transforms), and psi(x + b) = exp(2 pi i kappa / L) psi(x)
    cfg = W.tube(9, seed=14, n_c=20, n_perp=48, half_width=6.0, M0=1, m0_s=2, m0_pshell=1, lo=0.2, hi=9.0)
    Hj, Sj = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(Hj), oracle_mod.block_dft(Sj)
    eig, vecs, st = oracle_mod.k_point_eigenvectors(Hb, Sb)
    n, h, L = cfg["n"], cfg["h"], cfg["L"]
    M = [oracle_mod.p1_mass_matrix(n[l], h[l], bool(cfg["periodic"][l])) for l in range(3)]
    for k, r in [(0, 0), (2, 1), (4, 3)]:
        psi = oracle_mod.bloch_orbital(cfg, (k, 0, 0), vecs[k, r], (0, 0, 0), n)
        Mpsi = np.einsum("ai,ijk->ajk", M[0], psi)
        Mpsi = np.einsum("bj,ajk->abk", M[1], Mpsi)
        Mpsi = np.einsum("ck,abk->abc", M[2], Mpsi)
        norm = np.vdot(psi, Mpsi)
        assert abs(norm - 1.0) < 1e-10, (k, r, norm)
        # two different eigenvectors of one k-point are orthogonal in the same inner product
        phi = oracle_mod.bloch_orbital(cfg, (k, 0, 0), vecs[k, r + 1], (0, 0, 0), n)
        assert abs(np.vdot(phi, Mpsi)) < 1e-10
        # Bloch periodicity along the lattice direction
        nc = cfg["n_cell"][0]
        ph = np.exp(2j * np.pi * k / L[0])
        assert np.abs(psi[nc:] - ph * psi[:-nc]).max() < 1e-12 * np.abs(psi).max()
