"""Pin of the oracle's separable k-space route (Theorem 2.5; Prop. 4.2): the 1D DFTs of the
per-direction factors, combined by Hadamard products and the rank sum at each k-point, equal
the direct multilevel DFT of the assembled real-space blocks (Lemma 4.1, Prop. 6.1) -- the same
numbers reached through a different order of sums (rank sum then 3D DFT, against 1D DFTs then
rank sum)."""

import numpy as np
import pytest

import lhf_workloads as W


@pytest.mark.parametrize("cfg_fn", [
    lambda: W.tube(6, seed=21, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=2, m0_pshell=1, lo=0.3, hi=8.0),
    lambda: W.periodic_8(),
    lambda: W.cubic_32(seed=15, L=3, n_c=10),
], ids=["tube_6", "periodic_8", "cubic_3"])
def test_kspace_route_equals_dft_of_blocks(oracle_mod, cfg_fn):
    cfg = cfg_fn()
    H, S = oracle_mod.core_blocks(cfg)
    Hb, Sb = oracle_mod.block_dft(H), oracle_mod.block_dft(S)
    Hk, Sk = oracle_mod.kspace_blocks(cfg)
    nblk = H.shape[0] * H.shape[1] * H.shape[2]
    assert np.abs(Hk - Hb).max() <= 1e-12 * np.abs(H).max() * nblk
    assert np.abs(Sk - Sb).max() <= 1e-12 * np.abs(S).max() * nblk
    # Hermitian blocks and the conjugate k-points of a real lattice matrix
    L = H.shape[:3]
    for k in np.ndindex(*L):
        mk = tuple((-np.array(k)) % np.array(L))
        assert np.abs(Hk[k] - Hk[k].conj().T).max() <= 1e-12 * np.abs(Hk[k]).max()
        assert np.abs(Hk[mk] - Hk[k].conj()).max() <= 1e-12 * np.abs(Hk[k]).max()


def test_kspace_route_detects_a_wrong_twiddle_sign(oracle_mod):
    # the transform direction matters once the factors are not symmetric in j
    cfg = W.tube(6, seed=21, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=2, m0_pshell=1, lo=0.3, hi=8.0)
    H, _ = oracle_mod.core_blocks(cfg)
    Hk, _ = oracle_mod.kspace_blocks(cfg)
    wrong = np.fft.ifftn(H, axes=(0, 1, 2)) * 6  # omega^(-kappa j)
    assert np.abs(Hk - wrong).max() > 1e-6 * np.abs(H).max()
