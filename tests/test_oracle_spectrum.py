"""Pins of the oracle's energy per cell of the lowest states (Sec. 5's average energy per unit
cell of a chain against L) against facts other than itself: the sum of the n smallest values is
the smallest sum over all n-element subsets (brute force on small arrays, ties and +inf
included); the returned level is the n-th order statistic by counting; and the union of the
k-point spectra of a periodic chain, the input the energy is taken over, is the spectrum of the
whole block-circulant lattice matrix assembled entry by entry (Prop. 6.1), so both give the
same energy for every n.  A last check plants an off-by-one selection in a copy of the function
and shows the brute force catches it."""

import itertools

import numpy as np
import pytest

import lhf_workloads as W


def brute(values, n, cells):
    best = min(sum(c) for c in itertools.combinations(values, n))
    return best / cells


@pytest.mark.parametrize("seed", range(6))
def test_smallest_subset_sum_by_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 10))
    v = rng.normal(size=m).round(2) * 3.0          # rounded: ties are likely
    if m > 2 and seed % 2:
        v[rng.integers(0, m)] = np.inf             # a removed function
    for n in range(1, m + 1):
        e, level = oracle_mod.cell_energy(v, n, 3.0)
        want = brute(list(v), n, 3.0)
        if np.isinf(want):
            assert np.isinf(e)
        else:
            assert abs(e - want) <= 1e-12 * (1.0 + np.abs(v[np.isfinite(v)]).sum())
        # level is the n-th order statistic
        assert np.count_nonzero(v < level) < n <= np.count_nonzero(v <= level)


def test_energy_of_ties_and_multiplicity(oracle_mod):
    v = np.array([2.0, -1.0, 2.0, 2.0, -1.0, np.inf])
    assert oracle_mod.cell_energy(v, 3, 1.0) == (0.0, 2.0)
    assert oracle_mod.cell_energy(v, 5, 2.0) == (2.0, 2.0)
    assert oracle_mod.cell_energy(v, 6, 1.0)[0] == np.inf
    # the shape of the spectrum array does not matter (k-points x bands)
    assert oracle_mod.cell_energy(v.reshape(2, 3), 4, 1.0) == oracle_mod.cell_energy(v, 4, 1.0)


@pytest.mark.parametrize("L", [3, 8])
def test_union_of_k_point_spectra_is_the_lattice_spectrum(oracle_mod, L):
    # Prop. 6.1: the energies over the k-point spectra equal those over the eigenvalues of the
    # dense block-circulant matrix of the periodic chain, for every number of selected states
    cfg = W.chain(L, seed=6, periodic=True, n_perp=32)
    eig, st = oracle_mod.bloch_spectrum(cfg)
    assert np.all(st == 0)
    H, S = oracle_mod.core_dense(cfg)
    dense = oracle_mod.dense_gen_eigenvalues(H, S)
    scale = np.abs(dense).max()
    for n in (1, L, 2 * L + 1, 4 * L):
        e_k, lev_k = oracle_mod.cell_energy(eig, n, L)
        e_d, lev_d = oracle_mod.cell_energy(dense, n, L)
        assert abs(e_k - e_d) <= 1e-10 * scale * n / L, (n, e_k, e_d)
        assert abs(lev_k - lev_d) <= 1e-10 * scale


def test_open_and_periodic_chains_share_the_cell(oracle_mod):
    # the two boundary conditions of W.chain differ only in the lattice direction's boundary
    for L in (2, 5):
        p, b = W.chain(L, periodic=True), W.chain(L, periodic=False)
        for k in ("alpha", "kind", "centre", "a", "Z", "b", "h", "n_cell", "R", "u0", "du"):
            assert p[k] == b[k], k
        assert p["periodic"] == [1, 0, 0] and b["periodic"] == [0, 0, 0]
        assert b["n"][0] % 128 == 0 and b["n"][0] >= L * b["n_cell"][0]
        # the box holds every basis function of every cell within its padded grid
        cut = max(np.sqrt(b["rho"] / a) for a in b["alpha"])
        lo = b["x0"][0]
        hi = lo + b["n"][0] * b["h"][0]
        assert lo <= b["cell0"][0] - cut + 1e-12 and hi >= b["cell0"][0] + L * b["b"][0] + cut - 1e-12


def test_brute_force_catches_an_off_by_one_selection(oracle_mod):
    def planted(eig, n_low, cells):  # the oracle's steps with one value too few selected
        v = np.sort(np.ravel(np.asarray(eig, dtype=np.float64)))
        low = v[:max(int(n_low) - 1, 1)]
        return float(np.sum(low)) / cells, float(low[-1])

    v = [0.5, -2.0, 1.5, -0.25]
    assert planted(v, 3, 1.0)[0] != brute(v, 3, 1.0)
    assert oracle_mod.cell_energy(v, 3, 1.0)[0] == brute(v, 3, 1.0)


def test_band_table_round_trip(oracle_mod, tmp_path):
    # the band file holds every eigenvalue of every k-point exactly, with kappa and q = kappa / L
    from paper_1408_3839_gb300 import bands

    cfg = W.periodic_8()
    eig, st = oracle_mod.bloch_spectrum(cfg)
    eig = eig.copy()
    eig[3, -1] = np.inf  # a removed function
    path = tmp_path / "bands.txt"
    bands.write_bands(str(path), eig, cfg["L"], st, title="periodic_8")
    back = np.loadtxt(path)
    assert back.shape == (8, 7 + eig.shape[1])
    assert np.array_equal(back[:, 7:], eig)
    assert np.array_equal(back[:, 0], np.arange(8)) and np.all(back[:, 1:3] == 0)
    assert np.array_equal(back[:, 3], [0, 0.125, 0.25, 0.375, 0.5, -0.375, -0.25, -0.125])
    assert np.array_equal(back[:, 6], st)
    # band r at kappa and -kappa agree (real lattice matrix; the oracle solves both)
    assert np.allclose(back[1, 7:], back[7, 7:], rtol=0, atol=1e-10)
