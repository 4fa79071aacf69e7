"""lhf_cell_energies (the energy per cell of the lowest states, Sec. 5) against the oracle's
cell_energy: the selected level exactly and the energy to the summation-order bound, on random
spectra with ties, signed zeros and +inf in segments of 1 to 300 000 values in one launch; on the
GPU's own spectra of periodic and open chains (the paper's box-vs-periodic comparison) and of a
batch of tube_256 systems; end to end against the oracle's spectra of the chains; repeated calls
bit for bit."""

import numpy as np
import pytest

import lhf_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = np.finfo(np.float64).eps


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


def gpu_energies(ctx, flat, off, cnt, n_low, cells):
    d = torch.from_numpy(np.ascontiguousarray(flat, dtype=np.float64)).cuda()
    e = torch.empty(len(cnt), dtype=torch.float64, device="cuda")
    lev = torch.empty(len(cnt), dtype=torch.float64, device="cuda")
    ctx.cell_energies(d, off, cnt, n_low, cells, e, lev)
    torch.cuda.synchronize()
    return e.cpu().numpy(), lev.cpu().numpy()


def check_against_oracle(oracle_mod, flat, off, cnt, n_low, cells, e, lev):
    for s in range(len(cnt)):
        v = flat[off[s]:off[s] + cnt[s]]
        want, want_lev = oracle_mod.cell_energy(v, n_low[s], cells[s])
        if np.isinf(want):
            assert np.isinf(e[s]) and np.isinf(lev[s]), s
            continue
        assert lev[s] == want_lev, (s, lev[s], want_lev)  # the selection is exact
        sel = np.sort(v)[:n_low[s]]
        bound = 2.0 * n_low[s] * EPS * np.abs(sel).sum() / cells[s]
        assert abs(e[s] - want) <= bound, (s, e[s], want, bound)


def random_spectra(seed):
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 7, 31, 512, 513, 4096, 100_003, 300_000]
    parts = []
    for i, n in enumerate(sizes):
        v = rng.normal(size=n) * 10.0 ** rng.uniform(-3, 3)
        if i % 3 == 0:
            v = np.round(v, 1)                             # many ties
        if n >= 7:
            v[rng.integers(0, n, size=n // 7)] = np.inf    # removed functions
            v[:2] = (-0.0, 0.0)
        parts.append(v)
    off = np.cumsum([0] + sizes[:-1]).tolist()
    return np.concatenate(parts), off, sizes, rng


@pytest.mark.parametrize("seed", [1, 2])
def test_random_segments_match_the_oracle(ctx, oracle_mod, seed):
    flat, off, cnt, rng = random_spectra(seed)
    finite = [int(np.isfinite(flat[o:o + c]).sum()) for o, c in zip(off, cnt)]
    for choice in ("one", "all_finite", "middle", "all"):
        if choice == "one":
            n_low = [1] * len(cnt)
        elif choice == "all_finite":
            n_low = finite
        elif choice == "middle":
            n_low = [int(rng.integers(1, f + 1)) for f in finite]
        else:
            n_low = list(cnt)  # takes +inf where the segment has any: energy +inf
        cells = [float(rng.uniform(0.5, 300.0)) for _ in cnt]
        e, lev = gpu_energies(ctx, flat, off, cnt, n_low, cells)
        check_against_oracle(oracle_mod, flat, off, cnt, n_low, cells, e, lev)
        e2, lev2 = gpu_energies(ctx, flat, off, cnt, n_low, cells)
        assert np.array_equal(e, e2) and np.array_equal(lev, lev2)  # bit for bit


def test_arguments_are_checked(ctx, lhf):
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    for off, cnt, n_low, cells in (([0], [4], [5], [1.0]), ([0], [4], [0], [1.0]), ([0], [0], [1], [1.0]),
                                   ([0], [4], [2], [0.0]), ([-1], [4], [2], [1.0])):
        with pytest.raises(RuntimeError):
            ctx.cell_energies(d, off, cnt, n_low, cells, e)


def spectrum_of(ctx, cfg):
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    n = sz["n_basis"] if not sz["periodic"] else sz["n_kpoints"] * sz["m0"]
    eig = torch.empty(n, dtype=torch.float64, device="cuda")
    ctx.bloch_spectra([cfg], eig)
    torch.cuda.synchronize()
    return eig


@pytest.mark.parametrize("L", [4, 16])
def test_open_and_periodic_chains(ctx, oracle_mod, L):
    # the paper's comparison: energy per cell of the lowest states of the same chain, open box and
    # periodic supercell, from the GPU's spectra; exact selection on those spectra, and against
    # the oracle's spectra within the sorted spectra's largest difference per state
    ref = {}
    for periodic in (True, False):
        cfg = W.chain(L, periodic=periodic)
        eig = spectrum_of(ctx, cfg)
        host = eig.cpu().numpy()
        if periodic:
            ev, st = oracle_mod.bloch_spectrum(cfg)
            ev = ev.ravel()
        else:
            H, S = oracle_mod.core_dense(cfg)
            ev = oracle_mod.dense_gen_eigenvalues(H, S)
        gap = np.abs(np.sort(host) - np.sort(ev)).max()
        assert gap < 1e-8, gap
        n_low = [1, L, 2 * L, len(host)]
        e = torch.empty(4, dtype=torch.float64, device="cuda")
        lev = torch.empty(4, dtype=torch.float64, device="cuda")
        ctx.cell_energies(eig, [0] * 4, [len(host)] * 4, n_low, [float(L)] * 4, e, lev)
        torch.cuda.synchronize()
        e, lev = e.cpu().numpy(), lev.cpu().numpy()
        check_against_oracle(oracle_mod, host, [0] * 4, [len(host)] * 4, n_low, [float(L)] * 4, e, lev)
        for i, n in enumerate(n_low):
            want, _ = oracle_mod.cell_energy(ev, n, L)
            assert abs(e[i] - want) <= n * gap / L + 1e-12, (periodic, n, e[i], want)
        ref[periodic] = e
    # the open box's lowest states lie above the periodic chain's (no images beyond its ends)
    assert ref[False][1] > ref[True][1]


def test_batch_of_tube_spectra(ctx, oracle_mod, lhf):
    cfgs = W.tube_256_batch(4)
    ctx.setup(cfgs[0])
    sz = ctx.query_sizes()
    per = sz["n_kpoints"] * sz["m0"]
    eig = torch.empty(4 * per, dtype=torch.float64, device="cuda")
    ctx.bloch_spectra(cfgs, eig, None, lhf.MIXED)
    torch.cuda.synchronize()
    host = eig.cpu().numpy()
    off = [s * per for s in range(4)]
    cnt = [per] * 4
    n_low = [256, 512, 1, per - 300]
    cells = [256.0] * 4
    e, lev = gpu_energies(ctx, host, off, cnt, n_low, cells)
    check_against_oracle(oracle_mod, host, off, cnt, n_low, cells, e, lev)
