"""The heterogeneous batch (tubes and slabs of mixed L, m0, h and R in one batched pass) and the
CUDA-graph entry points: parity of every member with the oracle, batch = single runs, and graph
replays = direct runs, bit for bit."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import check_eigenvalues

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# small members of the heterogeneous batch (the oracle finishes them in well under a second)
SMALL = [3, 4, 7, 9, 15, 16, 17, 18, 23, 31, 40, 62]


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
def small_batch():
    full = W.hetero_batch()
    return [full[i] for i in SMALL]


def sizes_of(ctx, cfgs):
    out = []
    for c in cfgs:
        ctx.setup(c)
        s = ctx.query_sizes()
        out.append((s["n_kpoints"], s["m0"]))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_hetero_batch_parity_with_oracle(ctx, oracle_mod, small_batch, precision):
    sz = sizes_of(ctx, small_batch)
    eig = torch.empty(sum(k * m for k, m in sz), dtype=torch.float64, device="cuda")
    ks = torch.empty(sum(k for k, _ in sz), dtype=torch.int32, device="cuda")
    ctx.bloch_spectra(small_batch, eig, ks, precision)
    ctx.sync()
    got, gks = eig.cpu().numpy(), ks.cpu().numpy()
    eo = ko = 0
    for cfg, (K, m0) in zip(small_batch, sz):
        Hr, Sr = oracle_mod.core_blocks(cfg)
        Hb, Sb = oracle_mod.block_dft(Hr), oracle_mod.block_dft(Sr)
        ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
        assert np.array_equal(gks[ko:ko + K], st), (cfg["name"], cfg["seed"])
        worst, ratio = check_eigenvalues(got[eo:eo + K * m0].reshape(K, m0), ref, Hb, Sb, Hr, Sr, status=st)
        assert ratio <= 1.0, (cfg["name"], cfg["seed"], worst, ratio)
        eo += K * m0
        ko += K


def test_hetero_batch_equals_single_runs(ctx, small_batch):
    sz = sizes_of(ctx, small_batch)
    n = [k * m for k, m in sz]
    eig = torch.empty(sum(n), dtype=torch.float64, device="cuda")
    ctx.bloch_spectra(small_batch, eig)
    ctx.sync()
    batch = eig.cpu().numpy()
    off = 0
    for c, k in zip(small_batch, n):
        one = torch.empty(k, dtype=torch.float64, device="cuda")
        ctx.bloch_spectra([c], one)
        ctx.sync()
        assert np.array_equal(one.cpu().numpy(), batch[off:off + k]), c["name"]
        off += k


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replays_equal_direct_runs(ctx, lhf, small_batch, precision):
    sz = sizes_of(ctx, small_batch)
    ne, nk = sum(k * m for k, m in sz), sum(k for k, _ in sz)
    direct = torch.empty(ne, dtype=torch.float64, device="cuda")
    dks = torch.empty(nk, dtype=torch.int32, device="cuda")
    ctx.bloch_spectra(small_batch, direct, dks, precision)
    ctx.sync()
    eig = torch.full((ne,), float("nan"), dtype=torch.float64, device="cuda")
    ks = torch.full((nk,), -99, dtype=torch.int32, device="cuda")
    g = ctx.graph_create(small_batch, eig, ks, precision)
    try:
        g.launch()
        ctx.sync()
        first = eig.cpu().numpy().copy()
        assert np.array_equal(first, direct.cpu().numpy())
        assert np.array_equal(ks.cpu().numpy(), dks.cpu().numpy())
        # other work on the context in between (it reuses the context workspace, not the graph's)
        other = torch.empty(8 * 4, dtype=torch.float64, device="cuda")
        ctx.bloch_spectra([W.periodic_8()], other)
        eig.fill_(float("nan"))
        g.launch()
        ctx.sync()
        assert np.array_equal(eig.cpu().numpy(), first)
    finally:
        g.close()


def test_graph_rejects_open_boxes(ctx, lhf):
    box = W.box_64(seed=21, L=4, n_perp=64)
    eig = torch.empty(32, dtype=torch.float64, device="cuda")
    with pytest.raises(lhf.LhfError) as ei:
        ctx.graph_create([box], eig)
    assert ei.value.status == lhf.LHF_ERR_UNSUPPORTED


@pytest.mark.slow
def test_full_hetero_batch_runs_and_matches_single_runs_on_samples(ctx):
    """All 64 members in one batched pass (mixed route) and through a graph: finite spectra, no
    NOT_SPD k-point, and a sample of members equal to their single runs."""
    cfgs = W.hetero_batch()
    sz = sizes_of(ctx, cfgs)
    ne, nk = sum(k * m for k, m in sz), sum(k for k, _ in sz)
    eig = torch.empty(ne, dtype=torch.float64, device="cuda")
    ks = torch.empty(nk, dtype=torch.int32, device="cuda")
    ctx.bloch_spectra(cfgs, eig, ks, 1)
    ctx.sync()
    got = eig.cpu().numpy()
    assert np.all(ks.cpu().numpy() >= 0)
    assert np.all(np.isfinite(got) | np.isposinf(got))
    offs = np.cumsum([0] + [k * m for k, m in sz])
    for i in (5, 19, 25, 46, 60):
        one = torch.empty(int(offs[i + 1] - offs[i]), dtype=torch.float64, device="cuda")
        ctx.bloch_spectra([cfgs[i]], one, None, 1)
        ctx.sync()
        assert np.array_equal(one.cpu().numpy(), got[offs[i]:offs[i + 1]]), cfgs[i]["name"]
    g_eig = torch.empty(ne, dtype=torch.float64, device="cuda")
    g = ctx.graph_create(cfgs, g_eig, None, 1)
    try:
        g.launch()
        ctx.sync()
        assert np.array_equal(g_eig.cpu().numpy(), got)
    finally:
        g.close()


def test_graph_outliving_its_context(lhf):
    # a context destroyed before its graph detaches it: the graph refuses to launch (no stream to
    # launch on) and is still freed cleanly
    c = lhf.Context(0)
    cfg = W.periodic_8()
    c.setup(cfg)
    sz = c.query_sizes()
    eig = torch.empty((sz["n_kpoints"], sz["m0"]), dtype=torch.float64, device="cuda")
    g = c.graph_create([cfg], eig, None, lhf.FP64)
    g.launch()
    c.sync()
    c.close()
    with pytest.raises(lhf.LhfError) as ei:
        g.launch()
    assert ei.value.status == lhf.LHF_ERR_STATE
    g.close()
    torch.cuda.synchronize()
