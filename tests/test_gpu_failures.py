"""Failure detection on the GPU, in forms that fault nothing.

Time-outs: the dense eigensolver's grid barriers wait with a bound; lhf_inject_barrier_stall
makes the next solve's barriers expect one CTA more than the launch holds, so every wait runs out
(a count that nothing completes).  The context must report LHF_ERR_TIMEOUT at the next sync and
then solve correctly.  Allocation failure: lhf_set_workspace_limit caps the workspace; a call
that needs more returns LHF_ERR_NOMEM before any kernel launch, and the context works again once
the cap is lifted."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import check_dense_eigenvalues, check_eigenvalues

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


def _pencil(N, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, N))
    S = A @ A.T / N + np.eye(N) * 0.5
    B = rng.standard_normal((N, N))
    return (B + B.T) * 3.0, S


def test_barrier_wait_runs_out_and_context_recovers(lhf, oracle_mod):
    ctx = lhf.Context(0)
    try:
        N = 300  # more CTAs than one: every grid barrier is a real wait
        H, S = _pencil(N, 7)
        Hd, Sd = torch.from_numpy(H).cuda(), torch.from_numpy(S).cuda()
        eig = torch.empty(N, dtype=torch.float64, device="cuda")
        ref = oracle_mod.dense_gen_eigenvalues(H, S)
        for limit in (2_000_000, 0):  # ~1 ms, then the default ~1 s
            ctx.set_wait_limit(limit)
            ctx.inject_barrier_stall()
            ctx.dense_eigensolve(Hd, Sd, N, eig)
            with pytest.raises(lhf.LhfError) as ei:
                ctx.sync()
            assert ei.value.status == lhf.LHF_ERR_TIMEOUT
            # the stall is consumed: the same context solves the same pencil correctly
            ctx.dense_eigensolve(Hd, Sd, N, eig)
            ctx.sync()
            worst, ratio = check_dense_eigenvalues(eig.cpu().numpy(), ref, H, S)
            assert ratio <= 1.0, (limit, worst, ratio)
        # and the rest of the path still works on it: an open box end to end
        box = W.box_64(L=4, n_perp=64)
        Nb = len(box["alpha"]) * 4
        e2 = torch.empty(Nb, dtype=torch.float64, device="cuda")
        ctx.bloch_spectra([box], e2)
        ctx.sync()
        Hr, Sr = oracle_mod.core_dense(box)
        assert np.abs(e2.cpu().numpy() - oracle_mod.dense_gen_eigenvalues(Hr, Sr)).max() < 1e-8
    finally:
        ctx.close()


def test_workspace_limit_fails_before_any_launch(lhf, oracle_mod):
    ctx = lhf.Context(0)
    try:
        cfg = W.periodic_8()
        ctx.setup(cfg)
        sz = ctx.query_sizes()
        eig = torch.empty((sz["n_kpoints"], sz["m0"]), dtype=torch.float64, device="cuda")
        ctx.set_workspace_limit(4096)
        ctx.set_profiling(True)
        ctx.kernel_times()
        with pytest.raises(lhf.LhfError) as ei:
            ctx.bloch_spectra([cfg], eig)
        assert ei.value.status == lhf.LHF_ERR_NOMEM
        assert sum(n for _, n in ctx.kernel_times().values()) == 0  # nothing was launched
        # a graph needs its own workspace: refused as well
        with pytest.raises(lhf.LhfError) as ei:
            ctx.graph_create([cfg], eig, None, lhf.FP64)
        assert ei.value.status == lhf.LHF_ERR_NOMEM
        ctx.set_workspace_limit(0)
        ctx.bloch_spectra([cfg], eig)
        ctx.sync()
        assert sum(n for _, n in ctx.kernel_times().values()) > 0
        H, S = oracle_mod.core_blocks(cfg)
        Hb, Sb = oracle_mod.block_dft(H), oracle_mod.block_dft(S)
        ref, st = oracle_mod.k_point_eigenvalues(Hb, Sb)
        worst, ratio = check_eigenvalues(eig.cpu().numpy(), ref, Hb, Sb, H, S, status=st)
        assert ratio <= 1.0, (worst, ratio)
    finally:
        ctx.close()
