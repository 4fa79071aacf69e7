"""The batched entry points reuse a system's plan when a later call passes the same descriptor
content: a lattice that differs in any one descriptor field must get its own plan.  After a
context has solved a lattice, each one-field variant of it must give bit for bit the spectrum a
fresh context computes for the variant (both precisions)."""

import copy

import numpy as np
import pytest

import lhf_workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lhf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3839_gb300 import build, lhf as B

    build.build()
    return B


def base_system():
    return W.tube(12, seed=71, n_c=24, n_perp=48, m0_s=2, m0_pshell=1, lo=0.2, hi=9.0)


def variants():
    base = base_system()
    out = []
    v = copy.deepcopy(base)
    v["alpha"][1] *= 1.5  # one exponent
    out.append(("alpha", v))
    v = copy.deepcopy(base)
    v["rho"] = 30.0  # the truncation radius (support windows)
    out.append(("rho", v))
    v = copy.deepcopy(base)
    v["a"][0][0] += 0.1  # a nucleus position (the potential's image sums)
    out.append(("nucleus", v))
    v = copy.deepcopy(base)
    v["R"], v["u0"], v["du"] = 20, base["u0"] + 0.05, base["du"]  # the sinc nodes
    out.append(("sinc", v))
    return base, out


def spectrum(ctx, cfg, precision):
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    eig = torch.empty(sz["n_kpoints"] * sz["m0"], dtype=torch.float64, device="cuda")
    ctx.bloch_spectra([cfg], eig, None, precision)
    torch.cuda.synchronize()
    return eig.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_field_variants_get_their_own_plans(lhf, precision):
    base, vs = variants()
    warm = lhf.Context(0)
    try:
        spectrum(warm, base, precision)  # the base lattice's plan is now cached
        for name, v in vs:
            got = spectrum(warm, v, precision)
            fresh = lhf.Context(0)
            try:
                want = spectrum(fresh, v, precision)
            finally:
                fresh.close()
            assert np.array_equal(got, want), name
            # and the variant really differs from the base lattice
            assert not np.array_equal(got[np.isfinite(got)], spectrum(warm, base, precision)[np.isfinite(got)]), name
    finally:
        warm.close()


def test_prepared_batch_equals_the_dictionaries(lhf):
    """Context.prepare marshals the descriptor array once; the batched calls give the same
    spectra from it as from the list of workload dictionaries (device and host outputs)."""
    base, vs = variants()
    cfgs = [base] + [v for _, v in vs]
    ctx = lhf.Context(0)
    try:
        ctx.setup(base)
        sz = ctx.query_sizes()
        n = sum(c["L"][0] * c["L"][1] * c["L"][2] for c in cfgs) * sz["m0"]
        a = torch.empty(n, dtype=torch.float64, device="cuda")
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        ctx.bloch_spectra(cfgs, a, None, 1)
        prepared = ctx.prepare(cfgs)
        ctx.bloch_spectra(prepared, b, None, 1)
        host = np.empty(n)
        ctx.bloch_spectra_host(prepared, host, None, 1)
        torch.cuda.synchronize()
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
        assert np.array_equal(a.cpu().numpy(), host)
    finally:
        ctx.close()
