"""The allocation-free k-point eigensolve (lhf_k_point_eigensolve_noalloc), for callers that
cannot allocate device memory: services held to a fixed device-memory budget and hosts whose
allocator policy leaves the device memory to another framework.  Called through the C ABI and
compared with the context-based lhf_k_point_eigensolve on the same inputs, on calls in a row
(each with a different system, so that the shared scratch is reused with new contents): a small
tube, an odd tube, a tube with 32 functions per cell (the scratch's largest s0 and the
whole-warp solve), and a call without a k_status array.  This file is collected last."""

import numpy as np
import pytest

import lhf_workloads as W
from tests._numerics import check_eigenvalues

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _blocks(ctx, cfg):
    ctx.setup(cfg)
    sz = ctx.query_sizes()
    L, m0 = cfg["L"], sz["m0"]
    H = torch.empty((L[0], L[1], L[2], m0, m0), dtype=torch.float64, device="cuda")
    S = torch.empty_like(H)
    ctx.assemble_core_hamiltonian(H, S)
    Hb = torch.empty(H.shape + (2,), dtype=torch.float64, device="cuda")
    Sb = torch.empty_like(Hb)
    ctx.circulant_fft(H, S, Hb, Sb)
    ctx.sync()
    return Hb, Sb, sz


def test_noalloc_eigensolve_matches_context_eigensolve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_3839_gb300 import build, lhf

    build.build()
    ctx = lhf.Context(0)
    cases = [
        (W.tube(16, seed=11, n_c=32, n_perp=64, half_width=8.0), True),
        (W.tube(9, seed=14, n_c=20, n_perp=48, half_width=6.0, M0=1, m0_s=2, m0_pshell=1, lo=0.2, hi=9.0), True),
        (W.tube(6, seed=22, n_c=16, n_perp=32, half_width=5.0, M0=2, m0_s=2, m0_pshell=10, lo=0.4, hi=8.0), True),
        (W.tube(12, seed=15, n_c=24, n_perp=48, half_width=6.0), False),
    ]
    seen_m0 = set()
    for cfg, with_status in cases:  # calls in a row, different sizes
        Hb, Sb, sz = _blocks(ctx, cfg)
        K, m0 = sz["n_kpoints"], sz["m0"]
        seen_m0.add(m0)
        ref = torch.empty((K, m0), dtype=torch.float64, device="cuda")
        ref_st = torch.empty((K,), dtype=torch.int32, device="cuda")
        ctx.k_point_eigensolve(Hb, Sb, ref, ref_st)
        ctx.sync()
        got = torch.full((K, m0), np.nan, dtype=torch.float64, device="cuda")
        got_st = torch.full((K,), -99, dtype=torch.int32, device="cuda") if with_status else None
        lhf.k_point_eigensolve_noalloc(cfg["L"], m0, Hb, Sb, got, got_st)
        torch.cuda.synchronize()
        if with_status:
            assert np.array_equal(got_st.cpu().numpy(), ref_st.cpu().numpy())
        hb = Hb.cpu().numpy()
        sb = Sb.cpu().numpy()
        hb = hb[..., 0] + 1j * hb[..., 1]
        sb = sb[..., 0] + 1j * sb[..., 1]
        worst, ratio = check_eigenvalues(got.cpu().numpy(), ref.cpu().numpy(), hb, sb,
                                         status=ref_st.cpu().numpy())
        assert ratio <= 1.0, (m0, worst, ratio)
    assert 32 in seen_m0
    # sizes beyond the scratch's limit are rejected with a clear status
    with pytest.raises(lhf.LhfError) as ei:
        lhf.k_point_eigensolve_noalloc([4, 1, 1], 33, Hb, Sb, got, None)
    assert ei.value.status == lhf.LHF_ERR_ARG
    ctx.close()
