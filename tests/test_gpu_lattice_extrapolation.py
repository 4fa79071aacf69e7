"""Extrapolation of the lattice sum to the limit (lhf_extrapolate_lattice_sum, Sec. 4.1): spectra of
one (L,1,1) chain computed with growing image windows K_sum (K b / 2 inside the range on which
the sinc quadrature of 1/r was fitted); the far images add a potential that is constant over the
cell, so every eigenvalue drifts like -(2 Z_cell / b) rho ln K, rho the ratio of the
piecewise-constant (potential) mass form to the P1 (overlap) mass form on the state -- 1 for the
diffuse states of the lowest band, larger for states on tight functions that span few nodes.
The lowest band's fitted slopes reproduce -2 Z_cell / b, all slopes are negative, and the finite
parts agree between two disjoint sets of windows.  The fit itself is checked against numpy's
least squares on the same values."""

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


def _spectra(ctx, L, Ks):
    cfgs = []
    for K in Ks:
        c = W.chain(L)
        c["K_sum"] = [int(K), 1, 1]
        cfgs.append(c)
    eig = torch.empty((len(Ks), L * 4), dtype=torch.float64, device="cuda")
    ctx.bloch_spectra(cfgs, eig)
    ctx.sync()
    return cfgs[0], eig


def test_slopes_and_limits(lhf):
    ctx = lhf.Context(0)
    try:
        L = 16
        K1 = [64, 256, 1024]
        K2 = [80, 320, 1280]
        cfg, e1 = _spectra(ctx, L, K1)
        _, e2 = _spectra(ctx, L, K2)
        n = e1.shape[1]
        A1 = torch.empty(n, dtype=torch.float64, device="cuda")
        B1 = torch.empty_like(A1)
        A2 = torch.empty_like(A1)
        B2 = torch.empty_like(A1)
        ctx.extrapolate_lattice_sum(K1, e1, A1, B1)
        ctx.extrapolate_lattice_sum(K2, e2, A2, B2)
        ctx.sync()
    finally:
        ctx.close()
    y = e1.cpu().numpy()
    X = np.stack([np.ones(3), np.log(K1), 1.0 / np.array(K1, float)], axis=1)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    assert np.allclose(A1.cpu().numpy(), coef[0], rtol=0, atol=1e-9)
    assert np.allclose(B1.cpu().numpy(), coef[1], rtol=0, atol=1e-9)
    z_cell = float(np.sum(cfg["Z"]))
    expected = -2.0 * z_cell / cfg["b"][0]
    for B in (B1, B2):
        b = B.cpu().numpy().reshape(L, 4)
        assert np.abs(b[:, 0] - expected).max() <= 0.03 * abs(expected), b[:, 0]
        assert np.all(b < 0.5 * expected) and np.all(b > 2.0 * expected)
    # the finite parts from disjoint windows agree (the regularised spectrum) to what the sinc
    # quadrature's 1.5e-4 relative error over the image window allows, while the raw spectra move
    # by ~ (2 Z / b) ln(80 / 64) = 0.22 Ha between the two sets
    assert np.abs(A1.cpu().numpy() - A2.cpu().numpy()).max() <= 2e-3
    assert np.abs(e1.cpu().numpy() - e2.cpu().numpy()).min() > 0.15
