"""Shared tolerances of the parity tests.

Matrix entries (FP64 path): |x - x_ref| <= 1e-12 * max|block_ref| per m0 x m0 block (an entry-wise
relative bound fails on entries that are zero up to rounding).

Eigenvalues.  Both sides remove the Bloch functions whose overlap diagonal cancelled to rounding
level (Re Sbar_ii(kappa) <= DROP_TOL * mean_kappa Re Sbar_ii); the removed slots are +inf and must
coincide.  For the kept pencil, a perturbation (dH, dS) moves an eigenvalue by at most
(||dH|| + |lambda| ||dS||) ||u||^2 to first order (u S-normalised).  Two backward-stable FP64
computations therefore agree within c eps (N_H + |lambda| N_S) ||u||^2, floored at the 1e-10 Ha
target, with N_H, N_S the norms that bound the rounding of the inputs: ||Hbar_kappa|| when both
solvers read the same blocks, and || sum_j |H_j| || (the block DFT's absolute error bound) when each
side assembled and transformed its own blocks.  c = 64 covers the accumulation of the reduction
steps.  ||u||^2 is large only where the kept overlap is nearly singular.
"""

import numpy as np
import scipy.linalg as sla

DROP_TOL = 1e-6


def block_rel_err(X, Xref, m0):
    """max over blocks of max|X - Xref| / max|Xref| (blocks of m0 x m0 over the last two axes)."""
    X = np.asarray(X).reshape(-1, m0, m0)
    Xref = np.asarray(Xref).reshape(-1, m0, m0)
    num = np.abs(X - Xref).reshape(len(X), -1).max(axis=1)
    den = np.abs(Xref).reshape(len(X), -1).max(axis=1)
    ok_zero = den == 0
    out = np.where(ok_zero, num, num / np.where(ok_zero, 1.0, den))
    return float(out.max())


def kept_functions(Sbar):
    """[K, m] boolean mask of the Bloch functions whose overlap diagonal did not cancel."""
    m0 = Sbar.shape[-1]
    Sb = Sbar.reshape(-1, m0, m0)
    d = np.real(np.einsum("kii->ki", Sb))
    s0 = d.mean(axis=0)
    return d > DROP_TOL * s0


def _reduced(H, S, n_keep):
    """Eigenpairs of the pencil as the solvers reduce it: scaled to unit overlap diagonal and,
    when fewer than all directions are kept, restricted to the n_keep largest overlap
    eigen-directions (canonical orthogonalisation).  Returns (lambda, u) with u S-normalised in
    the unscaled coordinates."""
    d = 1.0 / np.sqrt(np.real(np.diag(S)))
    Hs = H * np.outer(d, d)
    Ss = S * np.outer(d, d)
    if n_keep == len(d):
        lam, Y = sla.eigh(Hs, Ss)
        return lam, d[:, None] * Y
    sig, Vs = np.linalg.eigh(Ss)
    X = Vs[:, -n_keep:] / np.sqrt(sig[-n_keep:])
    lam, Y = np.linalg.eigh(X.conj().T @ Hs @ X)
    return lam, d[:, None] * (X @ Y)


def check_eigenvalues(eig, eig_ref, Hbar_ref, Sbar_ref, H_blocks=None, S_blocks=None, status=None,
                      floor=1e-10, c=64.0):
    """Per k-point comparison; returns (max |d lambda| over finite eigenvalues, max ratio to
    tolerance).  status: the number of removed slots per k-point (the oracle's k_status); when
    omitted, only the diagonal-cancellation rule is assumed.  Removed (+inf) slots must
    coincide, else the ratio is inf."""
    m0 = Hbar_ref.shape[-1]
    Hb = Hbar_ref.reshape(-1, m0, m0)
    Sb = Sbar_ref.reshape(-1, m0, m0)
    eig = np.asarray(eig).reshape(-1, m0)
    eig_ref = np.asarray(eig_ref).reshape(-1, m0)
    keep = kept_functions(Sbar_ref)
    eps = np.finfo(float).eps
    absH = absS = None
    if H_blocks is not None:
        absH = np.abs(np.asarray(H_blocks).reshape(-1, m0, m0)).sum(axis=0)
        absS = np.abs(np.asarray(S_blocks).reshape(-1, m0, m0)).sum(axis=0)
    worst, ratio = 0.0, 0.0
    for k in range(len(Hb)):
        idx = np.where(keep[k])[0]
        n = len(idx) if status is None else m0 - int(np.asarray(status).ravel()[k])
        if not (np.all(np.isinf(eig[k, n:])) and np.all(np.isinf(eig_ref[k, n:]))
                and np.all(np.isfinite(eig[k, :n])) and np.all(np.isfinite(eig_ref[k, :n]))):
            return float("inf"), float("inf")
        if n == 0:
            continue
        H = Hb[k][np.ix_(idx, idx)]
        S = Sb[k][np.ix_(idx, idx)]
        lam, U = _reduced(H, S, n)
        u2 = (np.abs(U) ** 2).sum(axis=0)
        if absH is None:
            nH, nS = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
        else:
            nH = np.linalg.norm(absH[np.ix_(idx, idx)], 2)
            nS = np.linalg.norm(absS[np.ix_(idx, idx)], 2)
        tol = np.maximum(floor, c * eps * (nH + np.abs(lam) * nS) * u2)
        d = np.abs(eig[k, :n] - eig_ref[k, :n])
        worst = max(worst, float(d.max()))
        ratio = max(ratio, float((d / tol).max()))
    return worst, ratio


def check_dense_eigenvalues(eig, eig_ref, H, S, dH=None, dS=None, floor=1e-10, c=None):
    """Dense generalized symmetric-definite eigenvalues (open box).  Both solvers are backward
    stable: each eigenvalue may move by (||dH|| + |lambda| ||dS||) ||u||^2 (u S-normalised, first
    order), with ||dH|| <= c eps ||H|| from the reductions (c = N: the growth bound of the
    Cholesky and Householder steps) plus, when the two sides start from different matrices, the
    measured input difference (dH, dS).  Returns (max |d lambda|, max ratio to tolerance)."""
    H = np.asarray(H)
    S = np.asarray(S)
    N = H.shape[0]
    if c is None:
        c = float(N)
    eps = np.finfo(float).eps
    lam, U = _reduced(H, S, N)
    u2 = (U ** 2).sum(axis=0)
    nH, nS = np.linalg.norm(H, 2), np.linalg.norm(S, 2)
    pH = c * eps * nH + (np.linalg.norm(dH, 2) if dH is not None else 0.0)
    pS = c * eps * nS + (np.linalg.norm(dS, 2) if dS is not None else 0.0)
    tol = np.maximum(floor, (pH + np.abs(lam) * pS) * u2)
    eig = np.asarray(eig).ravel()
    eig_ref = np.asarray(eig_ref).ravel()
    if not (np.all(np.isfinite(eig)) and np.all(np.isfinite(eig_ref))):
        return float("inf"), float("inf")
    d = np.abs(eig - eig_ref)
    return float(d.max()), float((d / tol).max())
