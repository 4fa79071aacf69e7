"""Shared tolerances of the parity tests.

Matrix entries (FP64 path): |x - x_ref| <= 1e-12 * max|block_ref| per m0 x m0 block (an entry-wise
relative bound fails on entries that are zero up to rounding).

Eigenvalues: a backward-stable solver of H u = lambda S u returns eigenvalues of a pencil within
eps * (||H||, ||S||); to first order |d lambda| <= (||dH|| + |lambda| ||dS||) ||u||^2 for the
S-normalised eigenvector u.  Two such solvers (the GPU's and the oracle's) therefore agree within
c eps (||H|| + |lambda| ||S||) ||u||^2, floored at the 1e-10 Ha target; c = 64 covers the
accumulation of the DFT and reduction steps.  ||u||^2 is large only where S is nearly singular.
"""

import numpy as np
import scipy.linalg as sla


def block_rel_err(X, Xref, m0):
    """max over blocks of max|X - Xref| / max|Xref| (blocks of m0 x m0 over the last two axes)."""
    X = np.asarray(X).reshape(-1, m0, m0)
    Xref = np.asarray(Xref).reshape(-1, m0, m0)
    num = np.abs(X - Xref).reshape(len(X), -1).max(axis=1)
    den = np.abs(Xref).reshape(len(X), -1).max(axis=1)
    ok_zero = den == 0
    out = np.where(ok_zero, num, num / np.where(ok_zero, 1.0, den))
    return float(out.max())


def eig_tolerance(Hb, Sb, lam, floor=1e-10, c=64.0):
    eps = np.finfo(float).eps
    _, U = sla.eigh(Hb, Sb)
    u2 = (np.abs(U) ** 2).sum(axis=0)
    nH = np.linalg.norm(Hb, 2)
    nS = np.linalg.norm(Sb, 2)
    return np.maximum(floor, c * eps * (nH + np.abs(lam) * nS) * u2)


def check_eigenvalues(eig, eig_ref, Hbar_ref, Sbar_ref, floor=1e-10):
    """Per k-point conditioning-aware comparison; returns (max |d lambda|, max ratio to tol)."""
    m0 = Hbar_ref.shape[-1]
    Hb = Hbar_ref.reshape(-1, m0, m0)
    Sb = Sbar_ref.reshape(-1, m0, m0)
    eig = np.asarray(eig).reshape(-1, m0)
    eig_ref = np.asarray(eig_ref).reshape(-1, m0)
    worst, ratio = 0.0, 0.0
    for k in range(len(Hb)):
        tol = eig_tolerance(Hb[k], Sb[k], eig_ref[k], floor=floor)
        d = np.abs(eig[k] - eig_ref[k])
        worst = max(worst, float(d.max()))
        ratio = max(ratio, float((d / tol).max()))
    return worst, ratio
