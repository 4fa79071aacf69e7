"""Band data of a computed lattice spectrum as a text table (the spectral-band figures of Sec. 5,
written as data).

The spectrum of a periodic lattice is the union of the k-point spectra (Prop. 6.1); plotted
against the reduced wave vector q = kappa / L, the r-th eigenvalue of every k-point traces band r.
This module only formats host arrays already computed by the library (no arithmetic of the
method): one row per k-point in the library's order (kappa lexicographic over L0, L1, L2) with
kappa, q folded into (-1/2, 1/2], the status of the k-point, and the m0 eigenvalues ascending
(removed functions as inf).  Values are written with 17 significant digits, so a reader gets the
doubles back exactly."""

from __future__ import annotations

import numpy as np


def band_table(eig, L, k_status=None) -> np.ndarray:
    """Rows [n_kpoints, 7 + m0]: k0 k1 k2 q0 q1 q2 status e_1 .. e_m0 (float64)."""
    L = [int(v) for v in L]
    K = L[0] * L[1] * L[2]
    e = np.asarray(eig, dtype=np.float64).reshape(K, -1)
    st = np.zeros(K) if k_status is None else np.asarray(k_status, dtype=np.float64).reshape(K)
    k0, k1, k2 = np.meshgrid(np.arange(L[0]), np.arange(L[1]), np.arange(L[2]), indexing="ij")
    kap = np.stack([k0.ravel(), k1.ravel(), k2.ravel()], axis=1).astype(np.float64)
    q = kap / np.asarray(L, dtype=np.float64)
    q = np.where(q > 0.5, q - 1.0, q)
    return np.concatenate([kap, q, st[:, None], e], axis=1)


def write_bands(path: str, eig, L, k_status=None, title: str = "") -> None:
    """Writes band_table(eig, L, k_status) to path as whitespace-separated text with a header."""
    t = band_table(eig, L, k_status)
    m0 = t.shape[1] - 7
    head = (f"{title}\nL = {' '.join(str(int(v)) for v in L)}, m0 = {m0}\n"
            "k0 k1 k2 q0 q1 q2 status " + " ".join(f"e{r + 1}" for r in range(m0)))
    np.savetxt(path, t, fmt="%.17g", header=head.lstrip("\n"))
