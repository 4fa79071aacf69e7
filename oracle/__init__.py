"""Plain FP64 CPU oracle for the lattice core-Hamiltonian path (TEST INFRASTRUCTURE ONLY).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA library: the arithmetic lives in
``lhf_oracle.c`` (compiled with gcc, loaded through ctypes), except for the Bloch eigenvectors
(``k_point_eigenvectors``, ``lattice_eigenvector``), the Bloch orbitals on the grid
(``bloch_orbital``, ``p1_mass_matrix``), the separable k-space route (``kspace_blocks``) and the
energy per cell of the lowest states (``cell_energy``), written here in numpy; the rest of this
module only marshals arguments.  See ``lhf_oracle.c`` for the passages of the paper each function
follows.  ``oracle.extended`` compiles the same source with long double arithmetic and solves
pencils in 50 digits: the exact values against which the FP64 rounding of this oracle is pinned.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lhf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblhf_oracle.so")
# a test may point the wrapper at another build of the oracle source (planted-mistake checks)
_LIB_OVERRIDE = os.environ.get("LHF_ORACLE_LIB")
_lock = threading.Lock()
_lib = None

NOT_SPD = -3
# a Bloch function is removed at a k-point when its overlap diagonal is below this fraction of
# its cell-periodic norm (numerically absent in FP64; see orc_k_point_eigenvalues)
DROP_TOL = 1e-6
# canonical orthogonalisation: directions of the diagonally scaled overlap with eigenvalue below
# this threshold are dropped (near-linear dependence)
LINDEP_TOL = 1e-8


def compile_source(src: str, out: str) -> str:
    """gcc -O2 (no FMA contraction) of an oracle source file into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile lhf_oracle.c into liblhf_oracle.so (gcc, -O2, no FMA contraction)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


class _System(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int * 3),
        ("b", ctypes.c_double * 3),
        ("periodic", ctypes.c_int * 3),
        ("n", ctypes.c_int * 3),
        ("n_cell", ctypes.c_int * 3),
        ("h", ctypes.c_double * 3),
        ("x0", ctypes.c_double * 3),
        ("cell0", ctypes.c_double * 3),
        ("K_sum", ctypes.c_int * 3),
        ("M0", ctypes.c_int),
        ("Z", ctypes.POINTER(ctypes.c_double)),
        ("Z_cell", ctypes.POINTER(ctypes.c_double)),
        ("a", ctypes.POINTER(ctypes.c_double)),
        ("m0", ctypes.c_int),
        ("kind", ctypes.POINTER(ctypes.c_int)),
        ("alpha", ctypes.POINTER(ctypes.c_double)),
        ("centre", ctypes.POINTER(ctypes.c_double)),
        ("R", ctypes.c_int),
        ("u0", ctypes.c_double),
        ("du", ctypes.c_double),
        ("rho", ctypes.c_double),
    ]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            S = ctypes.POINTER(_System)
            sig = {
                "orc_sinc_nodes": (None, [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]),
                "orc_sinc_inverse_r": (ctypes.c_double, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                "orc_gauss_cell_integral": (ctypes.c_double, [ctypes.c_double] * 4),
                "orc_basis_sample": (ctypes.c_double, [S, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_potential_factor": (ctypes.c_double, [S, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_potential_factors": (None, [S, ctypes.c_int, _dp]),
                "orc_basis_samples": (None, [S, ctypes.c_int, ctypes.c_int, _dp]),
                "orc_gram_1d": (ctypes.c_int, [S, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]),
                "orc_core_blocks": (ctypes.c_int, [S, _dp, _dp]),
                "orc_core_dense": (ctypes.c_int, [S, _dp, _dp]),
                "orc_block_dft": (None, [_ip, ctypes.c_int, _dp, _dp]),
                "orc_jacobi_eigenvalues": (ctypes.c_int, [ctypes.c_int, _dp, _dp]),
                "orc_dense_gen_eigenvalues": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp]),
                "orc_herm_gen_eigenvalues": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp]),
                "orc_k_point_eigenvalues": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp, _ip]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    if a.dtype == np.float64:
        return a.ctypes.data_as(_dp)
    if a.dtype == np.int32:
        return a.ctypes.data_as(_ip)
    raise TypeError(a.dtype)


class System:
    """ctypes view of a workload dictionary (see lhf_workloads); keeps its arrays alive."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.Z = np.ascontiguousarray(cfg["Z"], dtype=np.float64)
        self.a = np.ascontiguousarray(cfg["a"], dtype=np.float64).reshape(-1)
        self.kind = np.ascontiguousarray(cfg["kind"], dtype=np.int32)
        self.alpha = np.ascontiguousarray(cfg["alpha"], dtype=np.float64)
        self.centre = np.ascontiguousarray(cfg["centre"], dtype=np.float64).reshape(-1)
        self.Z_cell = None if cfg.get("Z_cell") is None else np.ascontiguousarray(cfg["Z_cell"], dtype=np.float64).reshape(-1)
        s = _System()
        for f in ("L", "periodic", "n", "n_cell", "K_sum"):
            getattr(s, f)[:] = [int(v) for v in cfg[f]]
        for f in ("b", "h", "x0", "cell0"):
            getattr(s, f)[:] = [float(v) for v in cfg[f]]
        s.M0 = len(cfg["Z"])
        s.Z = _ptr(self.Z)
        s.Z_cell = _ptr(self.Z_cell) if self.Z_cell is not None else ctypes.cast(None, _dp)
        s.a = _ptr(self.a)
        s.m0 = len(cfg["alpha"])
        s.kind = _ptr(self.kind)
        s.alpha = _ptr(self.alpha)
        s.centre = _ptr(self.centre)
        s.R = int(cfg["R"])
        s.u0 = float(cfg["u0"])
        s.du = float(cfg["du"])
        s.rho = float(cfg["rho"])
        self.s = s
        self.m0 = s.m0
        self.Rt = s.M0 * s.R

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _sys(cfg) -> System:
    return cfg if isinstance(cfg, System) else System(cfg)


# --- quadrature and 1D factors ----------------------------------------------------------------

def sinc_nodes(R: int, u0: float, du: float):
    t = np.empty(R)
    w = np.empty(R)
    _load().orc_sinc_nodes(R, u0, du, _ptr(t), _ptr(w))
    return t, w


def sinc_inverse_r(R: int, u0: float, du: float, r) -> np.ndarray:
    lib = _load()
    r = np.atleast_1d(np.asarray(r, dtype=np.float64))
    return np.array([lib.orc_sinc_inverse_r(R, u0, du, float(x)) for x in r])


def gauss_cell_integral(t: float, lo: float, hi: float, c: float) -> float:
    return _load().orc_gauss_cell_integral(float(t), float(lo), float(hi), float(c))


def basis_samples(cfg, l: int, cell: int = 0) -> np.ndarray:
    s = _sys(cfg)
    out = np.empty((s.m0, s.cfg["n"][l]))
    _load().orc_basis_samples(s.ref, l, cell, _ptr(out))
    return out


def potential_factors(cfg, l: int) -> np.ndarray:
    """[R_tot][n_l] potential factors of direction l (periodic ones replicated per cell)."""
    s = _sys(cfg)
    out = np.empty((s.Rt, s.cfg["n"][l]))
    _load().orc_potential_factors(s.ref, l, _ptr(out))
    return out


def gram_1d(cfg, l: int, p: int, q: int, V: np.ndarray | None = None):
    """(C [R_tot][m0][m0], K [m0][m0], M [m0][m0]) between cell-p and cell-q copies along l."""
    s = _sys(cfg)
    if V is None:
        V = potential_factors(s, l)
    V = np.ascontiguousarray(V, dtype=np.float64)
    C = np.empty((s.Rt, s.m0, s.m0))
    K = np.empty((s.m0, s.m0))
    M = np.empty((s.m0, s.m0))
    rc = _load().orc_gram_1d(s.ref, l, p, q, _ptr(V), _ptr(C), _ptr(K), _ptr(M))
    if rc != 0:
        raise MemoryError(rc)
    return C, K, M


def rank_coefficients(cfg) -> np.ndarray:
    s = _sys(cfg)
    t, w = sinc_nodes(s.cfg["R"], s.cfg["u0"], s.cfg["du"])
    return np.concatenate([z * w for z in s.cfg["Z"]])


# --- assembled matrices -----------------------------------------------------------------------

def core_blocks(cfg):
    """First block column (H_j, S_j), shape [L0, L1, L2, m0, m0] each (periodic lattices)."""
    s = _sys(cfg)
    L = s.cfg["L"]
    H = np.empty((L[0], L[1], L[2], s.m0, s.m0))
    S = np.empty_like(H)
    rc = _load().orc_core_blocks(s.ref, _ptr(H), _ptr(S))
    if rc != 0:
        raise MemoryError(rc)
    return H, S


def core_dense(cfg):
    """Full N_b x N_b (H, S), index (cell, mu) with cell = (p0 L1 + p1) L2 + p2."""
    s = _sys(cfg)
    L = s.cfg["L"]
    Nb = s.m0 * L[0] * L[1] * L[2]
    H = np.empty((Nb, Nb))
    S = np.empty((Nb, Nb))
    rc = _load().orc_core_dense(s.ref, _ptr(H), _ptr(S))
    if rc != 0:
        raise MemoryError(rc)
    return H, S


def block_dft(A: np.ndarray) -> np.ndarray:
    """Direct DFT of blocks A[L0, L1, L2, m, m] -> complex128 of the same shape."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    L = np.ascontiguousarray(A.shape[:3], dtype=np.int32)
    m = A.shape[3]
    out = np.empty(A.shape + (2,))
    _load().orc_block_dft(_ptr(L), m, _ptr(A), _ptr(out))
    return out[..., 0] + 1j * out[..., 1]


def jacobi_eigenvalues(A: np.ndarray) -> np.ndarray:
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    ev = np.empty(A.shape[0])
    _load().orc_jacobi_eigenvalues(A.shape[0], _ptr(A), _ptr(ev))
    return ev


def dense_gen_eigenvalues(H: np.ndarray, S: np.ndarray) -> np.ndarray:
    H = np.ascontiguousarray(H, dtype=np.float64)
    S = np.ascontiguousarray(S, dtype=np.float64)
    ev = np.empty(H.shape[0])
    rc = _load().orc_dense_gen_eigenvalues(H.shape[0], _ptr(H), _ptr(S), _ptr(ev))
    if rc != 0:
        raise np.linalg.LinAlgError(f"overlap matrix not positive definite ({rc})")
    return ev


def _as_interleaved(X: np.ndarray) -> np.ndarray:
    X = np.asarray(X)
    out = np.empty(X.shape + (2,))
    out[..., 0] = X.real
    out[..., 1] = X.imag
    return np.ascontiguousarray(out)


def k_point_eigenvalues(Hbar: np.ndarray, Sbar: np.ndarray, tau: float = DROP_TOL,
                        tau2: float = LINDEP_TOL):
    """Eigenvalues [K, m] (ascending, removed slots +inf) and status [K] (number of removed
    Bloch functions, or NOT_SPD) for blocks Hbar, Sbar [..., m, m] of all k-points."""
    m = Hbar.shape[-1]
    Hi = _as_interleaved(Hbar.reshape(-1, m, m))
    Si = _as_interleaved(Sbar.reshape(-1, m, m))
    K = Hi.shape[0]
    eig = np.empty((K, m))
    st = np.empty(K, dtype=np.int32)
    _load().orc_k_point_eigenvalues(K, m, _ptr(Hi), _ptr(Si), float(tau), float(tau2), _ptr(eig), _ptr(st))
    return eig, st


def kspace_blocks(cfg):
    """k-point blocks (Hbar, Sbar) [L0, L1, L2, m0, m0] of a periodic lattice by the separable
    route (Theorem 2.5; Prop. 4.2): for every direction l the factors between the copy in cell j
    and cell 0, C_r[j], K[j], M[j] (gram_1d, the per-entry formula of Lemma 3.1), are transformed
    by the direct 1D DFT Fl(kappa) = sum_j omega^(kappa j) X[j], omega = exp(-2 pi i / L_l), and
    each k-point block is the Hadamard-product form of Lemma 4.1 in the transformed factors:
    Sbar = M0 M1 M2, Hbar = (K0 M1 M2 + M0 K1 M2 + M0 M1 K2) / 2 - sum_r c_r C0_r C1_r C2_r."""
    s = _sys(cfg)
    L = [int(v) for v in s.cfg["L"]]
    c = rank_coefficients(s)
    F = []
    for l in range(3):
        V = potential_factors(s, l)
        X = np.empty((L[l], s.Rt + 2, s.m0, s.m0))
        for j in range(L[l]):
            C, K, M = gram_1d(s, l, j, 0, V)
            X[j, :s.Rt], X[j, s.Rt], X[j, s.Rt + 1] = C, K, M
        j = np.arange(L[l])
        Wm = np.exp(-2j * np.pi * np.outer(j, j) / L[l])  # [kappa, j]
        F.append(np.einsum("kj,jsab->ksab", Wm, X))
    Hb = np.empty((L[0], L[1], L[2], s.m0, s.m0), dtype=np.complex128)
    Sb = np.empty_like(Hb)
    for k0 in range(L[0]):
        for k1 in range(L[1]):
            for k2 in range(L[2]):
                A0, A1, A2 = F[0][k0], F[1][k1], F[2][k2]
                Rt = s.Rt
                V = np.einsum("r,rab,rab,rab->ab", c, A0[:Rt], A1[:Rt], A2[:Rt])
                T = A0[Rt] * A1[Rt + 1] * A2[Rt + 1] + A0[Rt + 1] * A1[Rt] * A2[Rt + 1] \
                    + A0[Rt + 1] * A1[Rt + 1] * A2[Rt]
                Sb[k0, k1, k2] = A0[Rt + 1] * A1[Rt + 1] * A2[Rt + 1]
                Hb[k0, k1, k2] = 0.5 * T - V
    return Hb, Sb


def k_point_eigenvectors(Hbar: np.ndarray, Sbar: np.ndarray, tau: float = DROP_TOL,
                         tau2: float = LINDEP_TOL):
    """Eigenpairs of Hbar_k u = lambda Sbar_k u at every k-point (eq. (4.7); Prop. 6.1).

    Steps, in the order of k_point_eigenvalues (the readings of the removal rule and of the
    near-linear dependence are the same): functions i with Re Sbar_ii(k) <= tau s0_i (s0_i the
    mean over k of Re Sbar_ii) are removed at k; the kept pencil is scaled by D = diag(Sbar)^-1/2
    and its Hermitian part taken; canonical orthogonalisation of the scaled overlap,
    S~ = V diag(s) V^H, keeps the directions with s >= tau2, X = V_kept diag(s)^-1/2; the reduced
    Hermitian matrix C = X^H H~ X is diagonalised (numpy.linalg.eigh, the library step), and
    u = D X w.  Returns eig [K, m] ascending (+inf in removed slots), vecs [K, m, m] complex
    (row r: eigenvector of the r-th eigenvalue over the m cell functions, 0 on removed
    functions, u^H Sbar u = 1; the first component of largest magnitude real and positive;
    zero rows in removed slots) and status [K] (removed directions)."""
    m = Hbar.shape[-1]
    Hb = np.asarray(Hbar).reshape(-1, m, m)
    Sb = np.asarray(Sbar).reshape(-1, m, m)
    K = Hb.shape[0]
    s0 = np.mean(Sb[:, np.arange(m), np.arange(m)].real, axis=0)
    eig = np.full((K, m), np.inf)
    vecs = np.zeros((K, m, m), dtype=np.complex128)
    status = np.zeros(K, dtype=np.int32)
    for k in range(K):
        d = Sb[k].diagonal().real
        kept = np.nonzero(d > tau * s0)[0]
        Dk = 1.0 / np.sqrt(d[kept])
        Hs = Hb[k][np.ix_(kept, kept)] * np.outer(Dk, Dk)
        Ss = Sb[k][np.ix_(kept, kept)] * np.outer(Dk, Dk)
        Hs = 0.5 * (Hs + Hs.conj().T)
        Ss = 0.5 * (Ss + Ss.conj().T)
        sig, Vs = np.linalg.eigh(Ss)
        keep2 = sig >= tau2
        X = Vs[:, keep2] / np.sqrt(sig[keep2])
        C = X.conj().T @ Hs @ X
        C = 0.5 * (C + C.conj().T)
        lam, W = np.linalg.eigh(C)
        U = (Dk[:, None] * (X @ W))  # kept functions x eigenpairs
        n = lam.shape[0]
        eig[k, :n] = lam
        status[k] = m - n
        for r in range(n):
            u = U[:, r]
            big = np.argmax(np.abs(u) ** 2)  # first index of the largest magnitude
            mag = abs(u[big])
            u = u * (np.conj(u[big]) / mag)
            u[big] = mag  # exactly real
            vecs[k, r, kept] = u
    return eig, vecs, status


def lattice_eigenvector(u: np.ndarray, kappa, L) -> np.ndarray:
    """The eigenvector of the lattice matrix built from the Bloch vector u at k-point
    kappa = (k0, k1, k2) (Prop. 6.1, eq. (6.8)): x on cell p = (p0, p1, p2), index
    ((p0 L1 + p1) L2 + p2) m + mu, is exp(2 pi i kappa . p / L) u_mu / sqrt(L0 L1 L2)."""
    L = [int(v) for v in L]
    p0, p1, p2 = np.meshgrid(np.arange(L[0]), np.arange(L[1]), np.arange(L[2]), indexing="ij")
    ph = np.exp(2j * np.pi * (kappa[0] * p0 / L[0] + kappa[1] * p1 / L[1] + kappa[2] * p2 / L[2]))
    return (ph.reshape(-1, 1) * np.asarray(u)[None, :]).reshape(-1) / np.sqrt(L[0] * L[1] * L[2])


def bloch_orbital(cfg, kappa, u, lo, cnt) -> np.ndarray:
    """Values of the Bloch orbital psi(x) = N^-1/2 sum_p exp(2 pi i kappa . p / L) sum_mu u_mu
    phi_mu(x - p b) (eq. (6.8) expanded in the basis, eq. (3.14)) on the grid window
    lo[l] .. lo[l] + cnt[l] - 1, complex [cnt0, cnt1, cnt2]: the sum over every lattice cell p
    of the translated (periodised) basis functions, each a product of its 1D samples."""
    s = _sys(cfg)
    L = [int(v) for v in s.cfg["L"]]
    win = []
    for l in range(3):
        win.append(np.stack([basis_samples(s, l, p)[:, lo[l]:lo[l] + cnt[l]] for p in range(L[l])]))
    u = np.asarray(u, dtype=np.complex128)
    psi = np.zeros(tuple(int(c) for c in cnt), dtype=np.complex128)
    for p0 in range(L[0]):
        for p1 in range(L[1]):
            for p2 in range(L[2]):
                ph = np.exp(2j * np.pi * (kappa[0] * p0 / L[0] + kappa[1] * p1 / L[1] + kappa[2] * p2 / L[2]))
                psi += ph * np.einsum("m,mi,mj,mk->ijk", u, win[0][p0], win[1][p1], win[2][p2], optimize=True)
    return psi / np.sqrt(L[0] * L[1] * L[2])


def p1_mass_matrix(n: int, h: float, periodic: bool) -> np.ndarray:
    """The 1D P1 mass matrix (h / 6) tridiag(1, 4, 1) (Sec. 3.4), circulant when periodic."""
    M = np.diag(np.full(n, 4.0)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    if periodic and n > 2:
        M[0, -1] = M[-1, 0] = 1.0
    return M * (h / 6.0)


def cell_energy(eig, n_low: int, cells: float):
    """Energy per cell of the lowest states (Sec. 5: the average energy per unit cell of a chain
    against L): the n_low smallest values of the spectrum eig -- any shape; the union of the
    k-point spectra of a lattice is the lattice matrix's spectrum (Prop. 6.1), an open box's is its
    dense pencil's; +inf (removed functions) sorts last -- summed in ascending order and divided by
    cells.  Returns (energy, the n_low-th smallest value)."""
    v = np.sort(np.ravel(np.asarray(eig, dtype=np.float64)))
    low = v[:int(n_low)]
    total = 0.0
    for x in low:
        total += float(x)
    return total / float(cells), float(low[-1])


def bloch_spectrum(cfg):
    """The whole path for a periodic lattice: blocks -> DFT -> per-k eigenvalues [K, m0]."""
    H, S = core_blocks(cfg)
    Hb = block_dft(H)
    Sb = block_dft(S)
    eig, st = k_point_eigenvalues(Hb, Sb)
    return eig, st
