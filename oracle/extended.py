"""Extended-precision companion of the oracle (TEST INFRASTRUCTURE ONLY).

Only the tests may import this module.  It measures the rounding of the FP64 oracle: the same
source, ``lhf_oracle.c``, is compiled a second time with every ``double`` replaced by ``long
double`` and ``<math.h>`` by the type-generic ``<tgmath.h>``, so that each elementary function
and every sum runs in the extended format (x86: 64-bit significand, unit roundoff 5.4e-20, 2048
times finer than FP64; aarch64: IEEE quadruple).  Its assembled blocks are the exact discrete
blocks of eq. (3.10), Lemma 3.1 and Sec. 3.4 to about 1e-19 relative.  Generalized Hermitian
pencils (eq. (4.7)) are then solved in 50-digit arithmetic (mpmath: Cholesky, the standard
Hermitian problem, its eigen-decomposition), free of FP64 rounding.

What this pins: how far FP64 data and FP64 arithmetic move the spectrum of each k-point, i.e.
which Bloch eigenvalues FP64 can resolve to the 1e-10 Ha target at all (the removal rule of the
k-point solver) and whether the oracle's FP64 eigenvalues lie within the first-order
perturbation bound of the exact ones (the eigenvalue tolerance).  The formulas themselves are
pinned elsewhere (closed forms, brute force, invariants); this module adds only precision.
"""

from __future__ import annotations

import ctypes
import os
import re
import subprocess
import threading

import numpy as np

from . import _SRC, System

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liblhf_oracle_ld.so")
_lock = threading.Lock()
_lib = None

LD = np.longdouble
_ldp = ctypes.POINTER(ctypes.c_longdouble)
_ip = ctypes.POINTER(ctypes.c_int)


def extended_source(src_text: str) -> str:
    """The oracle source with long double arithmetic: the type replaced everywhere, the
    type-generic math header (exp, erf, sqrt, ... resolve to their long double versions), and
    the three literals whose double rounding would otherwise leak into the extended results (pi,
    e as exp(1.0), and the Newton stopping tolerance of the Gauss-Legendre nodes) written in long
    double."""
    t = src_text.replace("#include <math.h>", "#include <tgmath.h>")
    t = re.sub(r"\bdouble\b", "long double", t)
    t = t.replace("3.14159265358979323846;", "3.14159265358979323846264338327950288L;")
    t = t.replace("exp(1.0)", "exp(1.0L)")
    t = t.replace("fabs(dx) < 1e-17", "fabs(dx) < 1e-30L")
    if "long long double" in t:
        raise RuntimeError("oracle source already used long double")
    return t


def build(force: bool = False) -> str:
    """Compile the long double variant of lhf_oracle.c (gcc -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        src = _LIB_PATH + f".{os.getpid()}.c"
        with open(src, "w") as f:
            f.write(extended_source(open(_SRC).read()))
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        try:
            subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", src, "-o", tmp,
                            "-lm"], check=True)
            os.replace(tmp, _LIB_PATH)
        finally:
            if os.path.exists(src):
                os.unlink(src)
    return _LIB_PATH


class _SystemLD(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int * 3),
        ("b", ctypes.c_longdouble * 3),
        ("periodic", ctypes.c_int * 3),
        ("n", ctypes.c_int * 3),
        ("n_cell", ctypes.c_int * 3),
        ("h", ctypes.c_longdouble * 3),
        ("x0", ctypes.c_longdouble * 3),
        ("cell0", ctypes.c_longdouble * 3),
        ("K_sum", ctypes.c_int * 3),
        ("M0", ctypes.c_int),
        ("Z", _ldp),
        ("Z_cell", _ldp),
        ("a", _ldp),
        ("m0", ctypes.c_int),
        ("kind", _ip),
        ("alpha", _ldp),
        ("centre", _ldp),
        ("R", ctypes.c_int),
        ("u0", ctypes.c_longdouble),
        ("du", ctypes.c_longdouble),
        ("rho", ctypes.c_longdouble),
    ]


class _LDResult(ctypes.c_longdouble):
    """A long double result kept as a ctypes object (a plain c_longdouble result would be
    converted to a Python float, i.e. rounded to double)."""


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            S = ctypes.POINTER(_SystemLD)
            lib.orc_core_blocks.restype = ctypes.c_int
            lib.orc_core_blocks.argtypes = [S, _ldp, _ldp]
            lib.orc_block_dft.restype = None
            lib.orc_block_dft.argtypes = [_ip, ctypes.c_int, _ldp, _ldp]
            lib.orc_gauss_cell_integral.restype = _LDResult
            lib.orc_gauss_cell_integral.argtypes = [ctypes.c_longdouble] * 4
            _lib = lib
    return _lib


def _ld(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(LD).reshape(-1))


def _ldptr(a: np.ndarray):
    assert a.dtype == LD and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_ldp)


class _LDSystem:
    """long double view of a workload dictionary (the same input numbers as the FP64 oracle:
    every input is an FP64 number, held exactly in the wider format)."""

    def __init__(self, cfg: dict):
        base = System(cfg)
        self.cfg = cfg
        self.Z, self.a, self.alpha, self.centre = _ld(cfg["Z"]), _ld(cfg["a"]), _ld(cfg["alpha"]), _ld(cfg["centre"])
        self.kind = np.ascontiguousarray(cfg["kind"], dtype=np.int32)
        self.Z_cell = None if cfg.get("Z_cell") is None else _ld(cfg["Z_cell"])
        s = _SystemLD()
        b = base.s
        for f in ("L", "periodic", "n", "n_cell", "K_sum"):
            getattr(s, f)[:] = list(getattr(b, f))
        for f in ("b", "h", "x0", "cell0"):
            getattr(s, f)[:] = [float(v) for v in getattr(b, f)]
        s.M0, s.m0, s.R = b.M0, b.m0, b.R
        s.Z, s.a, s.alpha, s.centre = _ldptr(self.Z), _ldptr(self.a), _ldptr(self.alpha), _ldptr(self.centre)
        s.Z_cell = _ldptr(self.Z_cell) if self.Z_cell is not None else ctypes.cast(None, _ldp)
        s.kind = self.kind.ctypes.data_as(_ip)
        s.u0, s.du, s.rho = b.u0, b.du, b.rho
        self.s = s
        self.m0 = b.m0


def core_blocks(cfg):
    """First block column (H_j, S_j) [L0, L1, L2, m0, m0] in long double."""
    s = _LDSystem(cfg)
    L = cfg["L"]
    H = np.empty((L[0], L[1], L[2], s.m0, s.m0), dtype=LD)
    S = np.empty_like(H)
    rc = _load().orc_core_blocks(ctypes.byref(s.s), _ldptr(H), _ldptr(S))
    if rc != 0:
        raise MemoryError(rc)
    return H, S


def gauss_cell_integral(t: float, lo: float, hi: float, c: float):
    """The oracle's cell integral of exp(-t^2 (x - c)^2) over [lo, hi], in long double."""
    r = _load().orc_gauss_cell_integral(t, lo, hi, c)
    return np.frombuffer(bytes(r), dtype=LD)[0]


def block_dft(A: np.ndarray):
    """Direct DFT of long double blocks A[L0, L1, L2, m, m]: (real, imaginary) parts in long
    double, each of A's shape."""
    A = np.ascontiguousarray(A, dtype=LD)
    L = np.ascontiguousarray(A.shape[:3], dtype=np.int32)
    m = A.shape[3]
    out = np.empty(A.shape + (2,), dtype=LD)
    _load().orc_block_dft(L.ctypes.data_as(_ip), m, _ldptr(A), _ldptr(out))
    return out[..., 0], out[..., 1]


# --- 50-digit pencils ---------------------------------------------------------------------------

def _mpf(x):
    import mpmath

    # a long double is held exactly by its two nearest-double parts
    hi = float(x)
    lo = float(LD(x) - LD(hi))
    return mpmath.mpf(hi) + mpmath.mpf(lo)


def to_mp_matrix(re_part, im_part=None):
    """mpmath complex matrix from real and imaginary parts (float64 or long double arrays),
    converted exactly."""
    import mpmath

    m = re_part.shape[0]
    M = mpmath.matrix(m, m)
    for a in range(m):
        for b in range(m):
            v = _mpf(re_part[a, b])
            if im_part is not None:
                v = mpmath.mpc(v, _mpf(im_part[a, b]))
            M[a, b] = v
    return M


def pencil_eigen(Hm, Sm, dps: int = 50, vectors: bool = False):
    """Eigenvalues (ascending, as mpf) of the Hermitian pencil H u = lambda S u, S positive
    definite, in `dps`-digit arithmetic, of the Hermitian parts of H and S: S = G G^H,
    C = G^-1 H G^-H (its Hermitian part), then
    the Hermitian eigenproblem of C.  With vectors, also the S-normalised eigenvectors u_k
    (columns of an mpmath matrix).  The inputs are taken as exact."""
    import mpmath

    with mpmath.workdps(dps):
        m = Hm.rows
        # the Hermitian parts: a transformed block is Hermitian only up to its rounding
        Hm = (Hm + Hm.H) / 2
        Sm = (Sm + Sm.H) / 2
        G = mpmath.cholesky(Sm)
        Gi = mpmath.inverse(G)
        C = Gi * Hm * Gi.H
        C = (C + C.H) / 2
        E, Q = mpmath.eighe(C)
        order = sorted(range(m), key=lambda k: E[k])
        ev = [E[k] for k in order]
        if not vectors:
            return ev
        U = Gi.H * Q
        Us = mpmath.matrix(m, m)
        for c, k in enumerate(order):
            for a in range(m):
                Us[a, c] = U[a, k]
        return ev, Us


def canonical_eigen(Hm, Sm, sigma_cut: float, dps: int = 50):
    """Eigenvalues (ascending mpf) of the Hermitian pencil after the same two readings as the
    oracle, in `dps`-digit arithmetic: scaling to unit overlap diagonal (a congruence, D =
    diag(S)^-1/2), then canonical orthogonalisation -- the eigen-decomposition S~ = V diag(s) V^H
    of the scaled overlap, the directions with s >= sigma_cut kept, X = V_kept diag(s)^-1/2 and
    the Hermitian eigenproblem of X^H H~ X.  Returns (eigenvalues, number of directions
    dropped)."""
    import mpmath

    with mpmath.workdps(dps):
        m = Hm.rows
        Hm = (Hm + Hm.H) / 2
        Sm = (Sm + Sm.H) / 2
        d = [1 / mpmath.sqrt(mpmath.re(Sm[i, i])) for i in range(m)]
        Hs = mpmath.matrix(m, m)
        Ss = mpmath.matrix(m, m)
        for a in range(m):
            for b in range(m):
                Hs[a, b] = Hm[a, b] * d[a] * d[b]
                Ss[a, b] = Sm[a, b] * d[a] * d[b]
        s, V = mpmath.eighe(Ss)
        keep = [c for c in range(m) if s[c] >= sigma_cut]
        X = mpmath.matrix(m, len(keep))
        for cc, c in enumerate(keep):
            f = 1 / mpmath.sqrt(s[c])
            for a in range(m):
                X[a, cc] = V[a, c] * f
        if not keep:
            return [], m
        C = X.H * Hs * X
        C = (C + C.H) / 2
        E = mpmath.eighe(C, eigvals_only=True)
        return sorted(E[c] for c in range(len(keep))), m - len(keep)
