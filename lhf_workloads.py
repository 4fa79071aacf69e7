"""Seeded synthetic lattice workloads: inputs only.

This module draws the geometry of a lattice system (cells, nuclei, Gaussian basis, grid,
quadrature parameters) from a seeded PCG64 stream. It contains none of the method's
arithmetic: no basis sampling, no potential, no matrix entries. Both the CUDA path and the
CPU oracle consume the plain dictionaries it returns.

Conventions (atomic units: bohr, Hartree):
  * direction l = 0, 1, 2 (x, y, z); ``L[l]`` cells of side ``b[l]``; ``periodic[l]`` marks
    a block-circulant direction (supercell of ``L[l]`` cells, Sec. 4.1 of the paper).
  * grid nodes are cell centres ``x_i = x0 + (i + 1/2) h``, ``i = 0 .. n-1``; in a lattice
    direction (``L > 1`` or periodic) the cells of the lattice hold ``n_cell`` nodes each and
    lattice cell 0 starts at ``cell0``; a single-cell open direction has ``n_cell = n``.
  * nucleus ``nu`` of lattice cell ``k`` sits at ``a[nu] + k * b`` (lattice directions),
    with charge ``Z[nu]``, or ``Z_cell[k][nu]`` when given (open boxes with mixed charges).
  * basis function ``mu`` of cell ``k`` is the separable Gaussian of kind ``kind[mu]``
    (0 = s, 1/2/3 = p along x/y/z), exponent ``alpha[mu]``, centred at ``centre[mu] + k b``;
    its 1D factors are cut at radius ``sqrt(rho / alpha)``.
  * the Newton kernel is the sinc quadrature with ``R`` nodes ``t_q = exp(u0 + q du)``.
  * ``K_sum[l]`` lattice images enter the periodic potential sum of direction ``l``.
"""

from __future__ import annotations

import math

import numpy as np

# Sinc-quadrature parameters (u0, du) per (R, r_min, r_max) class. They were chosen by the
# committed search script ``oracle/sinc_fit.py`` (it minimises the max relative error of the
# exponential sum against 1/r on [r_min, r_max]); they are plain input numbers here.
SINC_TABLE = {
    # name: (R, u0, du)        max relative error of the sum against 1/r on [r_min, r_max]
    "periodic_8": (24, -5.9987, 0.4452),  # 7.9e-05 on [0.03125, 16]
    "tube_256": (32, -8.9662, 0.4586),  # 8.4e-05 on [0.0109, 362]
    "box_64": (32, -8.4614, 0.4223),  # 4.3e-05 on [0.025, 186]
    "cubic_32": (32, -8.0245, 0.4189),  # 2.3e-05 on [0.0156, 60]
    "small": (20, -6.8657, 0.557),  # 4.4e-04 on [0.04, 60]
    "hetero_24": (24, -9.7916, 0.6024),  # 8.7e-04 on [0.025, 1500]
    "hetero_32": (32, -10.1649, 0.4724),  # 1.5e-04 on [0.025, 1500]
}

RHO = 40.0  # basis truncation: exp(-40) ~ 4e-18 of the peak


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _stratified_loguniform(rng: np.random.Generator, count: int, lo: float, hi: float) -> np.ndarray:
    """One draw per equal log-width stratum of [lo, hi] (log-uniform overall, no near-duplicates
    within a stratum pair), returned in draw order."""
    u = rng.random(count)
    edges = np.log(lo) + (np.arange(count) + u) * (np.log(hi) - np.log(lo)) / count
    return np.exp(edges)


def _basis_s_p(rng, m0, n_s, n_pshell, lo, hi, nuclei_pos, extra_p_dir=None):
    """n_s s-functions and n_pshell p-shells (px, py, pz sharing one exponent); s-function k and
    p-shell k sit on nucleus k mod M0. ``extra_p_dir`` adds single p functions (own exponents)."""
    M0 = len(nuclei_pos)
    kinds, alphas, centres = [], [], []
    a_s = _stratified_loguniform(rng, n_s, lo, hi)
    for k in range(n_s):
        kinds.append(0)
        alphas.append(a_s[k])
        centres.append(nuclei_pos[k % M0])
    a_p = _stratified_loguniform(rng, n_pshell, lo, hi)
    for k in range(n_pshell):
        for d in range(3):
            kinds.append(1 + d)
            alphas.append(a_p[k])
            centres.append(nuclei_pos[k % M0])
    if extra_p_dir:
        a_x = _stratified_loguniform(rng, len(extra_p_dir), lo, hi)
        for k, d in enumerate(extra_p_dir):
            kinds.append(1 + d)
            alphas.append(a_x[k])
            centres.append(nuclei_pos[k % M0])
    assert len(kinds) == m0, (len(kinds), m0)
    return kinds, alphas, centres


def _system(L, b, periodic, n, n_cell, h, x0, cell0, K_sum, Z, a, kinds, alphas, centres,
            sinc_key, name, Z_cell=None, seed=None):
    R, u0, du = SINC_TABLE[sinc_key]
    return {
        "name": name,
        "seed": seed,
        "L": [int(v) for v in L],
        "b": [float(v) for v in b],
        "periodic": [int(v) for v in periodic],
        "n": [int(v) for v in n],
        "n_cell": [int(v) for v in n_cell],
        "h": [float(v) for v in h],
        "x0": [float(v) for v in x0],
        "cell0": [float(v) for v in cell0],
        "K_sum": [int(v) for v in K_sum],
        "Z": [float(v) for v in Z],
        "Z_cell": None if Z_cell is None else [[float(z) for z in row] for row in Z_cell],
        "a": [[float(c) for c in row] for row in a],
        "kind": [int(v) for v in kinds],
        "alpha": [float(v) for v in alphas],
        "centre": [[float(c) for c in row] for row in centres],
        "R": int(R),
        "u0": float(u0),
        "du": float(du),
        "rho": RHO,
    }


def _tube(seed, name, L, b, n_c, n_perp, half_width, M0, m0_s, m0_pshell, lo, hi, K_sum, sinc_key,
          extra_p_dir=None):
    """Periodic (L,1,1) tube: lattice direction x, open square cross-section [-w, w]^2."""
    rng = _rng(seed)
    h1 = b / n_c
    hp = 2.0 * half_width / n_perp
    pos = []
    for _ in range(M0):
        off = rng.uniform(-b / 4.0, b / 4.0, size=3)
        pos.append([b / 2.0 + off[0], off[1], off[2]])
    m0 = m0_s + 3 * m0_pshell + (len(extra_p_dir) if extra_p_dir else 0)
    kinds, alphas, centres = _basis_s_p(rng, m0, m0_s, m0_pshell, lo, hi, pos, extra_p_dir)
    return _system(
        L=[L, 1, 1], b=[b, 2 * half_width, 2 * half_width], periodic=[1, 0, 0],
        n=[L * n_c, n_perp, n_perp], n_cell=[n_c, n_perp, n_perp], h=[h1, hp, hp],
        x0=[0.0, -half_width, -half_width], cell0=[0.0, -half_width, -half_width],
        K_sum=[K_sum, 1, 1], Z=[1.0] * M0, a=pos, kinds=kinds, alphas=alphas, centres=centres,
        sinc_key=sinc_key, name=name, seed=seed)


def periodic_8(seed: int = 1) -> dict:
    """Periodic (8,1,1) lattice, b = 2.0, one Z=1 nucleus at a seeded offset, m0 = 4 s-type
    Gaussians with exponents 0.1*3^j on the nucleus, h = 0.0625 (n1 = 256, n2 = n3 = 256 on
    [-8, 8]), R = 24 sinc terms, K_sum = 8 images."""
    rng = _rng(seed)
    b = 2.0
    off = rng.uniform(-b / 4.0, b / 4.0, size=3)
    pos = [[b / 2.0 + off[0], off[1], off[2]]]
    alphas = [0.1 * 3.0 ** j for j in range(4)]
    return _system(
        L=[8, 1, 1], b=[b, 16.0, 16.0], periodic=[1, 0, 0], n=[256, 256, 256],
        n_cell=[32, 256, 256], h=[0.0625] * 3, x0=[0.0, -8.0, -8.0], cell0=[0.0, -8.0, -8.0],
        K_sum=[8, 1, 1], Z=[1.0], a=pos, kinds=[0] * 4, alphas=alphas, centres=pos * 4,
        sinc_key="periodic_8", name="periodic_8", seed=seed)


def tube_256(seed: int = 3) -> dict:
    """Periodic (256,1,1) tube, b = 2.8, two Z=1 nuclei at seeded offsets, m0 = 16 (4 s + 4
    p-shells) with exponents log-uniform in [0.04, 30], 128 nodes per cell along x
    (n1 = 32768), n2 = n3 = 256 on [-8, 8], R = 32 (R_tot = 64), K_sum = 256."""
    return _tube(seed, "tube_256", L=256, b=2.8, n_c=128, n_perp=256, half_width=8.0, M0=2,
                 m0_s=4, m0_pshell=4, lo=0.04, hi=30.0, K_sum=256, sinc_key="tube_256")


def tube(L: int, seed: int, n_c: int = 32, n_perp: int = 64, half_width: float = 8.0,
         M0: int = 2, m0_s: int = 4, m0_pshell: int = 4, lo: float = 0.04, hi: float = 30.0,
         b: float = 2.8, K_sum: int | None = None, sinc_key: str = "small") -> dict:
    """A smaller periodic tube of the tube_256 family (parity-test sizes)."""
    return _tube(seed, f"tube_{L}", L=L, b=b, n_c=n_c, n_perp=n_perp, half_width=half_width,
                 M0=M0, m0_s=m0_s, m0_pshell=m0_pshell, lo=lo, hi=hi,
                 K_sum=L if K_sum is None else K_sum, sinc_key=sinc_key)


def cubic_32(seed: int = 5, L: int = 32, n_c: int = 64) -> dict:
    """Periodic (L,L,L) lattice, b = 2.0, one Z=1 nucleus, m0 = 16 (4 s + 4 p-shells) with
    exponents log-uniform in [0.05, 20], n_c nodes per cell per direction, R = 32,
    K_sum = L per direction."""
    rng = _rng(seed)
    b = 2.0
    off = rng.uniform(-b / 4.0, b / 4.0, size=3)
    pos = [[b / 2.0 + off[0], b / 2.0 + off[1], b / 2.0 + off[2]]]
    kinds, alphas, centres = _basis_s_p(rng, 16, 4, 4, 0.05, 20.0, pos)
    return _system(
        L=[L] * 3, b=[b] * 3, periodic=[1, 1, 1], n=[L * n_c] * 3, n_cell=[n_c] * 3,
        h=[b / n_c] * 3, x0=[0.0] * 3, cell0=[0.0] * 3, K_sum=[L] * 3, Z=[1.0], a=pos,
        kinds=kinds, alphas=alphas, centres=centres, sinc_key="cubic_32",
        name=f"cubic_{L}", seed=seed)


def box_64(seed: int = 2, L: int = 64, n_perp: int = 320) -> dict:
    """Open-boundary (L,1,1) box, b = 2.0, one nucleus per cell with seeded charge Z in {1, 2}
    (same cell-relative position in every cell), m0 = 8 (4 s + px, py, pz, px; exponents
    log-uniform in [0.05, 20]), h = 0.05, x padded by ceil(rho_max/h) nodes per end and rounded
    up to a multiple of 128 nodes, n2 = n3 = n_perp on [-8, 8], R = 32."""
    rng = _rng(seed)
    b = 2.0
    h = 0.05
    n_c = int(round(b / h))
    off = rng.uniform(-b / 4.0, b / 4.0, size=3)
    pos = [[b / 2.0 + off[0], off[1], off[2]]]
    z_cell = rng.integers(1, 3, size=L).astype(float)
    kinds, alphas, centres = _basis_s_p(rng, 8, 4, 1, 0.05, 20.0, pos, extra_p_dir=[0])
    rho_max = math.sqrt(RHO / min(alphas))
    pad = int(math.ceil(rho_max / h))
    n1 = L * n_c + 2 * pad
    n1 = ((n1 + 127) // 128) * 128
    pad_left = (n1 - L * n_c) // 2
    x0 = -pad_left * h
    hp = 16.0 / n_perp
    return _system(
        L=[L, 1, 1], b=[b, 16.0, 16.0], periodic=[0, 0, 0], n=[n1, n_perp, n_perp],
        n_cell=[n_c, n_perp, n_perp], h=[h, hp, hp], x0=[x0, -8.0, -8.0],
        cell0=[0.0, -8.0, -8.0], K_sum=[1, 1, 1], Z=[1.0], a=pos, kinds=kinds, alphas=alphas,
        centres=centres, sinc_key="box_64", name=f"box_{L}", seed=seed,
        Z_cell=[[z] for z in z_cell])


def chain(L: int, seed: int = 6, periodic: bool = True, n_perp: int = 64) -> dict:
    """A (L,1,1) chain of identical cells, periodic (supercell of L cells, K_sum = L) or an open
    box, the same cell either way (the paper's box-vs-periodic comparisons): b = 2.0, h = 0.0625
    (n_cell = 32), one Z = 1 nucleus at a seeded offset, m0 = 4 s-type functions on it (exponents
    log-uniform in [0.05, 20]), open directions [-8, 8] with n_perp nodes, R = 32.  The open box
    pads x by ceil(rho_max / h) nodes per end and rounds up to a multiple of 128 nodes."""
    rng = _rng(seed)
    b = 2.0
    h = 0.0625
    n_c = int(round(b / h))
    off = rng.uniform(-b / 4.0, b / 4.0, size=3)
    pos = [[b / 2.0 + off[0], off[1], off[2]]]
    kinds, alphas, centres = _basis_s_p(rng, 4, 4, 0, 0.05, 20.0, pos)
    hp = 16.0 / n_perp
    if periodic:
        n1, x0 = L * n_c, 0.0
    else:
        pad = int(math.ceil(math.sqrt(RHO / min(alphas)) / h))
        n1 = ((L * n_c + 2 * pad + 127) // 128) * 128
        x0 = -((n1 - L * n_c) // 2) * h
    return _system(
        L=[L, 1, 1], b=[b, 16.0, 16.0], periodic=[1 if periodic else 0, 0, 0], n=[n1, n_perp, n_perp],
        n_cell=[n_c, n_perp, n_perp], h=[h, hp, hp], x0=[x0, -8.0, -8.0], cell0=[0.0, -8.0, -8.0],
        K_sum=[L if periodic else 1, 1, 1], Z=[1.0], a=pos, kinds=kinds, alphas=alphas, centres=centres,
        sinc_key="hetero_32", name=f"chain_{'periodic' if periodic else 'box'}_{L}", seed=seed)


def hetero(seed: int) -> dict:
    """One member of the heterogeneous batch: b = 2.0, one Z = 1 nucleus at a seeded offset,
    h drawn from {0.05, 0.0625, 0.08} (n_cell = 40, 32, 25), m0 from {4, 8, 16} (4 s; 4 s + px,
    py, pz, px; 4 s + 4 p-shells; exponents log-uniform in [0.05, 20]), R from {24, 32}; with
    probability 1/2 a periodic (L,1,1) tube with L log-uniform in [16, 512], else a periodic
    (L,L,1) slab with L uniform in [4, 32]; open directions span [-8, 8]; K_sum = L."""
    rng = _rng(seed)
    b = 2.0
    h = float(rng.choice([0.05, 0.0625, 0.08]))
    n_c = int(round(b / h))
    m0 = int(rng.choice([4, 8, 16]))
    sinc_key = "hetero_24" if rng.random() < 0.5 else "hetero_32"
    slab = rng.random() < 0.5
    if slab:
        L = int(rng.integers(4, 33))
        Ls, periodic = [L, L, 1], [1, 1, 0]
    else:
        L = int(round(math.exp(rng.uniform(math.log(16.0), math.log(512.0)))))
        Ls, periodic = [L, 1, 1], [1, 0, 0]
    off = rng.uniform(-b / 4.0, b / 4.0, size=3)
    pos = [[b / 2.0 + off[0], (b / 2.0 + off[1]) if slab else off[1], off[2]]]
    if m0 == 4:
        kinds, alphas, centres = _basis_s_p(rng, 4, 4, 0, 0.05, 20.0, pos)
    elif m0 == 8:
        kinds, alphas, centres = _basis_s_p(rng, 8, 4, 1, 0.05, 20.0, pos, extra_p_dir=[0])
    else:
        kinds, alphas, centres = _basis_s_p(rng, 16, 4, 4, 0.05, 20.0, pos)
    n_open = int(round(16.0 / h))
    n = [Ls[l] * n_c if periodic[l] else n_open for l in range(3)]
    n_cell = [n_c if periodic[l] else n_open for l in range(3)]
    bb = [b if periodic[l] else 16.0 for l in range(3)]
    x0 = [0.0 if periodic[l] else -8.0 for l in range(3)]
    return _system(
        L=Ls, b=bb, periodic=periodic, n=n, n_cell=n_cell, h=[h] * 3, x0=x0, cell0=x0,
        K_sum=[Ls[l] if periodic[l] else 1 for l in range(3)], Z=[1.0], a=pos, kinds=kinds,
        alphas=alphas, centres=centres, sinc_key=sinc_key,
        name=f"hetero_{'slab' if slab else 'tube'}_{L}", seed=seed)


def hetero_batch(count: int = 64, first_seed: int = 4000) -> list[dict]:
    """The heterogeneous batch: hetero(first_seed + s), s = 0 .. count-1."""
    return [hetero(first_seed + s) for s in range(count)]


def tube_256_batch(count: int, first_seed: int = 3000) -> list[dict]:
    """Seeded variants of tube_256 (seeds first_seed .. first_seed+count-1)."""
    return [tube_256(first_seed + s) for s in range(count)]


CONFIGS = {
    "periodic_8": periodic_8,
    "tube_256": tube_256,
    "cubic_32": cubic_32,
    "box_64": box_64,
}


def make_system(L, b, periodic, n_cell, h, x0, cell0, Z, a, kind, alpha, centre, R, u0, du,
                K_sum=None, n=None, Z_cell=None, name="custom", rho=RHO) -> dict:
    """Hand-made system (test cases): same dictionary layout as the named workloads.
    ``n`` defaults to L * n_cell per direction."""
    L = [int(v) for v in L]
    if n is None:
        n = [L[l] * int(n_cell[l]) for l in range(3)]
    if K_sum is None:
        K_sum = [L[l] if periodic[l] else 1 for l in range(3)]
    return {
        "name": name, "seed": None, "L": L, "b": [float(v) for v in b],
        "periodic": [int(v) for v in periodic], "n": [int(v) for v in n],
        "n_cell": [int(v) for v in n_cell], "h": [float(v) for v in h],
        "x0": [float(v) for v in x0], "cell0": [float(v) for v in cell0],
        "K_sum": [int(v) for v in K_sum], "Z": [float(v) for v in Z],
        "Z_cell": None if Z_cell is None else [[float(z) for z in row] for row in Z_cell],
        "a": [[float(c) for c in row] for row in a], "kind": [int(v) for v in kind],
        "alpha": [float(v) for v in alpha], "centre": [[float(c) for c in row] for row in centre],
        "R": int(R), "u0": float(u0), "du": float(du), "rho": float(rho),
    }
