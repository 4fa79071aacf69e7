"""Thin ctypes binding of liblhf.so (include/lhf.h).  Argument marshalling only: every step of
the path runs in the library's CUDA kernels.  Device buffers are passed as torch CUDA tensors
(or raw integer device pointers); the library never allocates them.  Loading fails loudly when
the library is missing: there is no fallback."""

from __future__ import annotations

import ctypes
import itertools
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "liblhf.so"

LHF_OK = 0
LHF_ERR_ARG = -1
LHF_ERR_CUDA = -2
LHF_ERR_NOT_SPD = -3
LHF_ERR_TIMEOUT = -4
LHF_ERR_UNSUPPORTED = -5
LHF_ERR_STATE = -6
LHF_ERR_NOMEM = -7
LHF_ERR_NOT_CONVERGED = -8

FP64 = 0
MIXED = 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class lhf_lattice_desc(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int * 3), ("b", ctypes.c_double * 3), ("periodic", ctypes.c_int * 3),
                ("K_sum", ctypes.c_int * 3), ("M0", ctypes.c_int), ("Z", _dp), ("a", _dp),
                ("Z_cell", _dp)]


class lhf_basis_desc(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_int), ("kind", _ip), ("alpha", _dp), ("centre", _dp),
                ("rho", ctypes.c_double)]


class lhf_grid_desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("n_cell", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("x0", ctypes.c_double * 3), ("cell0", ctypes.c_double * 3), ("R", ctypes.c_int),
                ("u0", ctypes.c_double), ("du", ctypes.c_double)]


class lhf_system_desc(ctypes.Structure):
    _fields_ = [("lattice", lhf_lattice_desc), ("basis", lhf_basis_desc), ("grid", lhf_grid_desc)]


class lhf_sizes(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_int), ("n_blocks", ctypes.c_int), ("n_kpoints", ctypes.c_int),
                ("n_basis", ctypes.c_int), ("rank", ctypes.c_int), ("window", ctypes.c_int * 3),
                ("n_potential", ctypes.c_int * 3), ("periodic", ctypes.c_int), ("desc_bytes", ctypes.c_int),
                ("overlap_rows", ctypes.c_int * 3)]


class LhfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"liblhf status {status}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return os.path.join(HERE, _LIB_NAME)


def load():
    """Load liblhf.so (built by paper_1408_3839_gb300.build).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run `python -m paper_1408_3839_gb300.build` "
                               "(the CUDA library is required; there is no CPU path)")
        lib = ctypes.CDLL(path)
        ctx = ctypes.c_void_p
        S = ctypes.POINTER(lhf_system_desc)
        st = ctypes.c_int
        sig = {
            "lhf_create": (st, [ctypes.POINTER(ctx), ctypes.c_int, ctypes.c_void_p]),
            "lhf_destroy": (None, [ctx]),
            "lhf_last_error": (ctypes.c_char_p, [ctx]),
            "lhf_set_stream": (st, [ctx, ctypes.c_void_p]),
            "lhf_sync": (st, [ctx]),
            "lhf_lattice_setup": (st, [ctx, ctypes.POINTER(lhf_lattice_desc)]),
            "lhf_basis_setup": (st, [ctx, ctypes.POINTER(lhf_basis_desc)]),
            "lhf_grid_setup": (st, [ctx, ctypes.POINTER(lhf_grid_desc)]),
            "lhf_query_sizes": (st, [ctx, ctypes.POINTER(lhf_sizes)]),
            "lhf_assemble_core_hamiltonian": (st, [ctx, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_circulant_fft": (st, [ctx] + [ctypes.c_void_p] * 4),
            "lhf_kspace_blocks": (st, [ctx, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_bloch_orbitals": (st, [ctx, _ip, ctypes.c_int, ctypes.c_void_p, _ip, _ip, ctypes.c_void_p]),
            "lhf_k_point_eigensolve": (st, [ctx] + [ctypes.c_void_p] * 4),
            "lhf_k_point_eigenvectors": (st, [ctx] + [ctypes.c_void_p] * 5),
            "lhf_dense_eigensolve": (st, [ctx, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
            "lhf_cell_energies": (st, [ctx, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), _ip, _ip,
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_bloch_spectra": (st, [ctx, ctypes.c_int, S, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_bloch_spectra_host": (st, [ctx, ctypes.c_int, S, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_basis_factors": (st, [ctx, ctypes.c_int, ctypes.c_void_p]),
            "lhf_potential_factors": (st, [ctx, ctypes.c_int, ctypes.c_void_p]),
            "lhf_gram_factors": (st, [ctx, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, _ip]),
            "lhf_set_profiling": (st, [ctx, ctypes.c_int]),
            "lhf_set_autotune": (st, [ctx, ctypes.c_int]),
            "lhf_launch_shapes": (st, [ctx, _ip, _ip]),
            "lhf_stage_times": (st, [ctx, _dp, _ip]),
            "lhf_kernel_times": (st, [ctx, _dp, _ip]),
            "lhf_kernel_name": (ctypes.c_char_p, [ctypes.c_int]),
            "lhf_eig_counters": (st, [ctx, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_ulonglong)]),
            "lhf_box_lowest_eigenvalues": (st, [ctx, S, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                                ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
            "lhf_set_rank_reduction": (st, [ctx, ctypes.c_double]),
            "lhf_rank_reduction_info": (st, [ctx, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
            "lhf_extrapolate_lattice_sum": (st, [ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_longlong,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
            "lhf_set_wait_limit": (st, [ctx, ctypes.c_longlong]),
            "lhf_inject_barrier_stall": (st, [ctx]),
            "lhf_set_workspace_limit": (st, [ctx, ctypes.c_size_t]),
            "lhf_k_point_eigensolve_noalloc": (st, [ctypes.POINTER(ctypes.c_int), ctypes.c_int] + [ctypes.c_void_p] * 5),
            "lhf_graph_create": (st, [ctx, ctypes.c_int, S, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
            "lhf_graph_launch": (st, [ctypes.c_void_p]),
            "lhf_graph_destroy": (None, [ctypes.c_void_p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(x) -> int | None:
    """Device pointer of a torch tensor (or an int pointer); None stays NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("device buffers must be contiguous")
        return x.data_ptr()
    raise TypeError(f"expected a device tensor or pointer, got {type(x)}")


class _Desc:
    """ctypes descriptors built from a workload dictionary; keeps the host arrays alive."""

    def __init__(self, cfg: dict):
        self.Z = np.ascontiguousarray(cfg["Z"], dtype=np.float64)
        self.a = np.ascontiguousarray(cfg["a"], dtype=np.float64).reshape(-1)
        self.Z_cell = (None if cfg.get("Z_cell") is None
                       else np.ascontiguousarray(cfg["Z_cell"], dtype=np.float64).reshape(-1))
        self.kind = np.ascontiguousarray(cfg["kind"], dtype=np.int32)
        self.alpha = np.ascontiguousarray(cfg["alpha"], dtype=np.float64)
        self.centre = np.ascontiguousarray(cfg["centre"], dtype=np.float64).reshape(-1)
        lat = lhf_lattice_desc()
        lat.L[:] = cfg["L"]
        lat.b[:] = cfg["b"]
        lat.periodic[:] = cfg["periodic"]
        lat.K_sum[:] = cfg["K_sum"]
        lat.M0 = len(cfg["Z"])
        lat.Z = self.Z.ctypes.data_as(_dp)
        lat.a = self.a.ctypes.data_as(_dp)
        lat.Z_cell = self.Z_cell.ctypes.data_as(_dp) if self.Z_cell is not None else ctypes.cast(None, _dp)
        bas = lhf_basis_desc()
        bas.m0 = len(cfg["alpha"])
        bas.kind = self.kind.ctypes.data_as(_ip)
        bas.alpha = self.alpha.ctypes.data_as(_dp)
        bas.centre = self.centre.ctypes.data_as(_dp)
        bas.rho = float(cfg["rho"])
        grd = lhf_grid_desc()
        grd.n[:] = cfg["n"]
        grd.n_cell[:] = cfg["n_cell"]
        grd.h[:] = cfg["h"]
        grd.x0[:] = cfg["x0"]
        grd.cell0[:] = cfg["cell0"]
        grd.R = int(cfg["R"])
        grd.u0 = float(cfg["u0"])
        grd.du = float(cfg["du"])
        self.lattice, self.basis, self.grid = lat, bas, grd
        self.system = lhf_system_desc(lat, bas, grd)


def _np_dtype(ct) -> np.dtype:
    """numpy structured dtype with the exact layout of a ctypes structure (pointers as uint64)."""
    names, formats, offsets = [], [], []
    for fname, ftype in ct._fields_:
        if hasattr(ftype, "_fields_"):
            fmt = _np_dtype(ftype)
        elif hasattr(ftype, "_length_"):
            fmt = (np.float64 if ftype._type_ is ctypes.c_double else np.int32, (ftype._length_,))
        elif ftype is ctypes.c_double:
            fmt = np.float64
        elif ftype is ctypes.c_int:
            fmt = np.int32
        else:  # pointers
            fmt = np.uint64
        names.append(fname)
        formats.append(fmt)
        offsets.append(getattr(ct, fname).offset)
    return np.dtype({"names": names, "formats": formats, "offsets": offsets, "itemsize": ctypes.sizeof(ct)})


_SYSTEM_DTYPE = None


class _Batch:
    """An array of lhf_system_desc for many workload dictionaries, filled column by column in one
    numpy structured array (its per-system host arrays packed into two buffers it keeps alive)."""

    def __init__(self, cfgs):
        global _SYSTEM_DTYPE
        if _SYSTEM_DTYPE is None:
            _SYSTEM_DTYPE = _np_dtype(lhf_system_desc)
        n = len(cfgs)
        arr = np.zeros(n, dtype=_SYSTEM_DTYPE)
        lat, bas, grd = arr["lattice"], arr["basis"], arr["grid"]
        for fld in ("L", "b", "periodic", "K_sum"):
            lat[fld] = [c[fld] for c in cfgs]
        lat["M0"] = [len(c["Z"]) for c in cfgs]
        m0 = np.array([len(c["alpha"]) for c in cfgs], dtype=np.int64)
        bas["m0"] = m0
        bas["rho"] = [c["rho"] for c in cfgs]
        for fld in ("n", "n_cell", "h", "x0", "cell0", "R", "u0", "du"):
            grd[fld] = [c[fld] for c in cfgs]
        # doubles per system: Z, a (flattened), alpha, centre (flattened), Z_cell (flattened, optional),
        # flattened at C speed (itertools) straight into the buffers
        flat = itertools.chain.from_iterable
        lens = np.empty((n, 5), dtype=np.int64)
        lens[:, 0] = lat["M0"]
        lens[:, 1] = 3 * lens[:, 0]
        lens[:, 2] = m0
        lens[:, 3] = 3 * m0
        lens[:, 4] = [0 if c.get("Z_cell") is None else sum(len(r) for r in c["Z_cell"]) for c in cfgs]

        def values(c):
            zc = c.get("Z_cell")
            return flat((c["Z"], flat(c["a"]), c["alpha"], flat(c["centre"]), () if zc is None else flat(zc)))

        self.dbuf = np.fromiter(flat(values(c) for c in cfgs), dtype=np.float64, count=int(lens.sum()))
        self.ibuf = np.fromiter(flat(c["kind"] for c in cfgs), dtype=np.int32, count=int(m0.sum()))
        start = np.concatenate([[0], np.cumsum(lens.ravel())[:-1]]).reshape(n, 5)
        addr = (start * 8 + self.dbuf.ctypes.data).astype(np.uint64)
        lat["Z"] = addr[:, 0]
        lat["a"] = addr[:, 1]
        bas["alpha"] = addr[:, 2]
        bas["centre"] = addr[:, 3]
        lat["Z_cell"] = np.where(lens[:, 4] > 0, addr[:, 4], 0).astype(np.uint64)
        bas["kind"] = (np.concatenate([[0], np.cumsum(m0)[:-1]]) * 4 + self.ibuf.ctypes.data).astype(np.uint64)
        self.arr = arr
        self.count = n

    def ptr(self):
        return self.arr.ctypes.data_as(ctypes.POINTER(lhf_system_desc))


class Context:
    """One lhf_ctx on one device and stream (torch.cuda stream or raw cudaStream_t)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        self._h = ctypes.c_void_p()
        raw = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = self.lib.lhf_create(ctypes.byref(self._h), int(device), raw)
        if st != LHF_OK:
            raise LhfError(st, "lhf_create failed")
        self._keep = []

    def _check(self, st: int):
        if st != LHF_OK:
            msg = self.lib.lhf_last_error(self._h)
            raise LhfError(st, msg.decode() if msg else "")
        return st

    def close(self):
        if self._h:
            self.lib.lhf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- setup -----------------------------------------------------------------------------
    def set_stream(self, stream):
        raw = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self._check(self.lib.lhf_set_stream(self._h, raw))

    def lattice_setup(self, cfg: dict):
        d = _Desc(cfg)
        self._check(self.lib.lhf_lattice_setup(self._h, ctypes.byref(d.lattice)))

    def basis_setup(self, cfg: dict):
        d = _Desc(cfg)
        self._check(self.lib.lhf_basis_setup(self._h, ctypes.byref(d.basis)))

    def grid_setup(self, cfg: dict):
        d = _Desc(cfg)
        self._check(self.lib.lhf_grid_setup(self._h, ctypes.byref(d.grid)))

    def setup(self, cfg: dict):
        """lattice_setup + basis_setup + grid_setup of one workload dictionary."""
        self.lattice_setup(cfg)
        self.basis_setup(cfg)
        self.grid_setup(cfg)

    def query_sizes(self) -> dict:
        out = lhf_sizes()
        self._check(self.lib.lhf_query_sizes(self._h, ctypes.byref(out)))
        return {"m0": out.m0, "n_blocks": out.n_blocks, "n_kpoints": out.n_kpoints,
                "n_basis": out.n_basis, "rank": out.rank, "window": list(out.window),
                "n_potential": list(out.n_potential), "periodic": out.periodic,
                "desc_bytes": out.desc_bytes, "overlap_rows": list(out.overlap_rows)}

    def sync(self):
        self._check(self.lib.lhf_sync(self._h))

    # -- path --------------------------------------------------------------------------------
    def assemble_core_hamiltonian(self, H, S, precision: int = FP64):
        self._check(self.lib.lhf_assemble_core_hamiltonian(self._h, precision, _ptr(H), _ptr(S)))

    def bloch_orbitals(self, kappa, coef, lo, cnt, out):
        """lhf_bloch_orbitals: coef device complex [norb][m0][2]; out device [norb][cnt0][cnt1][cnt2][2]."""
        k = (ctypes.c_int * 3)(*[int(v) for v in kappa])
        a = (ctypes.c_int * 3)(*[int(v) for v in lo])
        b = (ctypes.c_int * 3)(*[int(v) for v in cnt])
        norb = int(coef.shape[0]) if hasattr(coef, "shape") else 1
        self._check(self.lib.lhf_bloch_orbitals(self._h, k, norb, _ptr(coef), a, b, _ptr(out)))

    def kspace_blocks(self, Hbar, Sbar, precision: int = FP64):
        self._check(self.lib.lhf_kspace_blocks(self._h, int(precision), _ptr(Hbar), _ptr(Sbar)))

    def circulant_fft(self, H, S, Hbar, Sbar):
        self._check(self.lib.lhf_circulant_fft(self._h, _ptr(H), _ptr(S), _ptr(Hbar), _ptr(Sbar)))

    def k_point_eigensolve(self, Hbar, Sbar, eig, k_status=None):
        self._check(self.lib.lhf_k_point_eigensolve(self._h, _ptr(Hbar), _ptr(Sbar), _ptr(eig), _ptr(k_status)))

    def k_point_eigenvectors(self, Hbar, Sbar, eig, vecs, k_status=None):
        self._check(self.lib.lhf_k_point_eigenvectors(self._h, _ptr(Hbar), _ptr(Sbar), _ptr(eig), _ptr(vecs),
                                                      _ptr(k_status)))

    def box_lowest_eigenvalues(self, cfg, n_ev: int, eig, tol: float = 1e-7, max_iter: int = 300,
                               check: bool = True):
        """lhf_box_lowest_eigenvalues: the n_ev lowest eigenvalues of an open (L,1,1) box by
        preconditioned LOBPCG on its banded matrices; returns (status, iterations, residual)."""
        batch, arr = self._systems([cfg])
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        st = self.lib.lhf_box_lowest_eigenvalues(self._h, arr, int(n_ev), float(tol), int(max_iter), _ptr(eig),
                                                 ctypes.byref(it), ctypes.byref(res))
        if check:
            self._check(st)
        return st, it.value, res.value

    def dense_eigensolve(self, H, S, N: int, eig):
        self._check(self.lib.lhf_dense_eigensolve(self._h, _ptr(H), _ptr(S), int(N), _ptr(eig)))

    def cell_energies(self, eig, off, cnt, n_low, cells, energy, level=None):
        """lhf_cell_energies: eig, energy, level device float64; off, cnt, n_low, cells host sequences."""
        n = len(cnt)
        o = (ctypes.c_longlong * n)(*[int(v) for v in off])
        c = (ctypes.c_int * n)(*[int(v) for v in cnt])
        k = (ctypes.c_int * n)(*[int(v) for v in n_low])
        w = (ctypes.c_double * n)(*[float(v) for v in cells])
        self._check(self.lib.lhf_cell_energies(self._h, n, _ptr(eig), o, c, k, w, _ptr(energy), _ptr(level)))

    @staticmethod
    def prepare(cfgs) -> "_Batch":
        """The lhf_system_desc array of a list of workload dictionaries, marshalled once: every
        batched call below accepts it in place of the list (the array and the host arrays it
        points to live as long as the returned object)."""
        return _Batch(cfgs)

    @staticmethod
    def _systems(cfgs):
        """(keep-alive object, pointer to the lhf_system_desc array) for a list of workloads or a
        prepared batch."""
        batch = cfgs if isinstance(cfgs, _Batch) else _Batch(cfgs)
        return batch, batch.ptr()

    def bloch_spectra(self, cfgs, eig, k_status=None, precision: int = FP64):
        batch, arr = self._systems(cfgs)
        self._check(self.lib.lhf_bloch_spectra(self._h, batch.count, arr, precision, _ptr(eig), _ptr(k_status)))

    def bloch_spectra_host(self, cfgs, eig_host: np.ndarray, k_status_host: np.ndarray | None = None,
                           precision: int = FP64):
        assert eig_host.dtype == np.float64 and eig_host.flags["C_CONTIGUOUS"]
        batch, arr = self._systems(cfgs)
        kp = None
        if k_status_host is not None:
            assert k_status_host.dtype == np.int32 and k_status_host.flags["C_CONTIGUOUS"]
            kp = k_status_host.ctypes.data
        self._check(self.lib.lhf_bloch_spectra_host(self._h, batch.count, arr, precision,
                                                    eig_host.ctypes.data, kp))

    def graph_create(self, cfgs, eig, k_status=None, precision: int = FP64) -> "Graph":
        """lhf_graph_create: the batched path captured once into a CUDA graph."""
        batch, arr = self._systems(cfgs)
        h = ctypes.c_void_p()
        self._check(self.lib.lhf_graph_create(self._h, batch.count, arr, precision, _ptr(eig), _ptr(k_status),
                                              ctypes.byref(h)))
        return Graph(self, h, (eig, k_status))

    # -- live stage timing -------------------------------------------------------------------
    STAGES = ("basis", "potential", "gram", "ranksum", "dft", "eig", "unused", "upload", "gram_tc")

    def set_autotune(self, enable: bool):
        self._check(self.lib.lhf_set_autotune(self._h, 1 if enable else 0))

    def launch_shapes(self) -> dict:
        """Launch shapes of the last k-point solve: k_eig warps per CTA, tridiagonal threads per CTA."""
        a, b = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.lhf_launch_shapes(self._h, ctypes.byref(a), ctypes.byref(b)))
        return {"eig_warps": a.value, "tri_threads": b.value}

    def set_rank_reduction(self, eps: float):
        """Rank reduction of the direction-0 potential of (L,1,1) lattices (FP64 route); 0: off."""
        self._check(self.lib.lhf_set_rank_reduction(self._h, float(eps)))

    def rank_reduction_info(self) -> dict:
        """R_tot, the reduced rank r1, the largest dropped and the largest singular value for the
        current setup system."""
        ri, ro = ctypes.c_int(0), ctypes.c_int(0)
        dr, lg = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._check(self.lib.lhf_rank_reduction_info(self._h, ctypes.byref(ri), ctypes.byref(ro), ctypes.byref(dr),
                                                     ctypes.byref(lg)))
        return {"rank_in": ri.value, "rank_out": ro.value, "dropped": dr.value, "largest": lg.value}

    def extrapolate_lattice_sum(self, K, eig, eig_limit, slope=None):
        """lhf_extrapolate_lattice_sum: eig device [len(K)][n] -> eig_limit (and slope) device [n]."""
        Karr = (ctypes.c_double * len(K))(*[float(v) for v in K])
        n = eig_limit.numel() if hasattr(eig_limit, "numel") else int(eig_limit)
        self._check(self.lib.lhf_extrapolate_lattice_sum(self._h, len(K), Karr, int(n), _ptr(eig), _ptr(eig_limit),
                                                         _ptr(slope)))

    def set_wait_limit(self, cycles: int):
        """Bound (SM clock cycles) of the dense eigensolver's grid-barrier waits; <= 0: default."""
        self._check(self.lib.lhf_set_wait_limit(self._h, int(cycles)))

    def inject_barrier_stall(self):
        """Make the next dense eigensolve's barrier waits run out (failure-detection test)."""
        self._check(self.lib.lhf_inject_barrier_stall(self._h))

    def set_workspace_limit(self, nbytes: int):
        """Cap on the context's device workspace in bytes (0: none)."""
        self._check(self.lib.lhf_set_workspace_limit(self._h, int(nbytes)))

    def set_profiling(self, enable: bool):
        self._check(self.lib.lhf_set_profiling(self._h, 1 if enable else 0))

    def stage_times(self) -> dict:
        """{stage: (total ms, launches)} for launches recorded since the previous call."""
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        self._check(self.lib.lhf_stage_times(self._h, ms, cnt))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(self.STAGES)}

    NUM_KERNELS = 18

    def kernel_times(self) -> dict:
        """{kernel name: (total ms, launches)} for kernel launches recorded since the previous call."""
        n = self.NUM_KERNELS
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int * n)()
        self._check(self.lib.lhf_kernel_times(self._h, ms, cnt))
        return {self.lib.lhf_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(n)}

    def eig_counters(self) -> tuple[int, int]:
        """(FP64 polynomial passes of the tridiagonal stage, matrices solved) since the previous call."""
        a, b = ctypes.c_ulonglong(), ctypes.c_ulonglong()
        self._check(self.lib.lhf_eig_counters(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    # -- stage outputs -----------------------------------------------------------------------
    def basis_factors(self, l: int, G):
        self._check(self.lib.lhf_basis_factors(self._h, int(l), _ptr(G)))

    def potential_factors(self, l: int, V):
        self._check(self.lib.lhf_potential_factors(self._h, int(l), _ptr(V)))

    def gram_factors(self, l: int, C, precision: int = FP64) -> int:
        jlo = ctypes.c_int(0)
        self._check(self.lib.lhf_gram_factors(self._h, precision, int(l), _ptr(C), ctypes.byref(jlo)))
        return jlo.value


class Graph:
    """A captured batched path (lhf_graph): launch() replays it on the context stream."""

    def __init__(self, ctx: Context, handle, keep):
        self._ctx = ctx
        self._h = handle
        self._keep = keep  # the output buffers the graph writes

    def launch(self):
        st = self._ctx.lib.lhf_graph_launch(self._h)
        if st != LHF_OK and not self._ctx._h:
            raise LhfError(st, "the graph's context was destroyed")
        self._ctx._check(st)

    def close(self):
        if self._h is not None and self._h.value:
            self._ctx.lib.lhf_graph_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def k_point_eigensolve_noalloc(L, m0: int, Hbar, Sbar, eig, k_status=None, stream=None):
    """lhf_k_point_eigensolve_noalloc: the k-point eigensolve without a context or any device
    allocation (its scratch is a static device array inside the library).  stream: a torch
    stream or a raw cudaStream_t; None takes torch's current stream, the one on which the
    caller's tensors were written."""
    lib = load()
    Larr = (ctypes.c_int * 3)(*[int(v) for v in L])
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = lib.lhf_k_point_eigensolve_noalloc(Larr, int(m0), _ptr(Hbar), _ptr(Sbar), _ptr(eig), _ptr(k_status), raw)
    if st != LHF_OK:
        raise LhfError(st, "lhf_k_point_eigensolve_noalloc failed")
