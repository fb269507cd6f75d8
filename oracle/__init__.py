"""CPU oracle for the sparsified-AMG path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check and the benchmark's CPU-baseline leg may
import this package.  The product library never does, and shares no code with
it.  The arithmetic lives in ``amg_oracle.c`` (plain FP64, single-threaded,
compiled with ``-ffp-contract=off``); this module builds it with gcc, loads it
with ctypes and converts between numpy arrays and the C structs.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "amg_oracle.c")
_HDR = os.path.join(_HERE, "amg_oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def _compile(path: str, extra) -> None:
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", "-Wall", "-Wno-unknown-pragmas", *extra, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)


def build(force: bool = False, omp: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off): the
    sequential parity build, or with omp=True the all-core timing build of
    the same source (-fopenmp: the solve phase's row loops run in parallel)."""
    path = _OMP_PATH if omp else _LIB_PATH
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(path) or os.path.getmtime(path) < newest:
        _compile(path, ["-fopenmp"] if omp else [])
    return path


class _CSR(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int32),
                ("rowptr", C.POINTER(C.c_int32)), ("col", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


class _Info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("resets", C.c_int32),
                ("replacements", C.c_int32), ("final_relres", C.c_double),
                ("conv_factor", C.c_double)]


class _Window(C.Structure):
    _fields_ = [("steps", C.c_int32), ("action", C.c_int32), ("rstart", C.c_double),
                ("rend", C.c_double), ("factor", C.c_double)]


def _load(omp: bool = False):
    global _lib, _lib_omp
    with _lock:
        if (_lib_omp if omp else _lib) is not None:
            return _lib_omp if omp else _lib
        lib = C.CDLL(build(omp=omp))
        P = C.POINTER
        vp = C.c_void_p
        lib.orc_strength.argtypes = [P(_CSR), C.c_double, vp]
        lib.orc_pmis.argtypes = [P(_CSR), vp, C.c_uint64, C.c_int32, vp]
        lib.orc_direct_interp.argtypes = [P(_CSR), vp, vp]
        lib.orc_direct_interp.restype = P(_CSR)
        lib.orc_transpose.argtypes = [P(_CSR)]
        lib.orc_transpose.restype = P(_CSR)
        lib.orc_spgemm.argtypes = [P(_CSR), P(_CSR)]
        lib.orc_spgemm.restype = P(_CSR)
        lib.orc_minimal_pattern.argtypes = [P(_CSR), P(_CSR), vp, vp]
        lib.orc_sparsify_diag.argtypes = [P(_CSR), vp, C.c_double, vp]
        lib.orc_sparsify_diag.restype = P(_CSR)
        lib.orc_sparsify_full.argtypes = [P(_CSR), vp, C.c_double, C.c_double, vp]
        lib.orc_sparsify_full.restype = P(_CSR)
        lib.orc_l1_diag.argtypes = [P(_CSR), vp]
        lib.orc_cholesky.argtypes = [C.c_int32, vp]
        lib.orc_chol_solve.argtypes = [C.c_int32, vp, vp, vp]
        lib.orc_lu.argtypes = [C.c_int32, vp, vp]
        lib.orc_lu_solve.argtypes = [C.c_int32, vp, vp, vp, vp]
        lib.orc_spmv.argtypes = [P(_CSR), vp, vp]
        lib.orc_uniform_weight.argtypes = [C.c_uint64, C.c_int32, C.c_int64]
        lib.orc_uniform_weight.restype = C.c_double
        lib.orc_gamma_schedule.argtypes = [vp, C.c_int32, C.c_int32, C.c_double, vp]
        lib.orc_setup.argtypes = [P(_CSR), C.c_double, C.c_int32, C.c_int32, C.c_uint64,
                                  P(C.c_int32)]
        lib.orc_setup.restype = vp
        lib.orc_setup_nongalerkin.argtypes = [P(_CSR), C.c_double, C.c_int32, C.c_int32, C.c_uint64,
                                              vp, C.c_int32, C.c_int32, P(C.c_int32)]
        lib.orc_setup_nongalerkin.restype = vp
        lib.orc_sparsify.argtypes = [vp, vp, C.c_int32]
        lib.orc_reintroduce.argtypes = [vp, C.c_int32, C.c_double, vp]
        lib.orc_sparsify_method.argtypes = [vp, vp, C.c_int32, C.c_int32]
        lib.orc_sparsify_opts.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int32]
        lib.orc_gmres.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32, P(_Info)]
        lib.orc_gmres_plain.argtypes = [P(_CSR), vp, vp, C.c_double, C.c_int32, C.c_int32,
                                        P(_Info)]
        lib.orc_adaptive_gmres.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32,
                                           C.c_int32, C.c_int32, C.c_double, C.c_double,
                                           P(_Info)]
        lib.orc_vcycle.argtypes = [vp, vp, vp]
        lib.orc_pcg.argtypes = [vp, vp, vp, C.c_double, C.c_int32, P(_Info)]
        lib.orc_pcg_ex.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32, C.c_double,
                                   P(_Info)]
        lib.orc_adaptive_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32,
                                           C.c_int32, C.c_double, C.c_double, P(_Info)]
        lib.orc_adaptive_solve_ex.argtypes = [vp, vp, vp, C.c_double, C.c_int32, C.c_int32,
                                              C.c_int32, C.c_double, C.c_double, C.c_double,
                                              P(_Window), C.c_int32, P(C.c_int32), P(_Info)]
        lib.orc_free.argtypes = [vp]
        lib.orc_csr_free.argtypes = [P(_CSR)]
        lib.orc_num_levels.argtypes = [vp]
        lib.orc_level_matrix.argtypes = [vp, C.c_int32, C.c_int32]
        lib.orc_level_matrix.restype = P(_CSR)
        lib.orc_level_array.argtypes = [vp, C.c_int32, C.c_int32]
        lib.orc_level_array.restype = vp
        lib.orc_level_gamma.argtypes = [vp, C.c_int32]
        lib.orc_level_gamma.restype = C.c_double
        if omp:
            _lib_omp = lib
        else:
            _lib = lib
        return lib


# --------------------------------------------------------------------------
# numpy <-> C conversion
# --------------------------------------------------------------------------
@dataclass
class Mat:
    """Host CSR copy returned by the oracle (rectangular allowed)."""

    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.nrows, self.ncols))

    def todense(self):
        return self.to_scipy().toarray()


def _as_c(rowptr, col, val, nrows, ncols):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    s = _CSR(nrows, ncols, int(rowptr[-1]),
             rowptr.ctypes.data_as(C.POINTER(C.c_int32)),
             col.ctypes.data_as(C.POINTER(C.c_int32)),
             val.ctypes.data_as(C.POINTER(C.c_double)))
    s._keep = (rowptr, col, val)  # keep the buffers alive with the struct
    return s


def to_c(m) -> _CSR:
    """Accepts amg_inputs.CSR, Mat or scipy.sparse CSR."""
    if hasattr(m, "indptr"):
        return _as_c(m.indptr, m.indices, m.data, m.shape[0], m.shape[1])
    nrows = getattr(m, "nrows", None) or m.n
    ncols = getattr(m, "ncols", None) or m.n
    return _as_c(m.rowptr, m.col, m.val, nrows, ncols)


def _from_c(ptr, own: bool) -> Mat:
    if not ptr:
        raise MemoryError("oracle returned no matrix")
    s = ptr.contents
    nnz = s.nnz
    rowptr = np.ctypeslib.as_array(s.rowptr, shape=(s.nrows + 1,)).copy()
    col = np.ctypeslib.as_array(s.col, shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(s.val, shape=(max(nnz, 1),))[:nnz].copy()
    out = Mat(s.nrows, s.ncols, rowptr, col, val)
    if own:
        _load().orc_csr_free(ptr)
    return out


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------
def strength(A, theta: float = 0.25) -> np.ndarray:
    c = to_c(A)
    out = np.zeros(c.nnz, dtype=np.uint8)
    _load().orc_strength(C.byref(c), theta, _ptr(out))
    return out


def pmis(A, strong: np.ndarray, seed: int = 0, level: int = 0) -> np.ndarray:
    c = to_c(A)
    strong = np.ascontiguousarray(strong, dtype=np.uint8)
    cf = np.zeros(c.nrows, dtype=np.int8)
    st = _load().orc_pmis(C.byref(c), _ptr(strong), seed, level, _ptr(cf))
    if st:
        raise RuntimeError(f"orc_pmis status {st}")
    return cf


def uniform_weight(seed: int, level: int, i: int) -> float:
    return _load().orc_uniform_weight(seed, level, i)


def direct_interp(A, strong, cf) -> Mat:
    c = to_c(A)
    strong = np.ascontiguousarray(strong, dtype=np.uint8)
    cf = np.ascontiguousarray(cf, dtype=np.int8)
    return _from_c(_load().orc_direct_interp(C.byref(c), _ptr(strong), _ptr(cf)), True)


def transpose(M) -> Mat:
    return _from_c(_load().orc_transpose(C.byref(to_c(M))), True)


def spgemm(A, B) -> Mat:
    return _from_c(_load().orc_spgemm(C.byref(to_c(A)), C.byref(to_c(B))), True)


def minimal_pattern(Ac, AP, cf) -> np.ndarray:
    ca, cp = to_c(Ac), to_c(AP)
    cf = np.ascontiguousarray(cf, dtype=np.int8)
    out = np.zeros(ca.nnz, dtype=np.uint8)
    st = _load().orc_minimal_pattern(C.byref(ca), C.byref(cp), _ptr(cf), _ptr(out))
    if st:
        raise RuntimeError(f"orc_minimal_pattern status {st}")
    return out


def sparsify_diag(Ac, inM, gamma: float):
    """Returns (Ahat, keep mask over Ac's entries)."""
    ca = to_c(Ac)
    inM = np.ascontiguousarray(inM, dtype=np.uint8)
    keep = np.zeros(ca.nnz, dtype=np.uint8)
    H = _from_c(_load().orc_sparsify_diag(C.byref(ca), _ptr(inM), gamma, _ptr(keep)), True)
    return H, keep


def sparsify_full(Ac, inM, gamma: float, theta: float = 0.25):
    """Algorithm 3 with full lumping to strong neighbours; returns (Ahat, keep)."""
    ca = to_c(Ac)
    inM = np.ascontiguousarray(inM, dtype=np.uint8)
    keep = np.zeros(ca.nnz, dtype=np.uint8)
    H = _from_c(_load().orc_sparsify_full(C.byref(ca), _ptr(inM), gamma, theta, _ptr(keep)), True)
    return H, keep


def l1_diag(A) -> np.ndarray:
    c = to_c(A)
    d = np.zeros(c.nrows, dtype=np.float64)
    _load().orc_l1_diag(C.byref(c), _ptr(d))
    return d


def spmv(A, x) -> np.ndarray:
    c = to_c(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(c.nrows, dtype=np.float64)
    _load().orc_spmv(C.byref(c), _ptr(x), _ptr(y))
    return y


def cholesky(a: np.ndarray) -> np.ndarray:
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    st = _load().orc_cholesky(a.shape[0], _ptr(a))
    if st:
        raise np.linalg.LinAlgError("not positive definite")
    return a


def chol_solve(L: np.ndarray, b: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    _load().orc_chol_solve(L.shape[0], _ptr(L), _ptr(b), _ptr(x))
    return x


def lu(a: np.ndarray):
    """Dense LU with partial pivoting; returns (LU in place, pivot rows)."""
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    piv = np.zeros(a.shape[0], dtype=np.int32)
    st = _load().orc_lu(a.shape[0], _ptr(a), _ptr(piv))
    if st:
        raise np.linalg.LinAlgError("singular")
    return a, piv


def lu_solve(LU: np.ndarray, piv: np.ndarray, b: np.ndarray) -> np.ndarray:
    LU = np.ascontiguousarray(LU, dtype=np.float64)
    piv = np.ascontiguousarray(piv, dtype=np.int32)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    _load().orc_lu_solve(LU.shape[0], _ptr(LU), _ptr(piv), _ptr(b), _ptr(x))
    return x


def gmres_plain(A, b, tol: float = 1e-8, max_it: int = 500, restart: int = 30):
    """Unpreconditioned restarted GMRES from x0 = 0 (the oracle's GMRES core)."""
    c = to_c(A)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b)
    info = _Info()
    _load().orc_gmres_plain(C.byref(c), _ptr(b), _ptr(x), tol, max_it, restart, C.byref(info))
    return x, _info(info)


def gamma_schedule(gamma, s: int, gamma_min: float = 0.01):
    """One Algorithm-5 drop-tolerance update; returns (new gammas, changed flags)."""
    g = np.array(gamma, dtype=np.float64)
    ch = np.zeros(len(g), dtype=np.int32)
    _load().orc_gamma_schedule(_ptr(g), len(g), s, gamma_min, _ptr(ch))
    return g, ch.astype(bool)


# --------------------------------------------------------------------------
# hierarchy
# --------------------------------------------------------------------------
# names of the ORC_WIN_* codes of an Algorithm 5 check window
WIN_ACTIONS = ["continue", "restart_here", "restart_back", "converged", "nothing_left",
               "breakdown_stop", "breakdown_back", "diverged"]

# status codes of the oracle's solvers
OK, INVALID, OOM, NOT_CONVERGED, DIVERGED, BREAKDOWN = 0, 1, 2, 4, 5, 6


@dataclass
class SolveInfo:
    iterations: int
    status: int
    resets: int
    replacements: int
    final_relres: float
    conv_factor: float


def _info(i: _Info) -> SolveInfo:
    return SolveInfo(i.iterations, i.status, i.resets, i.replacements, i.final_relres,
                     i.conv_factor)


class Hierarchy:
    """Oracle AMG hierarchy (Algorithm 1 Galerkin setup + Algorithm 4 sparsify)."""

    def __init__(self, A, theta: float = 0.25, max_size: int = 100, max_levels: int = 25,
                 seed: int = 0, nongalerkin=None, lump: int = 0, omp: bool = False):
        """nongalerkin: per-level drop tolerances for Algorithm 1's in-loop
        (non-Galerkin) sparsify; None builds the Galerkin hierarchy.  omp:
        use the all-core timing build (the solve phase's row loops on every
        host thread; results differ from the sequential build only by the
        summation order of dot products)."""
        lib = _load(omp)
        self._lib = lib
        c = to_c(A)
        st = C.c_int32(0)
        if nongalerkin is None:
            self._h = lib.orc_setup(C.byref(c), theta, max_size, max_levels, seed, C.byref(st))
        else:
            g = np.ascontiguousarray(nongalerkin, dtype=np.float64)
            self._h = lib.orc_setup_nongalerkin(C.byref(c), theta, max_size, max_levels, seed, _ptr(g),
                                                len(g), lump, C.byref(st))
        if not self._h:
            raise RuntimeError(f"orc_setup failed with status {st.value}")
        self.n = c.nrows

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return self._lib.orc_num_levels(self._h)

    def matrix(self, level: int, which: str) -> Mat | None:
        code = {"A": 0, "Ahat": 1, "P": 2, "R": 3, "AP": 4}[which]
        p = self._lib.orc_level_matrix(self._h, level, code)
        return _from_c(p, False) if p else None

    def _array(self, level, code, dtype, count):
        p = self._lib.orc_level_array(self._h, level, code)
        if not p:
            return None
        return np.ctypeslib.as_array(C.cast(p, C.POINTER(np.ctypeslib.as_ctypes_type(dtype))),
                                     shape=(count,)).copy()

    def strong(self, level):
        return self._array(level, 0, np.uint8, self.matrix(level, "A").nnz)

    def cf(self, level):
        return self._array(level, 1, np.int8, self.matrix(level, "A").nrows)

    def inM(self, level):
        return self._array(level, 2, np.uint8, self.matrix(level, "A").nnz)

    def keep(self, level):
        return self._array(level, 3, np.uint8, self.matrix(level, "A").nnz)

    def l1(self, level):
        return self._array(level, 4, np.float64, self.matrix(level, "A").nrows)

    def gamma(self, level) -> float:
        return self._lib.orc_level_gamma(self._h, level)

    def sparsify(self, gamma, method: int = 0, lump: int = 0):
        """method 0: Sparse Galerkin; 1: Hybrid Galerkin.  lump 0: diagonal
        lumping (Algorithm 3b); 1: full lumping to strong neighbours (Algorithm 3)."""
        g = np.ascontiguousarray(gamma, dtype=np.float64)
        st = self._lib.orc_sparsify_opts(self._h, _ptr(g), len(g), method, lump)
        if st:
            raise RuntimeError(f"orc_sparsify status {st}")

    def reintroduce(self, s: int = 1, gamma_min: float = 0.01):
        ch = np.zeros(64, dtype=np.int32)
        cnt = self._lib.orc_reintroduce(self._h, s, gamma_min, _ptr(ch))
        if cnt < 0:
            raise RuntimeError(f"orc_reintroduce status {-cnt}")
        return cnt, ch[: self.num_levels].astype(bool)

    def vcycle(self, b) -> np.ndarray:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        self._lib.orc_vcycle(self._h, _ptr(b), _ptr(x))
        return x

    def pcg(self, b, tol: float = 1e-8, max_it: int = 500, k: int | None = None,
            div_factor: float | None = None):
        """PCG; k / div_factor set the divergence test (windows of k steps,
        growth factor div_factor, 0 = off; default 3 and 1e3)."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        info = _Info()
        if k is None and div_factor is None:
            self._lib.orc_pcg(self._h, _ptr(b), _ptr(x), tol, max_it, C.byref(info))
        else:
            self._lib.orc_pcg_ex(self._h, _ptr(b), _ptr(x), tol, max_it, 3 if k is None else k,
                                 1e3 if div_factor is None else div_factor, C.byref(info))
        return x, _info(info)

    def adaptive_solve(self, b, tol: float = 1e-8, max_it: int = 500, k: int = 3, s: int = 1,
                       gamma_min: float = 0.01, rho_max: float = 0.5, div_factor: float = 1e3,
                       trace: bool = False):
        """Algorithm 5 around PCG.  With trace=True also returns the list of
        check windows: dicts with steps, action (WIN_* names), rstart, rend,
        factor."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        info = _Info()
        cap = max_it + 1
        win = (_Window * cap)()
        nwin = C.c_int32(0)
        self._lib.orc_adaptive_solve_ex(self._h, _ptr(b), _ptr(x), tol, max_it, k, s, gamma_min,
                                        rho_max, div_factor, win, cap, C.byref(nwin),
                                        C.byref(info))
        if not trace:
            return x, _info(info)
        tr = [dict(steps=w.steps, action=WIN_ACTIONS[w.action], rstart=w.rstart, rend=w.rend,
                   factor=w.factor) for w in win[: min(nwin.value, cap)]]
        return x, _info(info), tr

    def gmres(self, b, tol: float = 1e-8, max_it: int = 500, restart: int = 30):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        info = _Info()
        self._lib.orc_gmres(self._h, _ptr(b), _ptr(x), tol, max_it, restart, C.byref(info))
        return x, _info(info)

    def adaptive_gmres(self, b, tol: float = 1e-8, max_it: int = 500, restart: int = 30,
                       k: int = 3, s: int = 1, gamma_min: float = 0.01, rho_max: float = 0.5):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        info = _Info()
        self._lib.orc_adaptive_gmres(self._h, _ptr(b), _ptr(x), tol, max_it, restart, k, s,
                                     gamma_min, rho_max, C.byref(info))
        return x, _info(info)

    def level_sizes(self):
        out = []
        for l in range(self.num_levels):
            A = self.matrix(l, "A")
            H = self.matrix(l, "Ahat")
            out.append((A.nrows, A.nnz, H.nnz))
        return out
