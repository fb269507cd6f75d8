"""ctypes binding of libamg.so (include/amg.h).

Argument marshalling only: every computation happens in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (their data pointers are
passed through); host buffers are numpy arrays.  If the library has not been
built, importing works but the first call raises -- there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libamg.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, NOT_CONVERGED, DIVERGED, BREAKDOWN, TIMEOUT, REJECTED = range(9)
METHOD_SPARSE, METHOD_HYBRID, METHOD_NONGALERKIN = 0, 1, 2
LUMP_DIAG, LUMP_STRONG = 0, 1
KRYLOV_CG, KRYLOV_GMRES = 0, 1
PREC_FP64, PREC_FP32, PREC_FP32_BF16 = 0, 1, 2
SPMV_AUTO, SPMV_CSR2, SPMV_CSR4, SPMV_CSR8, SPMV_CSR16, SPMV_CSR32, SPMV_SELL32, SPMV_CSR1 = -1, 1, 2, 3, 4, 5, 6, 7
SPMV_SELL16, SPMV_SELL8 = 8, 9
SPMV_NAMES = {1: "csr2", 2: "csr4", 3: "csr8", 4: "csr16", 5: "csr32", 6: "sell32", 7: "csr1", 8: "sell16",
              9: "sell8"}
# kernel classes of amg_timing_get
K_PRE, K_RESTRICT, K_PROLONG, K_POST, K_COARSE, K_AP, K_VEC = range(7)


class AmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "AMG_OK", 1: "AMG_ERR_INVALID", 2: "AMG_ERR_OOM", 3: "AMG_ERR_CUDA",
           4: "AMG_NOT_CONVERGED", 5: "AMG_DIVERGED", 6: "AMG_BREAKDOWN", 7: "AMG_TIMEOUT",
           8: "AMG_REJECTED"}


class CSRStruct(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int), ("ncols", C.c_int64)]


class Options(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_size", C.c_int), ("max_levels", C.c_int),
                ("seed", C.c_uint64), ("method", C.c_int), ("precision", C.c_int),
                ("k_check", C.c_int), ("s_levels", C.c_int), ("gamma_min", C.c_double),
                ("rho_max", C.c_double), ("level_offset", C.c_int), ("spmv_variant", C.c_int),
                ("use_graph", C.c_int), ("check_every", C.c_int),
                ("setup_timing", C.c_int), ("lump", C.c_int), ("krylov", C.c_int),
                ("restart", C.c_int), ("div_factor", C.c_double), ("transfer_variant", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("status", C.c_int), ("resets", C.c_int),
                ("replacements", C.c_int), ("final_relres", C.c_double),
                ("conv_factor", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LevelInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_galerkin", C.c_int64), ("nnz_operator", C.c_int64),
                ("nnz_p", C.c_int64), ("n_coarse", C.c_int64), ("gamma", C.c_double),
                ("spmv_variant", C.c_int), ("value_bytes", C.c_int), ("bytes_per_cycle", C.c_double),
                ("spmv_variant_p", C.c_int), ("spmv_variant_r", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CommInfo(C.Structure):
    _fields_ = [("parts", C.c_int), ("messages", C.c_int64), ("halo_values", C.c_int64),
                ("max_messages", C.c_int64), ("max_halo", C.c_int64), ("messages_galerkin", C.c_int64),
                ("halo_galerkin", C.c_int64), ("messages_p", C.c_int64), ("halo_p", C.c_int64),
                ("messages_r", C.c_int64), ("halo_r", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerOpts(C.Structure):
    _fields_ = [("max_batch", C.c_int), ("hbm_budget", C.c_int64), ("max_queue", C.c_int),
                ("max_it", C.c_int), ("stage_budget", C.c_int64), ("wait_limit_ms", C.c_int64)]


_lock = threading.Lock()
_lib = None

# symbol -> (restype, argtypes); the complete C ABI of include/amg.h
_vp, _i, _i64, _d, _u64 = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64
SIGNATURES = {
    "amg_options_default": (None, [C.POINTER(Options)]),
    "amg_setup": (_i, [C.POINTER(CSRStruct), _d, _vp, _i, C.POINTER(Options), _vp, C.POINTER(_vp)]),
    "amg_hierarchy_assemble": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _i, C.POINTER(Options), _vp,
                                    C.POINTER(_vp)]),
    "amg_sparsify": (_i, [_vp, _vp, _i]),
    "amg_reintroduce": (_i, [_vp, _i, C.POINTER(_i)]),
    "amg_solve": (_i, [_vp, _vp, _vp, _d, _i, _i, _i, _vp, C.POINTER(SolveInfo)]),
    "amg_solve_batch": (_i, [_vp, _i, _vp, _vp, _d, _i, _i, _vp, _vp]),
    "amg_precond_apply": (_i, [_vp, _vp, _vp, _vp]),
    "amg_num_levels": (_i, [_vp]),
    "amg_level_stats": (_i, [_vp, _i, C.POINTER(LevelInfo)]),
    "amg_level_export": (_i, [_vp, _i, _i, _vp, _vp, _vp, C.POINTER(_i64), C.POINTER(_i64),
                              C.POINTER(_i64)]),
    "amg_level_array": (_i, [_vp, _i, _i, _vp, C.POINTER(_i64)]),
    "amg_timing_enable": (_i, [_vp, _i]),
    "amg_timing_get": (_i, [_vp, _i, _i, C.POINTER(_i64), C.POINTER(_d), C.POINTER(_d)]),
    "amg_timing_reset": (_i, [_vp]),
    "amg_hierarchy_save": (_i, [_vp, C.c_char_p]),
    "amg_hierarchy_load": (_i, [C.c_char_p, C.POINTER(Options), _vp, C.POINTER(_vp)]),
    "amg_free": (None, [_vp]),
    "amg_status_str": (C.c_char_p, [_i]),
    "amg_last_error": (C.c_char_p, []),
    "amg_device_bytes": (_i64, [_vp]),
    "amg_kernel_launches": (_i64, []),
    "amg_debug_fail_allocation": (None, [_i64]),
    "amg_residual_noalloc": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "amg_halo_plan": (_i, [_i64, _i64, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp]),
    "amg_partition": (_i, [_vp, _i]),
    "amg_comm_stats": (_i, [_vp, _i, C.POINTER(CommInfo)]),
    "amg_partition_rows": (_i, [_vp, _i, _vp]),
    "amg_server_opts_default": (None, [C.POINTER(ServerOpts)]),
    "amg_server_create": (_i, [C.POINTER(ServerOpts), C.POINTER(_vp)]),
    "amg_server_register": (_i, [_vp, _vp, C.POINTER(_i)]),
    "amg_server_submit": (_i, [_vp, _i, _vp, _d, C.POINTER(_u64)]),
    "amg_server_wait": (_i, [_vp, _u64, _vp, _i, C.POINTER(SolveInfo)]),
    "amg_server_destroy": (None, [_vp]),
}


def lib():
    """Load libamg.so (raises if it was not built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1512_04629_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name, None)
                if f is None:
                    continue
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def _check(st: int, what: str = ""):
    if st != OK:
        msg = lib().amg_last_error().decode()
        raise AmgError(st, f"{what}: {msg}" if what else msg)


def default_options(**kw) -> Options:
    o = Options()
    lib().amg_options_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------------
# buffer helpers
# ---------------------------------------------------------------------------
def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch

        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return None


def csr_struct(rowptr, col, val, ncols: int = 0):
    """CSRStruct over numpy arrays or torch CUDA tensors (kept alive by the caller)."""
    on_dev = _is_torch_cuda(rowptr)
    if not on_dev:
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
    s = CSRStruct(len(rowptr) - 1, int(rowptr[-1]), _ptr(rowptr).value, _ptr(col).value,
                  _ptr(val).value, 1 if on_dev else 0, ncols)
    s._keep = (rowptr, col, val)
    return s


def _as_csr(A):
    if isinstance(A, CSRStruct):
        return A
    if hasattr(A, "indptr"):
        return csr_struct(A.indptr, A.indices, A.data, A.shape[1] if A.shape[1] != A.shape[0] else 0)
    nrows = getattr(A, "nrows", None) or A.n
    ncols = getattr(A, "ncols", None) or nrows
    return csr_struct(A.rowptr, A.col, A.val, ncols if ncols != nrows else 0)


def _gammas(gamma):
    if gamma is None:
        return None, 0
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    return g, len(g)


@dataclass
class Matrix:
    nrows: int
    ncols: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.nrows, self.ncols))


# ---------------------------------------------------------------------------
# hierarchy
# ---------------------------------------------------------------------------
class Hierarchy:
    """A device-resident AMG hierarchy (amg_setup / amg_hierarchy_assemble)."""

    def __init__(self, handle):
        self._h = handle
        self._lib = lib()

    @classmethod
    def setup(cls, A, theta: float = 0.25, gamma=None, stream=None, **opts):
        L = lib()
        o = default_options(theta=theta, **opts)
        a = _as_csr(A)
        g, ng = _gammas(gamma)
        out = C.c_void_p()
        st = L.amg_setup(C.byref(a), theta, _ptr(g), ng, C.byref(o), _stream_handle(stream),
                         C.byref(out))
        _check(st, "amg_setup")
        return cls(out)

    @classmethod
    def assemble(cls, A_levels, P_levels, cf_levels, inM_levels, gamma=None, stream=None, **opts):
        L = lib()
        o = default_options(**opts)
        nlev = len(A_levels)
        a_structs = [_as_csr(a) for a in A_levels]
        p_structs = [_as_csr(p) for p in P_levels]
        As = (CSRStruct * nlev)(*a_structs)
        keep = [a_structs, p_structs]
        Ps = (CSRStruct * max(1, nlev - 1))(*p_structs) if nlev > 1 else None
        cfs = [np.ascontiguousarray(c, dtype=np.int8) for c in cf_levels]
        ims = [np.ascontiguousarray(m, dtype=np.uint8) if m is not None else np.zeros(1, np.uint8)
               for m in inM_levels]
        cf_arr = (C.c_void_p * max(1, len(cfs)))(*[c.ctypes.data for c in cfs]) if cfs else None
        im_arr = (C.c_void_p * max(1, len(ims)))(*[m.ctypes.data for m in ims]) if ims else None
        g, ng = _gammas(gamma)
        out = C.c_void_p()
        st = L.amg_hierarchy_assemble(nlev, C.cast(As, C.c_void_p), C.cast(Ps, C.c_void_p) if Ps else None,
                                      C.cast(cf_arr, C.c_void_p) if cf_arr else None,
                                      C.cast(im_arr, C.c_void_p) if im_arr else None,
                                      _ptr(g), ng, C.byref(o), _stream_handle(stream), C.byref(out))
        del keep
        _check(st, "amg_hierarchy_assemble")
        return cls(out)

    @classmethod
    def load(cls, path: str, stream=None, **opts):
        o = default_options(**opts)
        out = C.c_void_p()
        _check(lib().amg_hierarchy_load(path.encode(), C.byref(o), _stream_handle(stream), C.byref(out)),
               "amg_hierarchy_load")
        return cls(out)

    def save(self, path: str):
        _check(self._lib.amg_hierarchy_save(self._h, path.encode()), "amg_hierarchy_save")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.amg_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def num_levels(self) -> int:
        return self._lib.amg_num_levels(self._h)

    def sparsify(self, gamma):
        g, ng = _gammas(gamma)
        _check(self._lib.amg_sparsify(self._h, _ptr(g), ng), "amg_sparsify")

    def reintroduce(self, s_levels: int = 1) -> int:
        c = C.c_int(0)
        _check(self._lib.amg_reintroduce(self._h, s_levels, C.byref(c)), "amg_reintroduce")
        return c.value

    def solve(self, b, x=None, tol: float = 1e-8, max_it: int = 500, adaptive: bool = False,
              stream=None, raise_on_status: bool = False):
        """Solve A x = b; b/x numpy (host) or torch CUDA tensors (device)."""
        on_dev = _is_torch_cuda(b)
        if x is None:
            if on_dev:
                import torch

                x = torch.zeros_like(b)
            else:
                b = np.ascontiguousarray(b, dtype=np.float64)
                x = np.zeros_like(b)
        info = SolveInfo()
        st = self._lib.amg_solve(self._h, _ptr(b), _ptr(x), tol, max_it, 1 if adaptive else 0,
                                 1 if on_dev else 0, _stream_handle(stream), C.byref(info))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA) or (raise_on_status and st != OK):
            _check(st, "amg_solve")
        return x, info

    def solve_batch(self, B, X=None, tol: float = 1e-8, max_it: int = 500, stream=None):
        """k solves; B is n x k row-major (numpy or torch CUDA)."""
        on_dev = _is_torch_cuda(B)
        k = B.shape[1]
        if X is None:
            if on_dev:
                import torch

                X = torch.zeros_like(B)
            else:
                B = np.ascontiguousarray(B, dtype=np.float64)
                X = np.zeros_like(B)
        infos = (SolveInfo * k)()
        st = self._lib.amg_solve_batch(self._h, k, _ptr(B), _ptr(X), tol, max_it, 1 if on_dev else 0,
                                       _stream_handle(stream), C.cast(infos, C.c_void_p))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "amg_solve_batch")
        return X, [infos[i] for i in range(k)]

    def precond_apply(self, r, z, stream=None):
        _check(self._lib.amg_precond_apply(self._h, _ptr(r), _ptr(z), _stream_handle(stream)),
               "amg_precond_apply")

    def level_stats(self, level: int) -> dict:
        li = LevelInfo()
        _check(self._lib.amg_level_stats(self._h, level, C.byref(li)), "amg_level_stats")
        return li.as_dict()

    def export(self, level: int, which: str = "A") -> Matrix:
        code = {"A": 0, "Ahat": 1, "P": 2, "R": 3}[which]
        nr, nc, nz = C.c_int64(), C.c_int64(), C.c_int64()
        _check(self._lib.amg_level_export(self._h, level, code, None, None, None, C.byref(nr), C.byref(nc),
                                          C.byref(nz)), "amg_level_export")
        rp = np.zeros(nr.value + 1, np.int32)
        ci = np.zeros(max(nz.value, 1), np.int32)
        v = np.zeros(max(nz.value, 1), np.float64)
        _check(self._lib.amg_level_export(self._h, level, code, _ptr(rp), _ptr(ci), _ptr(v), None, None, None),
               "amg_level_export")
        return Matrix(nr.value, nc.value, rp, ci[: nz.value], v[: nz.value])

    def level_array(self, level: int, which: str) -> np.ndarray:
        code, dt = {"cf": (0, np.int8), "keep": (1, np.uint8), "inM": (2, np.uint8),
                    "l1": (3, np.float64), "strong": (4, np.uint8)}[which]
        cnt = C.c_int64()
        _check(self._lib.amg_level_array(self._h, level, code, None, C.byref(cnt)), "amg_level_array")
        out = np.zeros(max(cnt.value, 1), dtype=dt)
        _check(self._lib.amg_level_array(self._h, level, code, _ptr(out), C.byref(cnt)), "amg_level_array")
        return out[: cnt.value]

    def partition(self, parts: int):
        """Split every level into `parts` row blocks (1 removes the split)."""
        _check(self._lib.amg_partition(self._h, parts), "amg_partition")
        self._parts = parts

    def comm_stats(self, level: int) -> dict:
        ci = CommInfo()
        _check(self._lib.amg_comm_stats(self._h, level, C.byref(ci)), "amg_comm_stats")
        return ci.as_dict()

    def partition_rows(self, level: int) -> np.ndarray:
        parts = getattr(self, "_parts", 1)
        out = np.zeros(max(parts, 1) + 1, dtype=np.int64)
        _check(self._lib.amg_partition_rows(self._h, level, _ptr(out)), "amg_partition_rows")
        return out

    def timing_enable(self, on: bool = True):
        _check(self._lib.amg_timing_enable(self._h, 1 if on else 0), "amg_timing_enable")

    def timing_reset(self):
        _check(self._lib.amg_timing_reset(self._h), "amg_timing_reset")

    def timing_get(self, kind: int, level: int):
        n, ms, by = C.c_int64(), C.c_double(), C.c_double()
        _check(self._lib.amg_timing_get(self._h, kind, level, C.byref(n), C.byref(ms), C.byref(by)),
               "amg_timing_get")
        return n.value, ms.value, by.value


def device_bytes() -> int:
    return lib().amg_device_bytes(None)


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return lib().amg_kernel_launches()


def halo_plan(rowptr, col, ncols: int, row0, col0):
    """Host-side halo plan of a row-partitioned CSR operator (amg_halo_plan;
    needs no GPU).  Returns (cext, goff, gcol, recv) with recv as a
    parts x parts array (values block p receives from block q)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    row0 = np.ascontiguousarray(row0, dtype=np.int64)
    col0 = np.ascontiguousarray(col0, dtype=np.int64)
    parts = len(row0) - 1
    nnz = int(rowptr[-1])
    cext = np.zeros(max(nnz, 1), dtype=np.int32)
    goff = np.zeros(parts + 1, dtype=np.int64)
    gcol = np.zeros(max(nnz, 1), dtype=np.int32)
    recv = np.zeros(parts * parts, dtype=np.int64)
    _check(lib().amg_halo_plan(len(rowptr) - 1, ncols, _ptr(rowptr), _ptr(col), parts, _ptr(row0), _ptr(col0),
                               _ptr(cext), _ptr(goff), _ptr(gcol), _ptr(recv)), "amg_halo_plan")
    return cext[:nnz], goff, gcol[: goff[-1]], recv.reshape(parts, parts)


def debug_fail_allocation(after: int) -> None:
    """Host-side fault injection: the device allocation `after` allocations
    from now fails as out of memory (-1 disarms)."""
    lib().amg_debug_fail_allocation(after)


# ---------------------------------------------------------------------------
# server
# ---------------------------------------------------------------------------
class Server:
    """Continuous-batching solve server (amg_server_*)."""

    def __init__(self, max_batch: int = 32, hbm_budget: int = 0, max_queue: int = 4096, max_it: int = 500,
                 stage_budget: int = 0, wait_limit_ms: int | None = None):
        L = lib()
        o = ServerOpts()
        L.amg_server_opts_default(C.byref(o))
        o.max_batch, o.hbm_budget, o.max_queue, o.max_it = max_batch, hbm_budget, max_queue, max_it
        o.stage_budget = stage_budget
        if wait_limit_ms is not None:
            o.wait_limit_ms = wait_limit_ms
        out = C.c_void_p()
        _check(L.amg_server_create(C.byref(o), C.byref(out)), "amg_server_create")
        self._s = out
        self._lib = L
        self._n = {}
        self._hier = []

    def register(self, h: Hierarchy) -> int:
        hid = C.c_int()
        _check(self._lib.amg_server_register(self._s, h.handle, C.byref(hid)), "amg_server_register")
        self._n[hid.value] = h.level_stats(0)["n"]
        self._hier.append(h)
        return hid.value

    def submit(self, hid: int, b: np.ndarray, tol: float = 1e-8) -> int:
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = C.c_uint64()
        st = self._lib.amg_server_submit(self._s, hid, _ptr(b), tol, C.byref(t))
        _check(st, "amg_server_submit")
        return t.value

    def try_submit(self, hid: int, b: np.ndarray, tol: float = 1e-8):
        b = np.ascontiguousarray(b, dtype=np.float64)
        t = C.c_uint64()
        st = self._lib.amg_server_submit(self._s, hid, _ptr(b), tol, C.byref(t))
        return st, t.value

    def wait(self, ticket: int, hid: int, timeout_ms: int = 60000):
        x = np.zeros(self._n[hid], dtype=np.float64)
        info = SolveInfo()
        st = self._lib.amg_server_wait(self._s, ticket, _ptr(x), timeout_ms, C.byref(info))
        if st in (ERR_INVALID, ERR_OOM, ERR_CUDA):
            _check(st, "amg_server_wait")
        return st, x, info

    def close(self):
        if getattr(self, "_s", None):
            self._lib.amg_server_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
