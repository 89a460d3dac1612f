"""ctypes bindings of the oracle's plain-C sparse routines (test infrastructure).

``build_library()`` compiles ``nle_oracle.c`` with gcc into
``oracle/_liboracle.so`` (git-ignored) the first time it is needed.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nle_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build_library(force: bool = False) -> str:
    """Compile the oracle's C file (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build_library()
            lib = ctypes.CDLL(_LIB)
            lib.orc_ict.restype = ctypes.c_int
            lib.orc_ict.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i64p]
            lib.orc_transpose.restype = None
            lib.orc_transpose.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _i64p, _i32p, _f64p]
            lib.orc_levels.restype = ctypes.c_int64
            lib.orc_levels.argtypes = [ctypes.c_int64, _i64p, _i32p, ctypes.c_int, _i32p]
            lib.orc_level_sets.restype = None
            lib.orc_level_sets.argtypes = [ctypes.c_int64, _i32p, ctypes.c_int64, _i64p, _i32p]
            for f in ("orc_spmv", "orc_lsolve", "orc_usolve"):
                getattr(lib, f).restype = None
                getattr(lib, f).argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p]
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr_args(rowptr, col, val):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return rowptr, col, val


@dataclasses.dataclass
class ICFactor:
    """IC factor in two CSR copies: L (lower, diagonal last in each row) and
    U = L^T (upper, diagonal first), plus the level of every row of each."""
    n: int
    Lrowptr: np.ndarray
    Lcol: np.ndarray
    Lval: np.ndarray
    Urowptr: np.ndarray
    Ucol: np.ndarray
    Uval: np.ndarray
    levL: np.ndarray
    levU: np.ndarray
    nlevL: int
    nlevU: int

    @property
    def nnz(self) -> int:
        return int(self.Lrowptr[-1])


class ICBreakdown(RuntimeError):
    pass


def ic_factor(A, lfil: int, tau: float) -> ICFactor:
    """IC(lfil, tau_IC) of A (Section 2; reading documented in nle_oracle.c)."""
    lib = _get()
    n = A.n
    rowptr, col, val = _csr_args(A.rowptr, A.col, A.val)
    cap = int(n) * (int(lfil) + 1)
    Urow = np.zeros(n + 1, dtype=np.int64)
    Ucol = np.zeros(max(cap, 1), dtype=np.int32)
    Uval = np.zeros(max(cap, 1), dtype=np.float64)
    nnz = np.zeros(1, dtype=np.int64)
    bad = np.full(1, -1, dtype=np.int64)
    rc = lib.orc_ict(n, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p), int(lfil), float(tau), cap,
                     _p(Urow, _i64p), _p(Ucol, _i32p), _p(Uval, _f64p), _p(nnz, _i64p), _p(bad, _i64p))
    if rc == -2:
        raise ICBreakdown(f"non-positive pivot in column {int(bad[0])}")
    if rc != 0:
        raise RuntimeError(f"orc_ict failed with {rc}")
    m = int(nnz[0])
    Ucol = Ucol[:m].copy()
    Uval = Uval[:m].copy()
    Lrow = np.zeros(n + 1, dtype=np.int64)
    Lcol = np.zeros(max(m, 1), dtype=np.int32)
    Lval = np.zeros(max(m, 1), dtype=np.float64)
    lib.orc_transpose(n, _p(Urow, _i64p), _p(Ucol, _i32p), _p(Uval, _f64p), _p(Lrow, _i64p), _p(Lcol, _i32p),
                      _p(Lval, _f64p))
    Lcol = Lcol[:m]
    Lval = Lval[:m]
    levL, nlL = levels(n, Lrow, Lcol, lower=True)
    levU, nlU = levels(n, Urow, Ucol, lower=False)
    return ICFactor(n, Lrow, Lcol, Lval, Urow, Ucol, Uval, levL, levU, nlL, nlU)


def levels(n, rowptr, col, lower: bool):
    lib = _get()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    lev = np.zeros(max(n, 1), dtype=np.int32)
    nl = lib.orc_levels(n, _p(rowptr, _i64p), _p(col, _i32p), 1 if lower else 0, _p(lev, _i32p))
    return lev[:n], int(nl)


def level_sets(lev: np.ndarray, nlev: int):
    """(lptr, rows): rows of level l are rows[lptr[l]:lptr[l+1]], ascending."""
    lib = _get()
    n = len(lev)
    lev = np.ascontiguousarray(lev, dtype=np.int32)
    lptr = np.zeros(nlev + 1, dtype=np.int64)
    rows = np.zeros(max(n, 1), dtype=np.int32)
    lib.orc_level_sets(n, _p(lev, _i32p), nlev, _p(lptr, _i64p), _p(rows, _i32p))
    return lptr, rows[:n]


def spmv(A, x: np.ndarray) -> np.ndarray:
    lib = _get()
    rowptr, col, val = _csr_args(A.rowptr, A.col, A.val)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n)
    lib.orc_spmv(A.n, _p(rowptr, _i64p), _p(col, _i32p), _p(val, _f64p), _p(x, _f64p), _p(y, _f64p))
    return y


def lsolve(ic: ICFactor, b: np.ndarray) -> np.ndarray:
    lib = _get()
    b = np.ascontiguousarray(b, dtype=np.float64)
    y = np.empty(ic.n)
    lib.orc_lsolve(ic.n, _p(ic.Lrowptr, _i64p), _p(ic.Lcol, _i32p), _p(ic.Lval, _f64p), _p(b, _f64p), _p(y, _f64p))
    return y


def usolve(ic: ICFactor, b: np.ndarray) -> np.ndarray:
    lib = _get()
    b = np.ascontiguousarray(b, dtype=np.float64)
    y = np.empty(ic.n)
    lib.orc_usolve(ic.n, _p(ic.Urowptr, _i64p), _p(ic.Ucol, _i32p), _p(ic.Uval, _f64p), _p(b, _f64p), _p(y, _f64p))
    return y
