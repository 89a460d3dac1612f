"""Thin Python binding of the nle C ABI (include/nle.h).

The functions below carry the C names and only marshal arguments (ctypes);
every step of the method runs in the CUDA library.  ``Eigensolver`` wraps a
handle with torch tensors: PyTorch supplies device memory and the stream.
Loading fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnle.so")

NLE_OK = 0
NLE_ERR_ARG, NLE_ERR_CSR, NLE_ERR_NOCONV, NLE_ERR_TIMEOUT = 1, 2, 5, 8
STATUS = {0: "NLE_OK", 1: "NLE_ERR_ARG", 2: "NLE_ERR_CSR", 3: "NLE_ERR_NOT_SPD", 4: "NLE_ERR_BREAKDOWN",
          5: "NLE_ERR_NOCONV", 6: "NLE_ERR_CUDA", 7: "NLE_ERR_OOM", 8: "NLE_ERR_TIMEOUT", 9: "NLE_ERR_STATE",
          10: "NLE_ERR_NO_DEVICE"}
NLE_FP64, NLE_MIXED = 0, 1
NLE_ORDER_NATURAL, NLE_ORDER_MULTICOLOR1, NLE_ORDER_MULTICOLOR2 = 0, 1, 2
NLE_BFGS_SIMPLIFIED, NLE_BFGS_FULL = 0, 1
NLE_SCHED_AUTO, NLE_SCHED_LEVEL, NLE_SCHED_CHAIN = 0, 1, 2
NLE_IC_AUTO, NLE_IC_HOST, NLE_IC_DEVICE = 0, 1, 2
SCHEDULES = {1: "level", 2: "chain"}
EXITS = ("tol", "maxit", "eigres", "stagnation", "breakdown")
PHASES = ("spmv", "update", "fwd_solve", "bwd_solve", "dots", "direction", "outer_fp64", "other")
NLE_MAX_P = 64

# every symbol include/nle.h declares
EXPORTS = ("nle_default_options", "nle_create", "nle_factor_ic", "nle_solve", "nle_backward", "nle_batch_solve",
           "nle_apply_shifted", "nle_apply_prec", "nle_pcg", "nle_get_factor", "nle_last_error", "nle_destroy",
           "nle_ic_apply_noalloc", "nle_multicolor_order", "nle_get_stats")
NLE_NOALLOC_MAX_N = 262144


class nle_options(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int), ("tau_pcg", ctypes.c_double), ("tau_dacg", ctypes.c_double),
                ("max_dacg", ctypes.c_int), ("precision", ctypes.c_int), ("exit_eigres", ctypes.c_int),
                ("exit_stagnation", ctypes.c_int), ("dacg_recompute", ctypes.c_int),
                ("spin_timeout_s", ctypes.c_double), ("grid_ctas", ctypes.c_int), ("trsv_warps", ctypes.c_int),
                ("ordering", ctypes.c_int), ("bfgs_update", ctypes.c_int), ("trsv_schedule", ctypes.c_int),
                ("trsv_poll_ns", ctypes.c_int), ("trsv_rows", ctypes.c_int),
                ("ic_device", ctypes.c_int)]


class nle_stats(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("dacg_its", ctypes.c_int * NLE_MAX_P), ("outer_its", ctypes.c_int * NLE_MAX_P),
                ("pcg_its", ctypes.c_int * NLE_MAX_P), ("converged", ctypes.c_int * NLE_MAX_P),
                ("final_res", ctypes.c_double * NLE_MAX_P), ("mvp_dacg", ctypes.c_int64),
                ("mvp_newton", ctypes.c_int64), ("exit_count", ctypes.c_int * 5), ("ms_dacg", ctypes.c_double),
                ("ms_newton", ctypes.c_double), ("ms_pcg_inner", ctypes.c_double),
                ("pcg_iterations", ctypes.c_int64), ("pcg_sum_m", ctypes.c_int64), ("pcg_sum_k", ctypes.c_int64),
                ("dacg_iterations", ctypes.c_int64), ("dacg_sum_m", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("ms_phase", ctypes.c_double * 8), ("ascending", ctypes.c_int),
                ("ms_batch", ctypes.c_double), ("trsv_schedule", ctypes.c_int), ("tune_ms_level", ctypes.c_double),
                ("tune_ms_chain", ctypes.c_double), ("tune_ms_level2", ctypes.c_double), ("strands", ctypes.c_int64),
                ("trsv_rows", ctypes.c_int), ("ic_on_device", ctypes.c_int), ("ms_ic_factor", ctypes.c_double),
                ("ms_ic_kernel", ctypes.c_double), ("ms_ic_setup", ctypes.c_double)]


class nle_pcg_info(ctypes.Structure):
    _fields_ = [("its", ctypes.c_int), ("exit", ctypes.c_int), ("gnorm0", ctypes.c_double),
                ("gnorm", ctypes.c_double), ("eigres", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_lib = None


def load_library(path: str = LIB_PATH):
    """Load libnle.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"nle CUDA library not built: {path} is missing")
    lib = ctypes.CDLL(path)
    sig = {
        "nle_default_options": (None, [ctypes.POINTER(nle_options)]),
        "nle_create": (ctypes.c_int, [_i64, _i64, _vp, _vp, _vp, ctypes.c_int, _vp, ctypes.POINTER(nle_options),
                                      ctypes.POINTER(_vp)]),
        "nle_factor_ic": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double]),
        "nle_solve": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                     ctypes.POINTER(nle_stats), ctypes.c_int]),
        "nle_backward": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int]),
        "nle_batch_solve": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, _vp, _vp, _vp, _vp]),
        "nle_apply_shifted": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int]),
        "nle_apply_prec": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int]),
        "nle_pcg": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, _vp, ctypes.c_int, _vp,
                                   ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(nle_pcg_info), ctypes.c_int]),
        "nle_get_factor": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "nle_multicolor_order": (ctypes.c_int, [_i64, _vp, _vp, ctypes.c_int, _vp, _vp]),
        "nle_get_stats": (ctypes.c_int, [_vp, ctypes.POINTER(nle_stats)]),
        "nle_last_error": (ctypes.c_char_p, [_vp]),
        "nle_destroy": (None, [_vp]),
        "nle_ic_apply_noalloc": (ctypes.c_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class NLEError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


# ---- functions with the C names (argument marshalling only) ---------------

def nle_default_options() -> nle_options:
    o = nle_options()
    load_library().nle_default_options(ctypes.byref(o))
    return o


def nle_last_error(h) -> str:
    m = load_library().nle_last_error(h)
    return m.decode() if m else ""


def nle_create(n, nnz, rowptr_ptr, col_ptr, val_ptr, on_device, stream_ptr, opt: Optional[nle_options]):
    out = _vp()
    st = load_library().nle_create(n, nnz, rowptr_ptr, col_ptr, val_ptr, int(on_device), stream_ptr,
                                   ctypes.byref(opt) if opt is not None else None, ctypes.byref(out))
    return st, out


def nle_factor_ic(h, lfil: int, tau_ic: float) -> int:
    return load_library().nle_factor_ic(h, int(lfil), float(tau_ic))


def nle_solve(h, p, tol, max_newton, max_pcg, X0_ptr, lambda_ptr, V_ptr, stats: Optional[nle_stats], on_device):
    return load_library().nle_solve(h, int(p), float(tol), int(max_newton), int(max_pcg), X0_ptr, lambda_ptr, V_ptr,
                                    ctypes.byref(stats) if stats is not None else None, int(on_device))


def nle_backward(h, gl_ptr, gv_ptr, grad_ptr, on_device) -> int:
    return load_library().nle_backward(h, gl_ptr, gv_ptr, grad_ptr, int(on_device))


def nle_batch_solve(count, handles_ptr, p, tol, max_newton, max_pcg, x0s_ptr, lambdas_ptr, vs_ptr, per_ptr) -> int:
    return load_library().nle_batch_solve(int(count), handles_ptr, int(p), float(tol), int(max_newton),
                                          int(max_pcg), x0s_ptr, lambdas_ptr, vs_ptr, per_ptr)


def nle_apply_shifted(h, theta, x_ptr, y_ptr, on_device) -> int:
    return load_library().nle_apply_shifted(h, float(theta), x_ptr, y_ptr, int(on_device))


def nle_apply_prec(h, k, S_ptr, R_ptr, m, Q_ptr, g_ptr, c_ptr, on_device) -> int:
    return load_library().nle_apply_prec(h, int(k), S_ptr, R_ptr, int(m), Q_ptr, g_ptr, c_ptr, int(on_device))


def nle_pcg(h, theta, tol, max_pcg, r_ptr, m, Q_ptr, k, S_ptr, R_ptr, s_ptr, info: nle_pcg_info, on_device) -> int:
    return load_library().nle_pcg(h, float(theta), float(tol), int(max_pcg), r_ptr, int(m), Q_ptr, int(k), S_ptr,
                                  R_ptr, s_ptr, ctypes.byref(info), int(on_device))


def nle_get_stats(h, stats: nle_stats) -> int:
    return _lib.nle_get_stats(h, ctypes.byref(stats))


def nle_multicolor_order(n, rowptr_ptr, col_ptr, distance, perm_ptr, ncolors_ptr) -> int:
    return _lib.nle_multicolor_order(n, rowptr_ptr, col_ptr, distance, perm_ptr, ncolors_ptr)


def multicolor_order(A, distance: int = 2):
    """(perm, ncolors) of nle_multicolor_order for a CSR with numpy arrays."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col, dtype=np.int32)
    perm = np.zeros(int(A.n), np.int32)
    nc = np.zeros(1, np.int32)
    st = nle_multicolor_order(int(A.n), _hptr(rp), _hptr(ci), distance, _hptr(perm), _hptr(nc))
    if st != NLE_OK:
        raise NLEError(st, nle_last_error(None))
    return perm, int(nc[0])


def nle_get_factor(h, nnz_ptr, rp_ptr, col_ptr, val_ptr, levL_ptr, levU_ptr, nlevL_ptr, nlevU_ptr) -> int:
    return load_library().nle_get_factor(h, nnz_ptr, rp_ptr, col_ptr, val_ptr, levL_ptr, levU_ptr, nlevL_ptr,
                                         nlevU_ptr)


def nle_destroy(h) -> None:
    load_library().nle_destroy(h)


def nle_ic_apply_noalloc(n, Lrp_ptr, Lcol_ptr, Lval_ptr, Urp_ptr, Ucol_ptr, Uval_ptr, diag_ptr, g_ptr, c_ptr,
                         stream_ptr) -> int:
    return load_library().nle_ic_apply_noalloc(int(n), Lrp_ptr, Lcol_ptr, Lval_ptr, Urp_ptr, Ucol_ptr, Uval_ptr,
                                               diag_ptr, g_ptr, c_ptr, stream_ptr)


# ---- convenience wrapper with torch tensors --------------------------------

def _dptr(t) -> int:
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class Eigensolver:
    """One SPD matrix on the current CUDA device.

    ``A`` is any object with ``n``, ``rowptr``, ``col``, ``val`` (numpy CSR as
    produced by ``workloads``).  ``options`` is a dict of nle_options fields.
    """

    def __init__(self, A, options: Optional[dict] = None, stream=None):
        import torch

        self.torch = torch
        opt = nle_default_options()
        for k, v in (options or {}).items():
            setattr(opt, k, v)
        self.opt = opt
        self.n = int(A.n)
        self.nnz = int(A.rowptr[-1])
        rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
        ci = np.ascontiguousarray(A.col, dtype=np.int32)
        va = np.ascontiguousarray(A.val, dtype=np.float64)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        st, h = nle_create(self.n, self.nnz, _hptr(rp), _hptr(ci), _hptr(va), 0, ctypes.c_void_p(self.stream.cuda_stream),
                           opt)
        if st != NLE_OK:
            raise NLEError(st, nle_last_error(None))
        self.h = h
        self.dev = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "h", None):
            nle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != NLE_OK and st not in allow:
            raise NLEError(st, nle_last_error(self.h))
        return st

    def factor_ic(self, lfil: int, tau_ic: float):
        self._check(nle_factor_ic(self.h, lfil, tau_ic))

    def get_factor(self):
        nnz = np.zeros(1, np.int64)
        nl = np.zeros(2, np.int64)
        self._check(nle_get_factor(self.h, _hptr(nnz), None, None, None, None, None, _hptr(nl), _hptr(nl[1:])))
        m = int(nnz[0])
        rp = np.zeros(self.n + 1, np.int64)
        col = np.zeros(m, np.int32)
        val = np.zeros(m, np.float64)
        levL = np.zeros(self.n, np.int32)
        levU = np.zeros(self.n, np.int32)
        self._check(nle_get_factor(self.h, _hptr(nnz), _hptr(rp), _hptr(col), _hptr(val), _hptr(levL), _hptr(levU),
                                   _hptr(nl), _hptr(nl[1:])))
        return dict(Lrowptr=rp, Lcol=col, Lval=val, levL=levL, levU=levU, nlevL=int(nl[0]), nlevU=int(nl[1]))

    def solve(self, p: int, tol: float, max_newton: int = 100, max_pcg: int = 20, X0=None, allow_noconv=False):
        """Returns (lambda (p,), V (p, n), stats dict) as float64 CUDA tensors."""
        torch = self.torch
        lam = torch.empty(p, dtype=torch.float64, device=self.dev)
        V = torch.empty((p, self.n), dtype=torch.float64, device=self.dev)
        x0 = None
        if X0 is not None:
            x0 = torch.as_tensor(X0, dtype=torch.float64).to(self.dev).contiguous()
        stats = nle_stats()
        st = nle_solve(self.h, p, tol, max_newton, max_pcg, _dptr(x0) if x0 is not None else None, _dptr(lam),
                       _dptr(V), stats, 1)
        self._check(st, allow=(5,) if allow_noconv else ())
        return lam, V, stats_dict(stats)

    def last_stats(self) -> dict:
        """Statistics of the last solve on this handle (single or batched); after
        factor_ic alone, only the set-up fields (schedule, autotuner, IC factor)."""
        st = nle_stats()
        self._check(nle_get_stats(self.h, st))
        return stats_dict(st)

    def backward(self, gbar_lambda=None, gbar_V=None, grad=None):
        """Accumulate dL/dA_e for every stored entry e into grad (created as
        zeros when None) for the last solve; gbar_V is (p, n)."""
        torch = self.torch
        if grad is None:
            grad = torch.zeros(self.nnz, dtype=torch.float64, device=self.dev)
        gl = None if gbar_lambda is None else torch.as_tensor(gbar_lambda, dtype=torch.float64).to(self.dev).contiguous()
        gv = None if gbar_V is None else torch.as_tensor(gbar_V, dtype=torch.float64).to(self.dev).contiguous()
        self._check(nle_backward(self.h, _dptr(gl) if gl is not None else None, _dptr(gv) if gv is not None else None,
                                 _dptr(grad), 1))
        return grad

    def apply_shifted(self, theta: float, x):
        torch = self.torch
        x = torch.as_tensor(x, dtype=torch.float64).to(self.dev).contiguous()
        y = torch.empty_like(x)
        self._check(nle_apply_shifted(self.h, theta, _dptr(x), _dptr(y), 1))
        return y

    def apply_prec(self, g, S=None, R=None, Q=None):
        torch = self.torch
        g = torch.as_tensor(g, dtype=torch.float64).to(self.dev).contiguous()
        k = 0 if S is None else len(S)
        m = 0 if Q is None else len(Q)
        St = torch.as_tensor(np.asarray(S), dtype=torch.float64).to(self.dev).contiguous() if k else None
        Rt = torch.as_tensor(np.asarray(R), dtype=torch.float64).to(self.dev).contiguous() if k else None
        Qt = torch.as_tensor(np.asarray(Q), dtype=torch.float64).to(self.dev).contiguous() if m else None
        c = torch.empty_like(g)
        self._check(nle_apply_prec(self.h, k, _dptr(St) if k else None, _dptr(Rt) if k else None, m,
                                   _dptr(Qt) if m else None, _dptr(g), _dptr(c), 1))
        return c

    def pcg(self, theta: float, tol: float, max_pcg: int, r, Q, S=None, R=None):
        """One inner solve; Q is (m, n) with the current iterate as its last row."""
        torch = self.torch
        r = torch.as_tensor(r, dtype=torch.float64).to(self.dev).contiguous()
        Qt = torch.as_tensor(np.asarray(Q), dtype=torch.float64).to(self.dev).contiguous()
        k = 0 if S is None else len(S)
        St = torch.as_tensor(np.asarray(S), dtype=torch.float64).to(self.dev).contiguous() if k else None
        Rt = torch.as_tensor(np.asarray(R), dtype=torch.float64).to(self.dev).contiguous() if k else None
        s = torch.empty_like(r)
        info = nle_pcg_info()
        self._check(nle_pcg(self.h, theta, tol, max_pcg, _dptr(r), Qt.shape[0], _dptr(Qt), k,
                            _dptr(St) if k else None, _dptr(Rt) if k else None, _dptr(s), info, 1))
        return s, dict(its=info.its, exit=EXITS[info.exit], gnorm0=info.gnorm0, gnorm=info.gnorm, eigres=info.eigres)


def batch_solve(solvers, p: int, tol: float, max_newton: int = 100, max_pcg: int = 20, X0s=None):
    """nle_batch_solve over Eigensolver objects (created with grid_ctas <= 8).
    Returns (lambdas, Vs, statuses): lists of CUDA tensors and status codes."""
    import torch

    count = len(solvers)
    dev = solvers[0].dev
    lams = [torch.empty(p, dtype=torch.float64, device=dev) for _ in solvers]
    Vs = [torch.empty((p, s.n), dtype=torch.float64, device=dev) for s in solvers]
    x0t = None
    if X0s is not None:
        x0t = [torch.as_tensor(x, dtype=torch.float64).to(dev).contiguous() for x in X0s]
    H = (ctypes.c_void_p * count)(*[s.h.value for s in solvers])
    L = (ctypes.c_void_p * count)(*[t.data_ptr() for t in lams])
    V = (ctypes.c_void_p * count)(*[t.data_ptr() for t in Vs])
    X = (ctypes.c_void_p * count)(*[t.data_ptr() for t in x0t]) if x0t is not None else None
    per = (ctypes.c_int * count)()
    st = nle_batch_solve(count, H, p, tol, max_newton, max_pcg, X, L, V, per)
    if st not in (NLE_OK, 5):
        raise NLEError(st, nle_last_error(solvers[0].h))
    return lams, Vs, list(per)


def stats_dict(s: nle_stats) -> dict:
    p = s.p
    return dict(p=p, dacg_its=list(s.dacg_its[:p]), outer_its=list(s.outer_its[:p]), pcg_its=list(s.pcg_its[:p]),
                converged=[bool(x) for x in s.converged[:p]], final_res=list(s.final_res[:p]),
                mvp_dacg=int(s.mvp_dacg), mvp_newton=int(s.mvp_newton),
                exits={EXITS[i]: int(s.exit_count[i]) for i in range(5)}, ms_dacg=float(s.ms_dacg),
                ms_newton=float(s.ms_newton), pcg_iterations=int(s.pcg_iterations), pcg_sum_m=int(s.pcg_sum_m),
                pcg_sum_k=int(s.pcg_sum_k), dacg_iterations=int(s.dacg_iterations), dacg_sum_m=int(s.dacg_sum_m),
                kernel_launches=int(s.kernel_launches),
                ms_phase=dict(zip(PHASES, [float(x) for x in s.ms_phase])), ascending=bool(s.ascending),
                ms_batch=float(s.ms_batch), trsv_schedule=SCHEDULES.get(int(s.trsv_schedule), "none"),
                tune_ms=dict(level=float(s.tune_ms_level), chain=float(s.tune_ms_chain),
                             level2=float(s.tune_ms_level2)), strands=int(s.strands), trsv_rows=int(s.trsv_rows),
                ic=dict(on_device=int(s.ic_on_device), factor_ms=float(s.ms_ic_factor),
                        kernel_ms=float(s.ms_ic_kernel), setup_ms=float(s.ms_ic_setup)))


def _eigsh_function():
    import torch

    class EigshFunction(torch.autograd.Function):
        """(lambda, V) = leftmost p eigenpairs of the SPD matrix with a fixed CSR
        pattern and values `values` (nnz, float64).  The backward pass is the
        library's adjoint (nle_backward): dlambda_j/dA_ab = v_ja v_jb and the
        eigenvector part through the projected PCG solve with shift lambda_j.
        Entries (a,b) and (b,a) are independent inputs; a symmetric
        parametrisation sums their gradients."""

        @staticmethod
        def forward(ctx, values, rowptr, col, p, tol, lfil, tau_ic, options, X0):
            class _A:
                pass

            A = _A()
            A.n = len(rowptr) - 1
            A.rowptr = np.asarray(rowptr, dtype=np.int64)
            A.col = np.asarray(col, dtype=np.int32)
            A.val = values.detach().to("cpu", torch.float64).numpy()
            s = Eigensolver(A, options)
            s.factor_ic(lfil, tau_ic)
            lam, V, stats = s.solve(p, tol, 100, 20, X0)
            ctx.solver = s
            return lam, V

        @staticmethod
        def backward(ctx, glam, gV):
            s = ctx.solver
            grad = s.backward(glam, gV)
            s.close()
            return grad.to(glam.device if glam is not None else grad.device), None, None, None, None, None, None, None, None

    return EigshFunction


def eigsh(values, rowptr, col, p: int, tol: float = 1e-8, lfil: int = 30, tau_ic: float = 1e-2, options=None,
          X0=None):
    """Differentiable leftmost eigenpairs (see EigshFunction)."""
    return _eigsh_function().apply(values, rowptr, col, p, tol, lfil, tau_ic, options, X0)
