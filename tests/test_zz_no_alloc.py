"""The allocation-free entry point nle_ic_apply_noalloc, called through the C
ABI, gives the same c = (L L^T)^{-1} g as the handle-based nle_apply_prec
(k = 0 pairs, no projection) and as the oracle's P0hat, on two calls in a
row; it rejects overlapping g and c and reports an entry that is not
strictly triangular.

The entry point exists for callers that cannot allocate device memory when
they apply the preconditioner (code inside another framework's memory pool,
real-time loops that cannot take cudaMalloc's synchronisation, programs that
allocate only at start-up); its scratch is a fixed array inside the
library.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _split_factor(F, n):
    """Strictly lower CSR, diagonal, and strictly upper CSR of U = L^T (natural order)."""
    rp, col, val = F["Lrowptr"], F["Lcol"], F["Lval"]
    rows = np.repeat(np.arange(n), np.diff(rp))
    off = col != rows
    diag = val[~off]
    assert len(diag) == n
    lr, lc, lv = rows[off], col[off].astype(np.int64), val[off]
    Lrp = np.zeros(n + 1, np.int64)
    np.add.at(Lrp, lr + 1, 1)
    Lrp = np.cumsum(Lrp)
    order = np.lexsort((lr, lc))  # transpose: sort by (column, row)
    Urp = np.zeros(n + 1, np.int64)
    np.add.at(Urp, lc + 1, 1)
    Urp = np.cumsum(Urp)
    return (Lrp.astype(np.int32), lc.astype(np.int32), lv.copy(), Urp.astype(np.int32),
            lr[order].astype(np.int32), lv[order].copy(), diag.copy())


def test_no_alloc_ic_apply_matches_handle_entry_point():
    import torch

    import oracle as O
    from oracle.solver import p0hat
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    nle.load_library()
    A, st = W.workload("diff3d7_24")
    n = A.n
    assert n <= nle.NLE_NOALLOC_MAX_N
    s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64))
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    parts = _split_factor(s.get_factor(), n)
    dev = [torch.from_numpy(a).cuda() for a in parts]
    stream = torch.cuda.current_stream()
    ptr = [ctypes.c_void_p(t.data_ptr()) for t in dev]
    for seed in (11, 12):  # two calls in a row share the fixed scratch
        g = W.rng_for(seed).standard_normal(n)
        ref = s.apply_prec(g).cpu().numpy()  # the existing entry point
        gd = torch.from_numpy(g).cuda()
        c = torch.empty(n, dtype=torch.float64, device="cuda")
        rc = nle.nle_ic_apply_noalloc(n, ptr[0], ptr[1], ptr[2], ptr[3], ptr[4], ptr[5], ptr[6],
                                      ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                      ctypes.c_void_p(stream.cuda_stream))
        assert rc == nle.NLE_OK, nle.nle_last_error(None)
        got = c.cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, err
        want = p0hat(ic, g)  # the oracle's (L L^T)^{-1} g
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err <= 1e-11, err
    # in-place use (c overlapping g) is rejected before any work
    rc = nle.nle_ic_apply_noalloc(n, ptr[0], ptr[1], ptr[2], ptr[3], ptr[4], ptr[5], ptr[6],
                                  ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(gd.data_ptr() + 8),
                                  ctypes.c_void_p(stream.cuda_stream))
    assert rc == nle.NLE_ERR_ARG and "overlap" in nle.nle_last_error(None)
    # an entry on the diagonal in the strictly lower part is skipped (before
    # any load) and reported
    Lcol_bad = parts[1].copy()
    r = int(np.flatnonzero(np.diff(parts[0]) > 0)[0])
    Lcol_bad[parts[0][r]] = r
    bad = torch.from_numpy(Lcol_bad).cuda()
    rc = nle.nle_ic_apply_noalloc(n, ptr[0], ctypes.c_void_p(bad.data_ptr()), ptr[2], ptr[3], ptr[4], ptr[5],
                                  ptr[6], ctypes.c_void_p(gd.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream))
    assert rc == nle.NLE_ERR_CSR, nle.nle_last_error(None)
    s.close()
    # beyond the fixed scratch: rejected before any memory is touched
    rc = nle.nle_ic_apply_noalloc(nle.NLE_NOALLOC_MAX_N + 1, *([None] * 9), None)
    assert rc == 1 and "scratch" in nle.nle_last_error(None)
