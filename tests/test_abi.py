"""The C-ABI library builds, loads and exports every symbol include/nle.h
declares; host-side argument and CSR validation work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    return nle.load_library()


def declared_functions():
    with open(os.path.join(ROOT, "include", "nle.h")) as fh:
        txt = fh.read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nle_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    from paper_1312_1553_gb300 import nle

    decl = declared_functions()
    assert len(decl) >= 12
    assert sorted(nle.EXPORTS) == decl
    for name in decl:
        assert hasattr(lib, name), name


def test_default_options(lib):
    from paper_1312_1553_gb300 import nle

    o = nle.nle_default_options()
    assert o.k_max == 5 and o.tau_pcg == 1e-2 and o.tau_dacg == 1e-2 and o.max_dacg == 5000
    assert o.precision == nle.NLE_FP64 and o.exit_eigres == 1 and o.exit_stagnation == 1
    assert o.trsv_schedule == nle.NLE_SCHED_AUTO and o.trsv_warps == 16 and o.trsv_rows == 0 and o.trsv_poll_ns == 0
    assert o.ic_device == nle.NLE_IC_AUTO


def _create(A, opt=None):
    from paper_1312_1553_gb300 import nle

    rp = np.ascontiguousarray(A.rowptr, np.int64)
    ci = np.ascontiguousarray(A.col, np.int32)
    va = np.ascontiguousarray(A.val, np.float64)
    st, h = nle.nle_create(A.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, 0, None, opt)
    return st, h, nle.nle_last_error(None)


def test_argument_errors_without_device(lib):
    A = W.tridiag(5)
    bad = W.CSR(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([1.0]))
    st, h, msg = _create(bad)
    assert st == 1 and not h.value
    from paper_1312_1553_gb300 import nle

    o = nle.nle_default_options()
    o.k_max = 99
    st, h, msg = _create(A, o)
    assert st == 1 and "k_max" in msg
    o = nle.nle_default_options()
    o.trsv_schedule = 7
    st, h, msg = _create(A, o)
    assert st == 1 and "trsv_schedule" in msg
    o = nle.nle_default_options()
    o.ic_device = 3
    st, h, msg = _create(A, o)
    assert st == 1 and "ic_device" in msg


@pytest.mark.parametrize("case", ["unsorted", "asym", "nodiag", "negdiag"])
def test_csr_validation_without_device(lib, case):
    A = W.tridiag(6)
    rp, col, val = A.rowptr.copy(), A.col.copy(), A.val.copy()
    if case == "unsorted":
        col[1], col[2] = col[2], col[1]
        expect = 2
    elif case == "asym":
        val[1] = -0.5
        expect = 2
    elif case == "nodiag":
        # drop the diagonal of row 0 (and the symmetric partner keeps the pattern asymmetric)
        rp = np.array([0] + list(A.rowptr[1:] - 1), np.int64)
        col = np.delete(col, 0)
        val = np.delete(val, 0)
        expect = 2
    else:
        val[0] = -1.0
        expect = 3
    st, h, msg = _create(W.CSR(6, rp, col, val))
    assert st == expect, msg


@pytest.mark.parametrize("name", ["aniso2d_30x37", "diff3d7_24", "rgg3000", "hex27_16"])
@pytest.mark.parametrize("distance", [1, 2])
def test_multicolor_order_matches_reference_and_is_greedy(lib, name, distance):
    """nle_multicolor_order (host C) equals the definition in workloads, and
    the colouring it encodes is proper and greedy: no neighbour (distance 1
    or 2) shares a row's colour, and every smaller colour is held by an
    earlier neighbour."""
    from paper_1312_1553_gb300 import nle

    A, _ = W.workload(name)
    perm, nc = nle.multicolor_order(A, distance)
    ref, nc_ref, color = W.multicolor_order(A, distance, return_colors=True)
    assert nc == nc_ref
    np.testing.assert_array_equal(perm, ref)
    assert np.array_equal(np.sort(perm), np.arange(A.n))
    # perm lists the colours in order, rows ascending inside each
    key = color[perm] * A.n + perm
    assert np.all(np.diff(key) > 0)
    S = A.to_scipy().tocsr()
    S.data[:] = 1.0
    G = (S @ S).tocsr() if distance == 2 else S
    rng = W.rng_for(5)
    for i in rng.choice(A.n, size=min(A.n, 300), replace=False):
        nb = G.indices[G.indptr[i]:G.indptr[i + 1]]
        nb = nb[nb != i]
        assert not np.any(color[nb] == color[i]), i
        earlier = set(color[nb[nb < i]].tolist())
        assert set(range(color[i])) <= earlier, i


def test_multicolor_order_argument_errors(lib):
    from paper_1312_1553_gb300 import nle

    A = W.tridiag(6)
    with pytest.raises(nle.NLEError):
        nle.multicolor_order(A, 3)
    bad = W.CSR(A.n, A.rowptr.copy(), A.col.copy(), A.val.copy())
    bad.col[3] = 99
    with pytest.raises(nle.NLEError) as e:
        nle.multicolor_order(bad, 1)
    assert e.value.args and "column" in str(e.value)


def test_permute_is_symmetric_permutation():
    """workloads.permute(A, perm) = P A P^T with row k = row perm[k] of A:
    the dense matrices agree entry by entry and the columns stay sorted."""
    A, _ = W.workload("aniso2d_30x37")
    perm, _ = W.multicolor_order(A, 2)
    B = W.permute(A, perm)
    np.testing.assert_array_equal(B.dense(), A.dense()[np.ix_(perm, perm)])
    for i in range(B.n):
        c = B.col[B.rowptr[i]:B.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
