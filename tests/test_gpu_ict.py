"""Device IC(lfil, tau_IC) factor (Section 2, the factor of Phat_0 =
(L L^T)^{-1}): the same columns as the oracle's factor, bit for bit, and the
same errors as the host factor.

Every expected factor comes from ``oracle.ic_factor`` (pinned in
``test_oracle_pins.py`` against exact Cholesky and the tridiagonal case)."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nle():
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    nle.load_library()
    return nle


def dense_csr(M):
    import scipy.sparse as sp

    S = sp.csr_matrix(M)
    S.sort_indices()
    return W.CSR(M.shape[0], S.indptr.astype(np.int64), S.indices.astype(np.int32), S.data.astype(np.float64))


def factored(nle, A, lfil, tau, where, **opts):
    o = dict(precision=nle.NLE_FP64, ic_device=where)
    o.update(opts)
    s = nle.Eigensolver(A, o)
    s.factor_ic(lfil, tau)
    return s


def assert_same_factor(F, ic):
    np.testing.assert_array_equal(F["Lrowptr"], ic.Lrowptr)
    np.testing.assert_array_equal(F["Lcol"], ic.Lcol)
    np.testing.assert_array_equal(F["Lval"].view(np.uint64), ic.Lval.view(np.uint64))
    np.testing.assert_array_equal(F["levL"], ic.levL)
    np.testing.assert_array_equal(F["levU"], ic.levU)
    assert F["nlevL"] == ic.nlevL and F["nlevU"] == ic.nlevU


@pytest.mark.parametrize("name", ["aniso2d_30x37", "diff3d7_24", "diff2d5_60x70", "rgg3000", "hex27_16"])
def test_device_factor_bit_exact(nle, name):
    A, st = W.workload(name)
    s = factored(nle, A, st["lfil"], st["tau_ic"], nle.NLE_IC_DEVICE)
    info = s.last_stats()["ic"]
    assert info["on_device"] == 1 and info["kernel_ms"] > 0
    assert_same_factor(s.get_factor(), O.ic_factor(A, st["lfil"], st["tau_ic"]))
    s.close()


# lfil 0 (diagonal only), tau 0 (nothing dropped by size), the largest lfil
# a column record holds, and a drop threshold that removes most fill
@pytest.mark.parametrize("lfil,tau", [(0, 1e-3), (1, 0.0), (5, 1e-2), (31, 0.0), (31, 1e-4)])
@pytest.mark.parametrize("name", ["diff3d7_24", "hex27_16"])
def test_device_factor_parameters(nle, name, lfil, tau):
    A, _ = W.workload(name)
    s = factored(nle, A, lfil, tau, nle.NLE_IC_DEVICE)
    assert_same_factor(s.get_factor(), O.ic_factor(A, lfil, tau))
    s.close()


def test_device_factor_is_exact_cholesky_without_dropping(nle):
    """tau = 0 and lfil above the bandwidth keep every entry: L L^T = A
    exactly (up to rounding), and the pattern is the full band."""
    n, bw = 300, 6
    rng = np.random.default_rng(11)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(max(0, i - bw), min(n, i + bw + 1)):
            if i != j:
                rows.append(i), cols.append(j), vals.append(-abs(np.sin(0.7 * i + 1.3 * j)) - 0.05)
    M = np.zeros((n, n))
    M[rows, cols] = vals
    M = 0.5 * (M + M.T)
    np.fill_diagonal(M, -M.sum(axis=1) + 0.1 + rng.random(n))
    A = dense_csr(M)
    s = factored(nle, A, 31, 0.0, nle.NLE_IC_DEVICE)
    F = s.get_factor()
    assert_same_factor(F, O.ic_factor(A, 31, 0.0))
    L = np.zeros((n, n))
    for i in range(n):
        L[i, F["Lcol"][F["Lrowptr"][i]:F["Lrowptr"][i + 1]]] = F["Lval"][F["Lrowptr"][i]:F["Lrowptr"][i + 1]]
    np.testing.assert_allclose(L, np.linalg.cholesky(M), rtol=0, atol=1e-12 * np.abs(M).max())
    s.close()


@pytest.mark.parametrize("name", ["diff3d7_100", "hex27_96"])
def test_device_factor_bit_exact_full_size(nle, name):
    A, st = W.workload(name)
    s = factored(nle, A, st["lfil"], st["tau_ic"], nle.NLE_IC_DEVICE, precision=nle.NLE_MIXED)
    info = s.last_stats()["ic"]
    assert info["on_device"] == 1
    print(f"\n{name}: device factor {info['kernel_ms']:.1f} ms kernel, {info['factor_ms']:.1f} ms with copies, "
          f"set-up {info['setup_ms']:.0f} ms")
    assert_same_factor(s.get_factor(), O.ic_factor(A, st["lfil"], st["tau_ic"]))
    s.close()


def test_device_factor_with_multicolor_ordering(nle):
    """The factor of P A P^T: device and host agree bit for bit."""
    A, st = W.workload("diff3d7_24")
    Fs = []
    for where in (nle.NLE_IC_DEVICE, nle.NLE_IC_HOST):
        s = factored(nle, A, st["lfil"], st["tau_ic"], where, ordering=1)
        assert s.last_stats()["ic"]["on_device"] == (1 if where == nle.NLE_IC_DEVICE else 0)
        Fs.append(s.get_factor())
        s.close()
    for key in ("Lrowptr", "Lcol", "levL", "levU"):
        np.testing.assert_array_equal(Fs[0][key], Fs[1][key])
    np.testing.assert_array_equal(Fs[0]["Lval"].view(np.uint64), Fs[1]["Lval"].view(np.uint64))


def test_device_factor_reports_the_failing_pivot(nle):
    """An SPD-looking matrix (positive diagonal, symmetric) whose IC factor
    breaks down: both factors name the same column."""
    n = 200
    M = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    M[120, 121] = M[121, 120] = -1.9  # with the next line: the pivot of column 120 is negative
    M[119, 120] = M[120, 119] = -1.9
    A = dense_csr(M)
    try:
        O.ic_factor(A, 5, 0.0)
        pytest.fail("the oracle factor should break down")
    except O.ic.ICBreakdown as e:
        want = str(e).split()[-1]
    msgs = []
    for where in (nle.NLE_IC_DEVICE, nle.NLE_IC_HOST):
        s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64, ic_device=where))
        with pytest.raises(nle.NLEError) as e:
            s.factor_ic(5, 0.0)
        assert e.value.code == 3  # NLE_ERR_NOT_SPD
        msgs.append(str(e.value))
        s.close()
    assert all(m.rstrip().endswith(want) for m in msgs), (msgs, want)


def test_device_factor_lfil_limit(nle):
    A, st = W.workload("diff2d5_60x70")
    s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64, ic_device=nle.NLE_IC_DEVICE))
    with pytest.raises(nle.NLEError) as e:
        s.factor_ic(32, 1e-3)
    assert e.value.code == nle.NLE_ERR_ARG
    s.close()
    s = factored(nle, A, 32, 1e-3, nle.NLE_IC_AUTO)  # beyond the device records: the host factor
    assert s.last_stats()["ic"]["on_device"] == 0
    assert_same_factor(s.get_factor(), O.ic_factor(A, 32, 1e-3))
    s.close()


def test_device_factor_wait_is_bounded(nle):
    """A wait limit far below any real wait: the factor returns
    NLE_ERR_TIMEOUT instead of waiting, and the device stays usable."""
    A, st = W.workload("diff3d7_24")
    s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64, ic_device=nle.NLE_IC_DEVICE, spin_timeout_s=1e-9))
    with pytest.raises(nle.NLEError) as e:
        s.factor_ic(st["lfil"], st["tau_ic"])
    assert e.value.code == nle.NLE_ERR_TIMEOUT
    s.close()
    s = factored(nle, A, st["lfil"], st["tau_ic"], nle.NLE_IC_DEVICE)
    assert_same_factor(s.get_factor(), O.ic_factor(A, st["lfil"], st["tau_ic"]))
    s.close()
