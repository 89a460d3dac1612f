"""Parity of the CUDA library (through its C ABI) with the oracle.

Inputs are the seeded workloads; every expected value comes from ``oracle/``
(or from tests/golden/*.json, written by tests/golden/make_golden.py, which
calls only the oracle).  Tolerances:
  FP64 path   eigenvalues 1e-10 relative, building blocks near FP64 rounding;
  mixed path  eigenvalues 1e-8 relative, eigenvector angles 1e-6, the
              FP32 SpMV within its rounding bound 30*eps32*sum|a_ij x_j|,
              FP32 preconditioner / inner solve within 1e-4 / 2e-3 relative
              (FP32 triangular solves and 20 FP32 CG steps; a logic error
              gives O(1) differences).
"""
import json
import math
import os

import numpy as np
import pytest

import fullsize_checks as FC
import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
PRECS = ["fp64", "mixed"]
EPS32 = 2.0 ** -24


@pytest.fixture(scope="session")
def nle():
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    nle.load_library()
    return nle


_cache = {}


def load(name):
    if name not in _cache:
        _cache[name] = W.workload(name)
    return _cache[name]


def solver(nle, A, prec, **opts):
    o = dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64)
    o.update(opts)
    return nle.Eigensolver(A, o)


def align(v, ref):
    return v if float(v @ ref) >= 0 else -v


def sin_angle(a, b):
    """sin of the angle between a and b as the norm of the rejection of a
    from b (no cancellation, unlike sqrt(1 - cos^2))."""
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return float(np.linalg.norm(a - (a @ b) * b))


# ---------------------------------------------------------------------------
# set-up: IC factor and levels are bit-exact
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["aniso2d_30x37", "diff3d7_24", "diff2d5_60x70", "rgg3000", "hex27_16"])
def test_factor_and_levels_bit_exact(nle, name):
    A, st = load(name)
    s = solver(nle, A, "fp64")
    s.factor_ic(st["lfil"], st["tau_ic"])
    F = s.get_factor()
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    np.testing.assert_array_equal(F["Lrowptr"], ic.Lrowptr)
    np.testing.assert_array_equal(F["Lcol"], ic.Lcol)
    np.testing.assert_array_equal(F["Lval"].view(np.uint64), ic.Lval.view(np.uint64))
    np.testing.assert_array_equal(F["levL"], ic.levL)
    np.testing.assert_array_equal(F["levU"], ic.levU)
    assert F["nlevL"] == ic.nlevL and F["nlevU"] == ic.nlevU
    s.close()


def test_factor_bit_exact_full_size_100cubed(nle):
    A, st = load("diff3d7_100")
    s = solver(nle, A, "mixed")
    s.factor_ic(st["lfil"], st["tau_ic"])
    F = s.get_factor()
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    np.testing.assert_array_equal(F["Lcol"], ic.Lcol)
    np.testing.assert_array_equal(F["Lval"].view(np.uint64), ic.Lval.view(np.uint64))
    np.testing.assert_array_equal(F["levL"], ic.levL)
    np.testing.assert_array_equal(F["levU"], ic.levU)
    s.close()


# ---------------------------------------------------------------------------
# building blocks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["aniso2d_30x37", "hex27_16", "rgg3000"])
def test_shifted_spmv(nle, name, prec):
    A, st = load(name)
    s = solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    x = W.rng_for(5).standard_normal(A.n)
    theta = 0.37
    y = s.apply_shifted(theta, x).cpu().numpy()
    ref = O.spmv(A, x) - theta * x
    absA = W.CSR(A.n, A.rowptr, A.col, np.abs(A.val))
    scale = O.spmv(absA, np.abs(x)) + abs(theta) * np.abs(x)
    tol = 1e-14 if prec == "fp64" else 30 * EPS32
    assert np.all(np.abs(y - ref) <= tol * scale)
    s.close()


def _pairs_and_Q(A, k, m, seed):
    """k pairs with s^T r < 0 (as the Newton iteration produces) and m orthonormal columns."""
    rng = W.rng_for(seed)
    n = A.n
    Qm, _ = np.linalg.qr(rng.standard_normal((n, max(m, 1))))
    Q = Qm[:, :m].T.copy()
    S, R = [], []
    for _ in range(k):
        r = rng.standard_normal(n)
        sv = -(r / A.to_scipy().diagonal()) + 0.05 * rng.standard_normal(n)
        if sv @ r > 0:
            sv = -sv
        S.append(sv)
        R.append(r)
    return np.array(S).reshape(k, n), np.array(R).reshape(k, n), Q


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("k,m", [(0, 0), (0, 3), (1, 1), (3, 2), (5, 4), (9, 2), (10, 5)])
def test_apply_prec(nle, prec, k, m):
    A, st = load("diff3d7_24")
    s = solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    S, R, Q = _pairs_and_Q(A, k, m, seed=10 * k + m)
    g = W.rng_for(3).standard_normal(A.n)
    if m:
        g = g - Q.T @ (Q @ g)
    if prec == "mixed":
        # the library recomputes alpha from its rounded vectors: give the
        # oracle the same rounded inputs
        S = S.astype(np.float32).astype(np.float64)
        R = R.astype(np.float32).astype(np.float64)
    alpha = [float(S[t] @ R[t]) for t in range(k)]
    c = s.apply_prec(g, S if k else None, R if k else None, Q if m else None).cpu().numpy()
    ref = O.bfgs_apply(g, list(S), list(R), alpha, ic, Q.T if m else None)
    err = np.linalg.norm(c - ref) / np.linalg.norm(ref)
    assert err <= (1e-11 if prec == "fp64" else 1e-4), err
    s.close()


def _newton_state(A, j_conv, seed):
    import scipy.sparse.linalg as spl

    lam, V = spl.eigsh(A.to_scipy(), k=j_conv + 2, sigma=0, which="LM")
    order = np.argsort(lam)
    lam, V = lam[order], V[:, order]
    Qt = V[:, :j_conv]
    d = W.rng_for(seed).standard_normal(A.n)
    u = V[:, j_conv] + 0.02 * d / np.linalg.norm(d)
    u = u - Qt @ (Qt.T @ u)
    u /= np.linalg.norm(u)
    Au = O.spmv(A, u)
    theta = float(u @ Au)
    r = Au - theta * u
    return Qt, u, theta, r


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("k", [0, 3])
def test_pcg_fixed_iterations(nle, prec, k):
    """Exits (iii) and (iv) off, tau_PCG = 0: both sides run the same 12 iterations."""
    A, st = load("diff2d5_60x70")
    s = solver(nle, A, prec, exit_eigres=0, exit_stagnation=0, tau_pcg=0.0)
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    Qt, u, theta, r = _newton_state(A, 2, seed=4)
    Q = np.concatenate([Qt, u[:, None]], axis=1)
    S, R, _ = _pairs_and_Q(A, k, 0, seed=7)
    if prec == "mixed":
        S = S.astype(np.float32).astype(np.float64)
        R = R.astype(np.float32).astype(np.float64)
    alpha = [float(S[t] @ R[t]) for t in range(k)]
    sg, info = s.pcg(theta, 1e-8, 12, r, Q.T, S if k else None, R if k else None)
    sg = sg.cpu().numpy()
    opt = O.OracleOptions(tau_pcg=0.0, max_pcg=12, exit_eigres=False, exit_stagnation=False)
    sref, rinfo = O.pcg_correction(A, theta, u, r, Q, list(S), list(R), alpha, ic, opt)
    assert info["its"] == rinfo["its"] == 12 and info["exit"] == "maxit"
    err = np.linalg.norm(sg - sref) / np.linalg.norm(sref)
    assert err <= (1e-9 if prec == "fp64" else 2e-3), err
    assert abs(info["gnorm0"] - np.linalg.norm(r - Q @ (Q.T @ r))) <= 1e-6 * info["gnorm0"]
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_pcg_exits_match_oracle(nle, prec):
    """Default exits: the same exit reason and iteration count as the oracle."""
    A, st = load("diff3d7_24")
    s = solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    Qt, u, theta, r = _newton_state(A, 1, seed=9)
    Q = np.concatenate([Qt, u[:, None]], axis=1)
    sg, info = s.pcg(theta, 1e-8, 20, r, Q.T)
    opt = O.OracleOptions()
    sref, rinfo = O.pcg_correction(A, theta, u, r, Q, [], [], [], ic, opt)
    assert info["exit"] == rinfo["exit"]
    assert abs(info["its"] - rinfo["its"]) <= (0 if prec == "fp64" else 1)
    s.close()


# ---------------------------------------------------------------------------
# whole solves
# ---------------------------------------------------------------------------

def _check_solution(A, lam, V, tol):
    Asp = A.to_scipy()
    p = len(lam)
    for j in range(p):
        res = np.linalg.norm(Asp @ V[j] - lam[j] * V[j]) / lam[j]
        assert res <= 1.5 * tol, (j, res)
        i = int(np.argmax(np.abs(V[j])))
        assert V[j, i] > 0
    np.testing.assert_allclose(V @ V.T, np.eye(p), atol=1e-10)
    assert np.all(np.diff(lam) > 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["aniso2d_30x37", "diff3d7_24", "diff2d5_60x70", "rgg3000", "hex27_16"])
def test_solve_matches_oracle(nle, name, prec):
    A, st = load(name)
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, st["tol"], 100, 20, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"])
    lref, Vref, rstats = O.dacg_newton(A, p, X0, opt)
    rtol = 1e-10 if prec == "fp64" else 1e-8
    np.testing.assert_allclose(lam, lref, rtol=rtol)
    for j in range(p):
        assert sin_angle(V[j], Vref[:, j]) <= (1e-8 if st["tol"] <= 1e-10 else 1e-6)
    _check_solution(A, lam, V, st["tol"])
    assert all(stats["converged"]) and stats["ascending"]
    if name == "aniso2d_30x37":
        np.testing.assert_allclose(lam, W.laplacian_2d_aniso_eigs(30, 37, 1.0, 1.7)[:p], rtol=1e-10)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["diff3d7_24", "diff2d5_60x70", "rgg3000", "hex27_16"])
def test_multicolor_ordering_matches_oracle_on_permuted_matrix(nle, name, prec):
    """nle_options.ordering = NLE_ORDER_MULTICOLOR2: the library factors
    P A P^T with P from the greedy distance-2 colouring, the oracle runs the
    same method on workloads.permute(A, perm).  Factor and levels bit-exact;
    eigenvalues and eigenvectors (returned in the caller's numbering) against
    the oracle's, mapped back through perm."""
    A, st = load(name)
    perm, ncolors = W.multicolor_order(A, 2)
    B = W.permute(A, perm)
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, prec, ordering=nle.NLE_ORDER_MULTICOLOR2)
    s.factor_ic(st["lfil"], st["tau_ic"])
    F = s.get_factor()
    ic = O.ic_factor(B, st["lfil"], st["tau_ic"])
    np.testing.assert_array_equal(F["Lrowptr"], ic.Lrowptr)
    np.testing.assert_array_equal(F["Lcol"], ic.Lcol)
    np.testing.assert_array_equal(F["Lval"].view(np.uint64), ic.Lval.view(np.uint64))
    np.testing.assert_array_equal(F["levL"], ic.levL)
    assert F["nlevL"] == ic.nlevL
    lam, V, stats = s.solve(p, st["tol"], 100, 20, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    s.close()
    opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"])
    lref, Vref, _ = O.dacg_newton(B, p, X0[:, perm], opt, ic=ic)
    np.testing.assert_allclose(lam, lref, rtol=1e-10 if prec == "fp64" else 1e-8)
    for j in range(p):
        assert sin_angle(V[j][perm], Vref[:, j]) <= 1e-6
    _check_solution(A, lam, V, st["tol"])
    assert all(stats["converged"]) and stats["ascending"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["aniso2d_30x37", "diff3d7_24", "rgg3000"])
def test_full_bfgs_update_matches_oracle(nle, name, prec):
    """nle_options.bfgs_update = NLE_BFGS_FULL (Section 3, y_k = r_{k+1} -
    r_k) against the oracle run with the same update."""
    A, st = load(name)
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, prec, bfgs_update=nle.NLE_BFGS_FULL)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, st["tol"], 100, 20, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    s.close()
    opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"], bfgs_full=True)
    lref, Vref, rstats = O.dacg_newton(A, p, X0, opt)
    np.testing.assert_allclose(lam, lref, rtol=1e-10 if prec == "fp64" else 1e-8)
    for j in range(p):
        assert sin_angle(V[j], Vref[:, j]) <= (1e-8 if st["tol"] <= 1e-10 else 1e-6)
    _check_solution(A, lam, V, st["tol"])
    assert all(stats["converged"]) and stats["ascending"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kmax,update", [(10, "simplified"), (9, "full")])
def test_solve_largest_pair_rings(nle, kmax, update, prec):
    """The largest ring of stored pairs (k_max = NLE_MAX_KMAX) and, with the
    full BFGS update, the largest ring plus its staging slot (k_max =
    NLE_MAX_KMAX - 1), against the oracle run with the same k_max and
    update.  Two inner iterations per Newton step make every eigenpair take
    more than k_max outer steps, so the ring wraps around."""
    A, st = load("diff3d7_24")
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    full = update == "full"
    s = solver(nle, A, prec, k_max=kmax, bfgs_update=nle.NLE_BFGS_FULL if full else nle.NLE_BFGS_SIMPLIFIED)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, st["tol"], 100, 2, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    s.close()
    opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"], k_max=kmax, bfgs_full=full,
                          max_pcg=2)
    lref, Vref, rstats = O.dacg_newton(A, p, X0, opt)
    np.testing.assert_allclose(lam, lref, rtol=1e-10 if prec == "fp64" else 1e-8)
    for j in range(p):
        assert sin_angle(V[j], Vref[:, j]) <= 1e-6
    _check_solution(A, lam, V, st["tol"])
    assert max(rstats["outer_its"]) > kmax and max(stats["outer_its"]) > kmax


@pytest.mark.parametrize("prec", PRECS)
def test_solve_full_size_100cubed(nle, prec):
    """n = 1e6, p = 10, IC(10, 1e-3), tol 1e-8: eigenvalues against the stored
    oracle run, eigenvector samples, whole eigenvectors through their sketches
    (within the residual bound, and within 1e-6 wherever that bound is below
    1e-6), residuals and orthogonality at full size."""
    with open(os.path.join(HERE, "golden", "diff3d7_100.json")) as fh:
        gold = json.load(fh)
    A, st = load("diff3d7_100")
    p = gold["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, st["tol"], 100, 20, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    np.testing.assert_allclose(lam, gold["lam"], rtol=1e-10 if prec == "fp64" else 1e-8)
    idx = np.array(gold["sample_index"])
    for j in range(p):
        ref = np.array(gold["sample_V"][j])
        v = align(V[j, idx], ref)
        assert np.abs(v - ref).max() <= 2e-6
    ang, bnd = FC.check_eigenvectors(A, V, gold, stats["final_res"], f"diff3d7_100 {prec}")
    FC.check_clusters(A, V, gold, stats["final_res"], f"diff3d7_100 {prec}")
    # the stated eigenvector tolerance, 1e-6, wherever the residual bound
    # allows it
    assert np.all(ang[bnd <= 1e-6] <= 1e-6), ang
    _check_solution(A, lam, V, st["tol"])
    s.close()


def test_solve_full_size_hex27_96(nle):
    """n = 884,736 (27-point trilinear hex stiffness), p = 20, IC(20, 1e-4),
    mixed precision: eigenvalues against the stored oracle run; eigenvector
    samples within 10 tol lambda_j / gap_j (the eigenvector error allowed by
    the residual test ||A v - lambda v|| <= tol lambda, on either side) and
    whole eigenvectors through their sketches within the residual bound;
    residuals, orthogonality, order; the eigenvalue backward against the
    identity sum_e A_e d(sum lambda)/dA_e = sum lambda (Rayleigh quotients
    are homogeneous of degree 1 in the entries); and the backward carried to
    the element coefficients (the paper-scale case of a loss on element
    parameters) against the oracle's."""
    import torch

    with open(os.path.join(HERE, "golden", "hex27_96.json")) as fh:
        gold = json.load(fh)
    A, st = load("hex27_96")
    p = gold["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, "mixed")
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam_t, V_t, stats = s.solve(p, st["tol"], st["max_newton"], 20, X0)
    grad = s.backward(torch.ones(p, dtype=torch.float64), None).cpu().numpy()
    s.close()
    lam = lam_t.cpu().numpy()
    V = V_t.cpu().numpy()
    assert all(gold["oracle_stats"]["converged"])
    glam = np.array(gold["lam"])
    np.testing.assert_allclose(lam, glam, rtol=1e-8)
    gaps = np.minimum(np.diff(glam, prepend=-np.inf), np.diff(glam, append=np.inf))
    idx = np.array(gold["sample_index"])
    for j in range(p):
        ref = np.array(gold["sample_V"][j])
        v = align(V[j, idx], ref)
        assert np.abs(v - ref).max() <= 10 * st["tol"] * glam[j] / gaps[j], j
    ang, bnd = FC.check_eigenvectors(A, V, gold, stats["final_res"], "hex27_96 mixed")
    assert np.all(ang[bnd <= 1e-6] <= 1e-6), ang
    # the pairs of a tight cluster are individually ill conditioned; the
    # span of each cluster is not
    FC.check_clusters(A, V, gold, stats["final_res"], "hex27_96 mixed")
    _check_solution(A, lam, V, st["tol"])
    assert abs(float(A.val @ grad) - lam.sum()) <= 1e-9 * lam.sum()
    # the backward of sum lambda_j with respect to the element coefficients
    # (chain rule through the hex assembly): the oracle's at 64 elements, its
    # norm, and the Euler identity sum_e kappa_e dL/dkappa_e = sum lambda_j
    kt = torch.tensor(A.meta["kappa"], dtype=torch.float64, requires_grad=True)
    (gk,) = torch.autograd.grad(W.hex_poisson_values_torch(kt), kt, grad_outputs=torch.tensor(grad))
    gk = gk.numpy().ravel()
    elems = np.array(gold["grad_elems"])
    ref = np.array(gold["grad_kappa"])
    # the gradient of sum lambda_j is the trace of dA against the spectral
    # projector V V^T of all p pairs, which does not depend on how the pairs
    # of a cluster are rotated inside it: it is held to the stated gradient
    # tolerance, relative 1e-6 (the per-pair angle bounds, summed, would
    # allow 2 sum(bnd))
    gerr = np.linalg.norm(gk[elems] - ref) / np.linalg.norm(ref)
    print(f"element gradient: relative error {gerr:.2e} (per-pair bound {2 * float(np.sum(bnd)):.2e}), "
          f"norm {np.linalg.norm(gk):.6e} vs {gold['grad_kappa_norm']:.6e}")
    assert gerr <= 1e-6, gerr
    assert abs(np.linalg.norm(gk) - gold["grad_kappa_norm"]) <= 1e-6 * gold["grad_kappa_norm"]
    assert abs(float(A.meta["kappa"].ravel() @ gk) - lam.sum()) <= 1e-9 * lam.sum()


# ---------------------------------------------------------------------------
# edge cases and failure reporting
# ---------------------------------------------------------------------------

def test_default_start_and_host_buffers(nle):
    """X0 = NULL (the library's fixed pseudo-random starts) still finds the
    closed-form leftmost eigenvalues; the same solve through host buffers
    (buffers_on_device = 0) returns exactly the device-buffer results."""
    A, st = load("aniso2d_30x37")
    p = 3
    exact = W.laplacian_2d_aniso_eigs(30, 37, 1.0, 1.7)[:p]
    s = solver(nle, A, "fp64")
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, 1e-10, 100, 20, None)
    np.testing.assert_allclose(lam.cpu().numpy(), exact, rtol=1e-10)
    X0 = np.ascontiguousarray(W.start_vectors(A.n, p, st["seed"]))
    lam_d, V_d, _ = s.solve(p, 1e-10, 100, 20, X0)
    lam_h = np.zeros(p)
    V_h = np.zeros((p, A.n))
    stats_h = nle.nle_stats()
    rc = nle.nle_solve(s.h, p, 1e-10, 100, 20, nle._hptr(X0), nle._hptr(lam_h), nle._hptr(V_h), stats_h, 0)
    assert rc == nle.NLE_OK, nle.nle_last_error(s.h)
    np.testing.assert_array_equal(lam_h, lam_d.cpu().numpy())
    np.testing.assert_array_equal(V_h, V_d.cpu().numpy())
    s.close()


def test_p1_and_tiny_problem(nle):
    A = W.tridiag(7, 2.0, -1.0)
    s = solver(nle, A, "fp64")
    s.factor_ic(2, 0.0)
    lam, V, stats = s.solve(1, 1e-10, 50, 20, W.start_vectors(7, 1, 3))
    exact = 2 - 2 * math.cos(math.pi / 8)
    assert abs(lam.item() - exact) <= 1e-12
    s.close()


def test_state_and_argument_errors(nle):
    A, st = load("aniso2d_30x37")
    s = solver(nle, A, "fp64")
    with pytest.raises(nle.NLEError) as e:
        s.solve(2, 1e-8)
    assert e.value.code == 9
    s.factor_ic(5, 1e-2)
    with pytest.raises(nle.NLEError) as e:
        s.solve(A.n, 1e-8)
    assert e.value.code == 1
    s.close()


def test_ic_breakdown_reported(nle):
    """Indefinite matrix with positive diagonal: IC(0) exists, the complete
    factor meets a negative pivot in column 2 (worked by hand: w2 = -3.26)."""
    A = W.CSR(3, np.array([0, 3, 5, 7], np.int64), np.array([0, 1, 2, 0, 1, 0, 2], np.int32),
              np.array([1.0, 0.9, 0.9, 0.9, 1.0, 0.9, 1.0]))
    s = solver(nle, A, "fp64")
    s.factor_ic(0, 0.0)
    with pytest.raises(nle.NLEError) as e:
        s.factor_ic(3, 0.0)
    assert e.value.code == 3
    s.close()


def test_bounded_wait_reports_timeout_and_context_survives(nle):
    """A device wait limit far below any real wait makes the solve report
    NLE_ERR_TIMEOUT; the kernels return on their own and the same process
    then solves normally."""
    A, st = load("diff3d7_24")
    # the factor on the host: the device factor's own bounded wait is
    # tested in test_gpu_ict.py; here the solver's waits run out
    s = solver(nle, A, "mixed", spin_timeout_s=1e-9, ic_device=nle.NLE_IC_HOST)
    s.factor_ic(st["lfil"], st["tau_ic"])
    with pytest.raises(nle.NLEError) as e:
        s.solve(2, 1e-8, 100, 20, W.start_vectors(A.n, 2, 1))
    assert e.value.code == 8
    s.close()
    s = solver(nle, A, "mixed")
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(2, 1e-8, 100, 20, W.start_vectors(A.n, 2, 1))
    assert all(stats["converged"])
    s.close()
