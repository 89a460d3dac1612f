"""nle_backward (through the C ABI) against the oracle's adjoint, the closed
form d lambda / d a, and the autograd wrapper."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "mixed"]


@pytest.fixture(scope="module")
def nle():
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    nle.load_library()
    return nle


def _solver(nle, A, prec):
    return nle.Eigensolver(A, dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64))


@pytest.mark.parametrize("prec", PRECS)
def test_backward_matches_oracle_adjoint(nle, prec):
    """Loss of the 2D diffusion workload: sum lambda_j + sum_i w_i (v_1)_i^2."""
    A, st = W.workload("diff2d5_60x70")
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = _solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, 1e-10, 100, 20, X0)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    w = A.meta["w"]
    gl = np.ones(p)
    gV = np.zeros((p, A.n))
    gV[0] = 2 * w * V[0]
    grad = s.backward(gl, gV).cpu().numpy()
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    lref, Vref, _ = O.dacg_newton(A, p, X0, O.OracleOptions(tol=1e-10, lfil=st["lfil"], tau_ic=st["tau_ic"]), ic=ic)
    gVref = np.zeros((A.n, p))
    gVref[:, 0] = 2 * w * Vref[:, 0]
    ref = O.adjoint_grad(A, lref, Vref, gl, gVref, ic)
    err = np.linalg.norm(grad - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err
    s.close()


@pytest.mark.parametrize("prec", PRECS)
def test_backward_with_multicolour_ordering(nle, prec):
    """The gradient does not depend on the preconditioner: with the
    distance-2 multicolour ordering (factor of P A P^T, device order through
    P) nle_backward still returns dL/dA per stored entry of A in the
    caller's numbering, equal to the oracle's adjoint on A itself."""
    A, st = W.workload("diff2d5_60x70")
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = nle.Eigensolver(A, dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64,
                                ordering=nle.NLE_ORDER_MULTICOLOR2))
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, 1e-10, 100, 20, X0)
    V = V.cpu().numpy()
    w = A.meta["w"]
    gl = np.ones(p)
    gV = np.zeros((p, A.n))
    gV[0] = 2 * w * V[0]
    grad = s.backward(gl, gV).cpu().numpy()
    s.close()
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    lref, Vref, _ = O.dacg_newton(A, p, X0, O.OracleOptions(tol=1e-10, lfil=st["lfil"], tau_ic=st["tau_ic"]), ic=ic)
    gVref = np.zeros((A.n, p))
    gVref[:, 0] = 2 * w * Vref[:, 0]
    ref = O.adjoint_grad(A, lref, Vref, gl, gVref, ic)
    err = np.linalg.norm(grad - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err


@pytest.mark.parametrize("prec", PRECS)
def test_backward_eigenvalue_closed_form(nle, prec):
    """d lambda_{k,l}/d a = 2 - 2 cos(k pi/(nx+1)) for the anisotropic Laplacian (a = 1, b = 1.7)."""
    nx, ny = 30, 37
    A, st = W.workload("aniso2d_30x37")
    s = _solver(nle, A, prec)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, _ = s.solve(5, 1e-10, 100, 20, W.start_vectors(A.n, 5, st["seed"]))
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dA = np.where(rows == A.col, 2.0, np.where(np.abs(rows - A.col) == 1, -1.0, 0.0))
    kl = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 1)]
    for j, (k, l) in enumerate(kl):
        gl = np.zeros(5)
        gl[j] = 1.0
        grad = s.backward(gl, None).cpu().numpy()
        assert abs(grad @ dA - (2 - 2 * math.cos(k * math.pi / (nx + 1)))) <= 1e-9
    s.close()


def test_autograd_function_matches_backward(nle):
    import torch

    A, st = W.workload("diff3d7_24")
    p = 3
    X0 = W.start_vectors(A.n, p, st["seed"])
    vals = torch.tensor(A.val, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(W.rng_for(8).random(A.n), dtype=torch.float64, device="cuda")
    lam, V = nle.eigsh(vals, A.rowptr, A.col, p, 1e-10, st["lfil"], st["tau_ic"], dict(precision=nle.NLE_FP64), X0)
    loss = lam.sum() + (w * V[1] ** 2).sum()
    (g,) = torch.autograd.grad(loss, vals)
    s = _solver(nle, A, "fp64")
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam2, V2, _ = s.solve(p, 1e-10, 100, 20, X0)
    gV = torch.zeros((p, A.n), dtype=torch.float64, device="cuda")
    gV[1] = 2 * w * V2[1]
    g2 = s.backward(torch.ones(p, dtype=torch.float64), gV)
    assert torch.linalg.norm(g - g2) <= 1e-8 * torch.linalg.norm(g2)
    s.close()


def test_backward_requires_solve(nle):
    A, st = W.workload("aniso2d_30x37")
    s = _solver(nle, A, "fp64")
    s.factor_ic(5, 1e-2)
    with pytest.raises(nle.NLEError) as e:
        s.backward(np.ones(2), None)
    assert e.value.code == 9
    s.close()
