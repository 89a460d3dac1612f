"""Gradients with respect to the coefficients of the assembly, through
nle_backward (C ABI) and the chain rule of the assembly (torch):
  2D diffusion, cell coefficients: loss = sum_j lambda_j + sum_i w_i (v_1)_i^2,
  w ~ U[0,1] seeded;
  27-point hex stiffness, element coefficients: loss = sum_j lambda_j."""
import json
import os

import numpy as np
import pytest

import fullsize_checks as FC
import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def nle():
    from paper_1312_1553_gb300 import _build, nle

    _build.build()
    nle.load_library()
    return nle


def _solve_and_kappa_grad(nle, A, kappa, p, st, prec, tol, X0):
    """Returns (loss, dloss/dkappa, d(sum lambda)/dkappa, lambda, stats, V);
    the gradients are flattened over the cells."""
    import torch

    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    vals = W.diffusion_2d_values_torch(kt)
    B = W.CSR(A.n, A.rowptr, A.col, vals.detach().numpy())
    s = nle.Eigensolver(B, dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64))
    try:
        s.factor_ic(st["lfil"], st["tau_ic"])
        lam, V, stats = s.solve(p, tol, 200, 20, X0)
        w = torch.tensor(A.meta["w"], dtype=torch.float64, device=V.device)
        loss = float(lam.sum() + (w * V[0] ** 2).sum())
        gV = torch.zeros_like(V)
        gV[0] = 2 * w * V[0]
        gA = s.backward(torch.ones(p, dtype=torch.float64), gV).cpu()
        gA_lam = s.backward(torch.ones(p, dtype=torch.float64), None).cpu()
    finally:
        s.close()
    (gk,) = torch.autograd.grad(vals, kt, grad_outputs=gA, retain_graph=True)
    (gk_lam,) = torch.autograd.grad(vals, kt, grad_outputs=gA_lam)
    return loss, gk.numpy().ravel(), gk_lam.numpy().ravel(), lam.cpu().numpy(), stats, V.cpu().numpy()


def test_kappa_gradient_central_differences_64_coefficients(nle):
    """Reduced size of the same recipe (60 x 70 cells): the adjoint gradient
    against central differences of FP64 solves at 64 seeded coefficients,
    and the Euler identity sum_c kappa_c d(sum lambda)/dkappa_c = sum_j
    lambda_j of the degree-1 homogeneous assembly (it holds for the Rayleigh
    quotients of any unit vectors, so only rounding enters)."""
    A, st = W.workload("diff2d5_60x70")
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    kappa = A.meta["kappa"]
    tol = 1e-10
    _, gk, gk_lam, lam, _, _ = _solve_and_kappa_grad(nle, A, kappa, p, st, "fp64", tol, X0)
    assert abs(float((kappa.ravel() * gk_lam).sum()) - lam.sum()) <= 1e-10 * lam.sum()
    cells = W.rng_for(99).choice(A.n, size=64, replace=False)
    errs = []
    for c in cells:
        h = 1e-3 * kappa.flat[c]
        kp = kappa.copy()
        kp.flat[c] += h
        km = kappa.copy()
        km.flat[c] -= h
        Lp = _solve_and_kappa_grad(nle, A, kp, p, st, "fp64", tol, X0)[0]
        Lm = _solve_and_kappa_grad(nle, A, km, p, st, "fp64", tol, X0)[0]
        errs.append(abs((Lp - Lm) / (2 * h) - gk[c]))
    scale = np.abs(gk[cells]).max()
    # step h = 1e-3 kappa_c: truncation about 1e-7 of the scale; the solve
    # error (residual 1e-10 theta) over 2h about 1e-6 of it
    assert max(errs) <= 1e-5 * scale, (max(errs), scale)


def test_full_size_600x700_eigenpairs_and_gradient(nle):
    """n = 420,000, p = 8, mixed precision: eigenvalues against the stored
    oracle run, whole eigenvectors through their sketches within the residual
    bound, the cell-coefficient gradient against the oracle's FP64 adjoint at
    64 cells, and the Euler identity over all 420,000 cells.

    Tolerance of the gradient: each side's eigenvector v_j is off by about
    tol * lambda_j / gap_j (residual test ||A v - lambda v|| <= tol lambda),
    and the gradient is linear in each v_j; ten times the largest such
    figure bounds the difference of the two sides."""
    with open(os.path.join(HERE, "golden", "diff2d5_600x700.json")) as fh:
        gold = json.load(fh)
    assert "grad_kappa" in gold, "golden file lacks the gradient sample"
    A, st = W.workload("diff2d5_600x700")
    p = gold["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    loss, gk, gk_lam, lam, stats, V = _solve_and_kappa_grad(nle, A, A.meta["kappa"], p, st, "mixed", st["tol"], X0)
    glam = np.array(gold["lam"])
    np.testing.assert_allclose(lam, glam, rtol=1e-8)
    ang, bnd = FC.check_eigenvectors(A, V, gold, stats["final_res"], "diff2d5_600x700 mixed")
    assert np.all(ang[bnd <= 1e-6] <= 1e-6), ang
    gaps = np.minimum(np.diff(glam, prepend=-np.inf)[:], np.diff(glam, append=np.inf))
    bound = 10 * st["tol"] * float(np.max(glam / gaps))
    assert abs(loss - gold["loss"]) <= bound * abs(gold["loss"]), (loss, gold["loss"], bound)
    cells = np.array(gold["grad_cells"])
    ref = np.array(gold["grad_kappa"])
    err = np.linalg.norm(gk[cells] - ref) / np.linalg.norm(ref)
    assert err <= bound, (err, bound)
    assert abs(np.linalg.norm(gk) - gold["grad_kappa_norm"]) <= bound * gold["grad_kappa_norm"]
    assert abs(float((A.meta["kappa"].ravel() * gk_lam).sum()) - lam.sum()) <= 1e-10 * lam.sum()


def _hex_sum_lambda_grad(nle, kappa, p, st, tol, X0):
    """(sum lambda_j, d(sum lambda)/dkappa_e flattened, lambda) for the hex
    stiffness with element coefficients kappa, FP64 solve."""
    import torch

    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    vals = W.hex_poisson_values_torch(kt)
    A = W.hex_poisson_from_kappa(kappa)
    s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64))
    try:
        s.factor_ic(st["lfil"], st["tau_ic"])
        lam, V, stats = s.solve(p, tol, 400, 20, X0)
        gA = s.backward(torch.ones(p, dtype=torch.float64), None).cpu()
    finally:
        s.close()
    (gk,) = torch.autograd.grad(vals, kt, grad_outputs=gA)
    lam = lam.cpu().numpy()
    return float(lam.sum()), gk.numpy().ravel(), lam


def test_hex_element_gradient_central_differences(nle):
    """Reduced size of the 27-point recipe (16^3 nodes, 17^3 elements): the
    gradient of sum lambda_j with respect to the element coefficients
    (nle_backward, then the chain rule through the hex assembly) against
    central differences of FP64 solves at 12 seeded elements, and the Euler
    identity.  Step h = 1e-4 kappa_e: truncation about 1e-8 of the scale;
    eigenvalues of the solves are exact to far below that (tolerance 1e-11,
    Rayleigh quotients err by the residual squared over the gap)."""
    A, st = W.workload("hex27_16")
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    kappa = A.meta["kappa"]
    tol = 1e-11
    L0, gk, lam = _hex_sum_lambda_grad(nle, kappa, p, st, tol, X0)
    assert abs(float(kappa.ravel() @ gk) - lam.sum()) <= 1e-10 * lam.sum()
    elems = W.rng_for(77).choice(kappa.size, size=12, replace=False)
    scale = np.abs(gk).max()
    for e in elems:
        h = 1e-4 * kappa.flat[e]
        kp = kappa.copy()
        kp.flat[e] += h
        km = kappa.copy()
        km.flat[e] -= h
        fd = (_hex_sum_lambda_grad(nle, kp, p, st, tol, X0)[0] - _hex_sum_lambda_grad(nle, km, p, st, tol, X0)[0]) / (2 * h)
        assert abs(fd - gk[e]) <= 1e-6 * scale, (e, fd, gk[e], scale)
