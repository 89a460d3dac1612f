"""The condition-number study of the BFGS-updated preconditioner (the
analogue of the paper's study of P_k J_k, Section 5) run through the
library: P_k = Algorithm 3.1 applied by nle_apply_prec (C ABI) to a basis of
the complement of u_k, along the Newton steps of the first eigenpair of the
30 x 37 anisotropic Laplacian with k_max = 10.  The spectrum of P_k J_k on
u_k's complement (dense eigenvalues, n = 1110) must match the oracle's
(Algorithm 3.1 in numpy on the same pairs), and show the paper's effect:
every stored pair raises the smallest eigenvalue, the largest stays, the
condition number falls."""
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


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_condition_study_through_the_library(nle, prec):
    A, st = W.workload("aniso2d_30x37")
    n = A.n
    Ad = A.to_scipy().toarray()
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    s = nle.Eigensolver(A, dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64))
    s.factor_ic(st["lfil"], st["tau_ic"])
    x0 = W.start_vectors(n, 1, st["seed"])[0]
    opt = O.OracleOptions(tol=1e-12, lfil=st["lfil"], tau_ic=st["tau_ic"], k_max=10)
    u, _, _ = O.solver.dacg(A, x0, np.zeros((n, 0)), ic, 1e-2, 5000)
    u = u / np.linalg.norm(u)
    theta = u @ Ad @ u
    r = Ad @ u - theta * u
    S, R = [], []
    lib, ora = [], []
    for step in range(5):
        Z = np.linalg.qr(np.concatenate([u[:, None], np.eye(n)], axis=1))[0][:, 1:n]
        K = Z.T @ (Ad - theta * np.eye(n)) @ Z
        Sr, Rr = np.array(S).reshape(-1, n), np.array(R).reshape(-1, n)
        if prec == "mixed":
            # the library keeps the pairs in FP32 and recomputes alpha from them
            Sr = Sr.astype(np.float32).astype(np.float64)
            Rr = Rr.astype(np.float32).astype(np.float64)
        al = [float(a @ b) for a, b in zip(Sr, Rr)]
        k = len(S)
        PZ = np.stack([s.apply_prec(Z[:, i], Sr if k else None, Rr if k else None, u[None, :]).cpu().numpy()
                       for i in range(n - 1)], axis=1)
        PZo = np.stack([O.bfgs_apply(Z[:, i], list(Sr), list(Rr), al, ic, u[:, None]) for i in range(n - 1)], axis=1)
        for M, out in ((Z.T @ PZ, lib), (Z.T @ PZo, ora)):
            ev = np.sort(np.linalg.eigvals(M @ K).real)
            out.append((k, ev[0], ev[-1], ev[-1] / ev[0]))
        sv, _ = O.solver.pcg_correction(A, theta, u, r, u[:, None], S, R, [a @ b for a, b in zip(S, R)], ic, opt)
        if sv @ r < 0:
            S.append(sv)
            R.append(r)
        t = u + sv
        u = t / np.linalg.norm(t)
        theta = u @ Ad @ u
        r = Ad @ u - theta * u
    s.close()
    tol = 1e-9 if prec == "fp64" else 1e-4
    print("\nstep  pairs  lambda_min (library / oracle)  lambda_max  condition")
    for (k, a0, a1, c), (_, b0, b1, d) in zip(lib, ora):
        print(f"  {k}    {a0:.6f} / {b0:.6f}    {a1:.6f} / {b1:.6f}   {c:.3f} / {d:.3f}")
        assert abs(a0 - b0) <= tol * b0 and abs(a1 - b1) <= tol * b1 and abs(c - d) <= 2 * tol * d
    lmin = [x[1] for x in lib]
    assert [x[0] for x in lib] == [0, 1, 2, 3, 4]
    assert all(lmin[i + 1] >= lmin[i] * (1 - 1e-6) for i in range(4))
    assert lmin[-1] > 1.5 * lmin[0]
    assert lib[-1][3] < 0.6 * lib[0][3]
