"""nle_batch_solve: many grounded graph Laplacians of uneven size in one
persistent launch, against the single-problem solve and the oracle."""
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


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_matches_single_and_oracle(nle, prec):
    sizes = [2400, 5200, 3100, 7000, 2000, 4300]
    mats = [W.geometric_graph_laplacian(n, 900 + i) for i, n in enumerate(sizes)]
    p = 4
    opts = dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64, grid_ctas=4,
                trsv_schedule=nle.NLE_SCHED_LEVEL)
    solvers = []
    X0s = []
    for i, A in enumerate(mats):
        s = nle.Eigensolver(A, opts)
        s.factor_ic(30, 1e-2)
        solvers.append(s)
        X0s.append(W.start_vectors(A.n, p, 700 + i))
    st0 = solvers[0].last_stats()  # nothing solved yet: set-up fields only
    assert st0["p"] == 0 and st0["pcg_iterations"] == 0 and st0["trsv_schedule"] == "level"
    lams, Vs, per = nle.batch_solve(solvers, p, 1e-8, 100, 20, X0s)
    assert all(x == 0 for x in per), per
    for s in solvers:
        st = s.last_stats()
        assert st["p"] == p and all(st["converged"]) and st["ascending"]
        assert st["pcg_iterations"] > 0 and st["dacg_iterations"] > 0 and st["ms_batch"] > 0
        assert st["pcg_iterations"] == sum(st["pcg_its"])
    rtol = 1e-8 if prec == "mixed" else 1e-10
    for i, A in enumerate(mats):
        lam = lams[i].cpu().numpy()
        V = Vs[i].cpu().numpy()
        assert abs(lam[0] - 1e-3) <= 1e-3 * rtol * 10
        lref, Vref, _ = O.dacg_newton(A, p, X0s[i], O.OracleOptions(tol=1e-8, lfil=30, tau_ic=1e-2))
        np.testing.assert_allclose(lam, lref, rtol=rtol)
        Asp = A.to_scipy()
        for j in range(p):
            assert np.linalg.norm(Asp @ V[j] - lam[j] * V[j]) <= 1.5e-8 * lam[j]
        # the single-problem path gives the same eigenvalues
        l1, _, _ = solvers[i].solve(p, 1e-8, 100, 20, X0s[i])
        np.testing.assert_allclose(l1.cpu().numpy(), lam, rtol=rtol)
    for s in solvers:
        s.close()


def test_batch_rejects_wide_layout(nle):
    """A handle factored for more than 8 CTAs cannot join a batch (its slab
    layout is tied to its CTA count)."""
    B = W.geometric_graph_laplacian(40000, 6)  # 10,000 row groups: 20 CTAs wanted
    s = nle.Eigensolver(B, dict(precision=nle.NLE_MIXED, grid_ctas=16))
    s.factor_ic(30, 1e-2)
    with pytest.raises(nle.NLEError) as e:
        nle.batch_solve([s], 2, 1e-8)
    assert e.value.code == 1
    s.close()


def test_batch_groups_of_eight_fp64(nle):
    """A handle factored for 8 CTAs (FP64, n = 36,000) makes the batch run in
    groups of 8; every problem matches its single-problem solve, the
    smallest also the oracle."""
    sizes = [36000, 2600, 4100]
    mats = [W.geometric_graph_laplacian(n, 950 + i) for i, n in enumerate(sizes)]
    p = 3
    solvers, X0s = [], []
    for i, A in enumerate(mats):
        s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64, grid_ctas=8, trsv_schedule=nle.NLE_SCHED_LEVEL))
        s.factor_ic(30, 1e-2)
        solvers.append(s)
        X0s.append(W.start_vectors(A.n, p, 720 + i))
    lams, Vs, per = nle.batch_solve(solvers, p, 1e-8, 400, 20, X0s)
    assert all(x == 0 for x in per), per
    for i, A in enumerate(mats):
        lam = lams[i].cpu().numpy()
        l1, V1, _ = solvers[i].solve(p, 1e-8, 400, 20, X0s[i])
        np.testing.assert_allclose(lam, l1.cpu().numpy(), rtol=1e-10)
        Asp = A.to_scipy()
        V = Vs[i].cpu().numpy()
        for j in range(p):
            assert np.linalg.norm(Asp @ V[j] - lam[j] * V[j]) <= 1.5e-8 * lam[j]
    lref, _, _ = O.dacg_newton(mats[1], p, X0s[1], O.OracleOptions(tol=1e-8, lfil=30, tau_ic=1e-2, max_newton=400))
    np.testing.assert_allclose(lams[1].cpu().numpy(), lref, rtol=1e-10)
    for s in solvers:
        s.close()


def test_batch_on_non_blocking_stream(nle):
    """Handles created on a non-blocking stream (which does not wait for the
    legacy default stream): the set-up uploads, the batch's control words and
    the launch are all ordered on that stream, and the results equal the
    single-problem solves on the same stream."""
    import torch

    stream = torch.cuda.Stream()
    sizes = [3300, 2100, 4800]
    mats = [W.geometric_graph_laplacian(n, 960 + i) for i, n in enumerate(sizes)]
    p = 3
    with torch.cuda.stream(stream):
        solvers, X0s = [], []
        for i, A in enumerate(mats):
            s = nle.Eigensolver(A, dict(precision=nle.NLE_FP64, grid_ctas=4, trsv_schedule=nle.NLE_SCHED_LEVEL),
                                stream=stream)
            s.factor_ic(30, 1e-2)
            solvers.append(s)
            X0s.append(W.start_vectors(A.n, p, 740 + i))
        lams, Vs, per = nle.batch_solve(solvers, p, 1e-8, 400, 20, X0s)
        assert all(x == 0 for x in per), per
        for i, A in enumerate(mats):
            l1, _, _ = solvers[i].solve(p, 1e-8, 400, 20, X0s[i])
            np.testing.assert_allclose(lams[i].cpu().numpy(), l1.cpu().numpy(), rtol=1e-10)
            assert abs(lams[i][0].item() - 1e-3) <= 1e-12
    stream.synchronize()
    for s in solvers:
        s.close()


def test_batch_bounded_wait_reports_timeout_and_context_survives(nle):
    """A wait limit far below any real wait makes every problem of the batch
    report NLE_ERR_TIMEOUT (problem barriers and the group barriers are all
    bounded); the kernel returns on its own and the next batch in the same
    process solves normally."""
    mats = [W.geometric_graph_laplacian(n, 970 + i) for i, n in enumerate([2500, 3500])]
    p = 2
    X0s = [W.start_vectors(A.n, p, 760 + i) for i, A in enumerate(mats)]
    bad = []
    for A in mats:
        # factor on the host (the device factor's own bounded wait is tested
        # in test_gpu_ict.py)
        s = nle.Eigensolver(A, dict(precision=nle.NLE_MIXED, grid_ctas=4, spin_timeout_s=1e-9,
                                    trsv_schedule=nle.NLE_SCHED_LEVEL, ic_device=nle.NLE_IC_HOST))
        s.factor_ic(30, 1e-2)
        bad.append(s)
    with pytest.raises(nle.NLEError) as e:
        nle.batch_solve(bad, p, 1e-8, 100, 20, X0s)
    assert e.value.code == nle.NLE_ERR_TIMEOUT
    for s in bad:
        s.close()
    good = []
    for A in mats:
        s = nle.Eigensolver(A, dict(precision=nle.NLE_MIXED, grid_ctas=4, trsv_schedule=nle.NLE_SCHED_LEVEL))
        s.factor_ic(30, 1e-2)
        good.append(s)
    lams, Vs, per = nle.batch_solve(good, p, 1e-8, 100, 20, X0s)
    assert all(x == 0 for x in per), per
    for s in good:
        s.close()


def _gold(name):
    import json
    import os

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"{name}.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_failures_are_the_oracles(nle, prec):
    """Problems 63 and 232 of the 256-graph batched workload do not converge
    within 400 Newton steps on the oracle (stored runs, tests/golden): the
    Newton iteration of eigenpair 2 settles between lambda_2 and lambda_3
    (0.2 % apart) from the DACG start, and eigenpairs 3-4, deflated against
    that vector, fail too.  The batched library, with the same start
    vectors, reports NLE_ERR_NOCONV for both, for the same eigenpairs; in
    FP64 with the oracle's final residual of eigenpair 2 to 1e-3 relative
    and its converged eigenvalue to 1e-10, in mixed precision without
    failing anywhere the oracle converges."""
    probs = (63, 232)
    golds = [_gold(f"graph_batch_{b}") for b in probs]
    mats = [W.graph_batch_problem(b) for b in probs]
    X0s = [W.graph_batch_start(A, b, 4) for A, b in zip(mats, probs)]
    opts = dict(precision=nle.NLE_FP64 if prec == "fp64" else nle.NLE_MIXED, grid_ctas=8 if prec == "fp64" else 4,
                trsv_schedule=nle.NLE_SCHED_LEVEL)
    solvers = []
    for A in mats:
        s = nle.Eigensolver(A, opts)
        s.factor_ic(30, 1e-2)
        solvers.append(s)
    lams, Vs, per = nle.batch_solve(solvers, 4, 1e-8, 400, 20, X0s)
    assert per == [nle.NLE_ERR_NOCONV, nle.NLE_ERR_NOCONV], per
    for s, g, lam in zip(solvers, golds, lams):
        st = s.last_stats()
        conv_or = g["oracle_stats"]["converged"]
        assert not all(conv_or)
        lam = lam.cpu().numpy()
        if prec == "fp64":
            assert st["converged"] == conv_or
            first = conv_or.index(False)
            for j, c in enumerate(conv_or):
                if c:
                    assert abs(lam[j] - g["lam"][j]) <= 1e-10 * g["lam"][j]
            # the first failing eigenpair follows the oracle's path; the
            # later ones are deflated against its unconverged vector
            ref = g["oracle_stats"]["final_res"][first]
            assert abs(st["final_res"][first] - ref) <= 1e-3 * ref, (first, st["final_res"][first], ref)
        else:
            assert all(c or not co for c, co in zip(st["converged"], conv_or)), (st["converged"], conv_or)
    for s in solvers:
        s.close()
