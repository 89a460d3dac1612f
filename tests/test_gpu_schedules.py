"""The schedules of the triangular solves (nle_options.trsv_schedule, and
the rows per warp step of the level schedule, nle_options.trsv_rows) and the
autotuner that picks between them, against the oracle.

Both schedules apply the same (L L^T)^{-1} of Section 2 (only the order in
which warps take the rows differs), so each is held to the oracle's P0hat
and to the oracle's whole solve at the parity tolerances of
test_gpu_parity.py; the chain schedule is also run on matrices whose rows do
not form chains (a random geometric graph) and whose grid lines are not a
multiple of the task size (30 x 37)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.solver import p0hat

pytestmark = pytest.mark.gpu
PRECS = ["fp64", "mixed"]
SCHEDS = ["level", "level2", "chain"]
NAMES = ["aniso2d_30x37", "diff3d7_24", "diff2d5_60x70", "hex27_16", "rgg3000"]


@pytest.fixture(scope="module")
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


def solver(nle, A, prec, sched, **opts):
    """sched: auto, level (4 rows per warp step), level2 (2 rows), chain."""
    o = dict(precision=nle.NLE_MIXED if prec == "mixed" else nle.NLE_FP64,
             trsv_schedule={"auto": nle.NLE_SCHED_AUTO, "level": nle.NLE_SCHED_LEVEL, "level2": nle.NLE_SCHED_LEVEL,
                            "chain": nle.NLE_SCHED_CHAIN}[sched])
    if sched == "level2":
        o["trsv_rows"] = 2
    o.update(opts)
    return nle.Eigensolver(A, o)


def sin_angle(a, b):
    a = a / np.linalg.norm(a)
    b = b / np.linalg.norm(b)
    return float(np.linalg.norm(a - (a @ b) * b))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("name", NAMES)
def test_ic_application_matches_oracle(nle, name, sched, prec):
    """c = (L L^T)^{-1} g (k = 0 pairs, no projection) on two right-hand
    sides in a row, against the oracle's forward and backward substitution."""
    A, st = load(name)
    s = solver(nle, A, prec, sched)
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    for seed in (3, 4):
        g = W.rng_for(seed).standard_normal(A.n)
        c = s.apply_prec(g).cpu().numpy()
        ref = p0hat(ic, g)
        err = np.linalg.norm(c - ref) / np.linalg.norm(ref)
        assert err <= (1e-11 if prec == "fp64" else 1e-4), (seed, err)
    s.close()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("name", NAMES)
def test_solve_matches_oracle_with_schedule(nle, name, sched, prec):
    A, st = load(name)
    p = st["p"]
    X0 = W.start_vectors(A.n, p, st["seed"])
    s = solver(nle, A, prec, sched)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(p, st["tol"], 100, 20, X0)
    s.close()
    assert stats["trsv_schedule"] == ("level" if sched == "level2" else sched)
    if sched != "chain":
        assert stats["trsv_rows"] == (2 if sched == "level2" else 4)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy()
    lref, Vref, _ = O.dacg_newton(A, p, X0, O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"]))
    np.testing.assert_allclose(lam, lref, rtol=1e-10 if prec == "fp64" else 1e-8)
    for j in range(p):
        assert sin_angle(V[j], Vref[:, j]) <= (1e-8 if st["tol"] <= 1e-10 else 1e-6)
    assert all(stats["converged"]) and stats["ascending"]


def test_autotuner_times_both_and_keeps_the_faster(nle):
    """NLE_SCHED_AUTO: nle_factor_ic times one application with each schedule
    and keeps the faster; the statistics report both timings and the
    choice.  Under a multicolour ordering only the level schedule applies."""
    A, st = load("diff3d7_24")
    s = solver(nle, A, "mixed", "auto")
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(2, 1e-8, 100, 20, W.start_vectors(A.n, 2, 1))
    s.close()
    t = stats["tune_ms"]
    assert t["level"] > 0 and t["chain"] > 0 and t["level2"] > 0
    best = min(t, key=t.get)
    assert stats["trsv_schedule"] == ("chain" if best == "chain" else "level")
    if best != "chain":
        assert stats["trsv_rows"] == (2 if best == "level2" else 4)
    assert all(stats["converged"])
    s = solver(nle, A, "mixed", "auto", ordering=nle.NLE_ORDER_MULTICOLOR1)
    s.factor_ic(st["lfil"], st["tau_ic"])
    lam, V, stats = s.solve(2, 1e-8, 100, 20, W.start_vectors(A.n, 2, 1))
    s.close()
    assert stats["trsv_schedule"] == "level" and stats["tune_ms"]["chain"] == 0 and stats["tune_ms"]["level2"] > 0
    with pytest.raises(nle.NLEError) as e:
        s = solver(nle, A, "mixed", "chain", ordering=nle.NLE_ORDER_MULTICOLOR1)
        s.factor_ic(st["lfil"], st["tau_ic"])
    assert e.value.code == nle.NLE_ERR_ARG


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sched", SCHEDS)
def test_fewer_solve_warps(nle, sched, prec):
    """trsv_warps = 3: the task lists (chain) or the group rotation (level)
    are built for three warps per CTA; same P0hat as the oracle."""
    A, st = load("hex27_16")
    s = solver(nle, A, prec, sched, trsv_warps=3)
    s.factor_ic(st["lfil"], st["tau_ic"])
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    g = W.rng_for(8).standard_normal(A.n)
    c = s.apply_prec(g).cpu().numpy()
    ref = p0hat(ic, g)
    assert np.linalg.norm(c - ref) / np.linalg.norm(ref) <= (1e-11 if prec == "fp64" else 1e-4)
    s.close()
