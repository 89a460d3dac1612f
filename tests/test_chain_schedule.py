"""Host logic of the schedules of the triangular solves (CPU, no GPU).

The library's own set-up code (nle_setup.cpp: IC factor + build_chain) is
compiled here with g++ through a small shim and its output executed by a
plain sequential simulation of the kernel's rules (trsv_chain): warps take
their tasks in order; a task may run once every external entry it reads is
computed; entries stored as register markers (col = -2 - d) are resolved
from the current task and the warp's previous task's last row.  Checked:
every row is solved exactly once, the simulation never stalls (the
topological dealing of strands), and the result equals a triangular solve
with scipy on the same factor.  A planted mistake in the marker distance is
caught."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
ROWS = 4  # TRSV_ROWS
NWARP = 16


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = tmp_path_factory.mktemp("shim") / "libchainshim.so"
    src = [os.path.join(HERE, "chain_shim.cpp"), os.path.join(ROOT, "paper_1312_1553_gb300", "csrc", "nle_setup.cpp")]
    inc = [f"-I{d}" for d in ("/usr/local/cuda/include", os.path.join(ROOT, "include"))]
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", *inc, *src, "-o", str(out)],
                   check=True)
    lib = ctypes.CDLL(str(out))
    lib.shim_factor.restype = ctypes.c_int
    lib.shim_factor.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                ctypes.c_double]
    lib.shim_chain.restype = ctypes.c_int64
    lib.shim_chain.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)]
    lib.shim_chain_get.restype = None
    lib.shim_chain_get.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7
    lib.shim_level.restype = ctypes.c_int64
    lib.shim_level.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64)]
    lib.shim_level_get.restype = None
    lib.shim_level_get.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 7
    return lib


def schedule(lib, A, lfil, tau, bsize, nwarps, lower):
    rp = np.ascontiguousarray(A.rowptr, np.int64)
    ci = np.ascontiguousarray(A.col, np.int32)
    va = np.ascontiguousarray(A.val, np.float64)
    assert lib.shim_factor(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, lfil, tau) == 0
    nent, nslab = ctypes.c_int64(), ctypes.c_int64()
    ntask = lib.shim_chain(1 if lower else 0, bsize, nwarps, ctypes.byref(nent), ctypes.byref(nslab))
    ns = nslab.value
    off = np.zeros(ns + 1, np.int64)
    width = np.zeros(ns, np.int32)
    col = np.zeros(nent.value, np.int32)
    val = np.zeros(nent.value)
    wptr = np.zeros(ns * (NWARP + 1), np.int32)
    task = np.zeros(2 * ntask, np.int32)
    diag = np.zeros(A.n)
    lib.shim_chain_get(1 if lower else 0, off.ctypes.data, width.ctypes.data, col.ctypes.data, val.ctypes.data,
                       wptr.ctypes.data, task.ctypes.data, diag.ctypes.data)
    return dict(off=off, width=width, col=col, val=val, wptr=wptr, task=task.reshape(-1, 2), diag=diag, ns=ns)


def simulate(S, n, npad, bsize, rhs, lower, plant=None):
    """Run the schedule as the kernel would, one ready task at a time."""
    x = np.full(npad, np.nan)
    done = np.zeros(npad, bool)
    solved = np.zeros(npad, np.int64)
    queues = []
    for s in range(S["ns"]):
        for w in range(NWARP):
            t0, t1 = S["wptr"][s * (NWARP + 1) + w], S["wptr"][s * (NWARP + 1) + w + 1]
            queues.append(dict(s=s, tasks=list(range(t0, t1)), pos=0, xprev=0.0))
    b = np.zeros(npad)
    b[:n] = rhs
    while True:
        progress = False
        for qd in queues:
            while qd["pos"] < len(qd["tasks"]):
                r0, meta = S["task"][qd["tasks"][qd["pos"]]]
                cnt = meta & 7
                s = qd["s"]
                b0 = s * bsize
                wd = S["width"][s]
                rows = [r0 + a if lower else r0 - a for a in range(cnt)]
                ready = True
                for r in rows:
                    e = S["off"][s] + (r - b0) * wd
                    for k in range(wd):
                        c = S["col"][e + k]
                        if c >= 0 and not done[c]:
                            ready = False
                if not ready:
                    break
                xs = []
                for a, r in enumerate(rows):
                    e = S["off"][s] + (r - b0) * wd
                    v = b[r]
                    for k in range(wd):
                        c, av = S["col"][e + k], S["val"][e + k]
                        if c >= 0:
                            v -= av * x[c]
                        elif c <= -2:
                            d = -2 - c
                            if plant == "distance":
                                d = d + 1 if d < a + 1 else d
                            src = a - d
                            assert -1 <= src < a, (r, d, a)
                            v -= av * (qd["xprev"] if src == -1 else xs[src])
                    xs.append(v / S["diag"][r] if r < n else v)
                for r, v in zip(rows, xs):
                    x[r] = v
                    done[r] = True
                    solved[r] += 1
                qd["xprev"] = xs[-1]
                qd["pos"] += 1
                progress = True
        if not progress:
            break
    return x, solved, all(qd["pos"] == len(qd["tasks"]) for qd in queues)


CASES = [("aniso2d_30x37", 5, 1e-2), ("diff3d7_24", 10, 1e-3), ("hex27_16", 20, 1e-4), ("rgg3000", 30, 1e-2)]


@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("name,lfil,tau", CASES)
def test_chain_schedule_solves_and_never_stalls(shim, name, lfil, tau, lower):
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve_triangular

    A, _ = W.workload(name)
    n = A.n
    npad = (n + 127) // 128 * 128
    grid = 8
    bsize = (npad + ROWS * grid - 1) // (ROWS * grid) * ROWS
    S = schedule(shim, A, lfil, tau, bsize, NWARP, lower)
    rhs = W.rng_for(12).standard_normal(n)
    x, solved, complete = simulate(S, n, npad, bsize, rhs, lower)
    assert complete, "the schedule stalled"
    assert np.all(solved == 1)
    # reference: the same factor through the oracle's C code
    import oracle as O

    ic = O.ic_factor(A, lfil, tau)
    L = sp.csr_matrix((ic.Lval, ic.Lcol, ic.Lrowptr), shape=(n, n))
    ref = spsolve_triangular(L, rhs, lower=True) if lower else spsolve_triangular(L.T.tocsr(), rhs, lower=False)
    np.testing.assert_allclose(x[:n], ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
    assert np.all(x[n:] == 0)


def test_chain_schedule_strands_follow_grid_lines(shim):
    """On the 7-point 24^3 grid in natural order every row but the first of
    each x-line depends on its predecessor: the strands of a slab are its
    x-lines (cut at slab boundaries), and tasks never straddle two lines."""
    A, _ = W.workload("diff3d7_24")
    n = A.n
    npad = (n + 127) // 128 * 128
    bsize = (npad + ROWS * 8 - 1) // (ROWS * 8) * ROWS
    S = schedule(shim, A, 10, 1e-3, bsize, NWARP, True)
    for r0, meta in S["task"]:
        cnt = meta & 7
        if r0 < n:
            assert (r0 % 24) + cnt <= 24 or r0 + cnt > n, (r0, cnt)


def test_planted_marker_mistake_is_caught(shim):
    A, _ = W.workload("diff3d7_24")
    n = A.n
    npad = (n + 127) // 128 * 128
    bsize = (npad + ROWS * 8 - 1) // (ROWS * 8) * ROWS
    S = schedule(shim, A, 10, 1e-3, bsize, NWARP, True)
    rhs = W.rng_for(12).standard_normal(n)
    x_ok, _, _ = simulate(S, n, npad, bsize, rhs, True)
    with pytest.raises(AssertionError):
        x_bad, _, _ = simulate(S, n, npad, bsize, rhs, True, plant="distance")
        assert np.allclose(x_bad[:n], x_ok[:n])


def level_layout(lib, A, lfil, tau, bsize, R, lower):
    rp = np.ascontiguousarray(A.rowptr, np.int64)
    ci = np.ascontiguousarray(A.col, np.int32)
    va = np.ascontiguousarray(A.val, np.float64)
    assert lib.shim_factor(A.n, rp.ctypes.data, ci.ctypes.data, va.ctypes.data, lfil, tau) == 0
    nent, nslab = ctypes.c_int64(), ctypes.c_int64()
    npad = lib.shim_level(1 if lower else 0, bsize, R, ctypes.byref(nent), ctypes.byref(nslab))
    ns = nslab.value
    E = dict(off=np.zeros(ns + 1, np.int64), width=np.zeros(ns, np.int32), col=np.zeros(nent.value, np.int32),
             val=np.zeros(nent.value), round=np.zeros(npad, np.uint16), rdiag=np.zeros(npad),
             perm=np.zeros(A.n, np.int32), ns=ns, npad=npad)
    lib.shim_level_get(1 if lower else 0, E["off"].ctypes.data, E["width"].ctypes.data, E["col"].ctypes.data,
                       E["val"].ctypes.data, E["round"].ctypes.data, E["rdiag"].ctypes.data, E["perm"].ctypes.data)
    return E


def simulate_level(E, n, bsize, R, rhs_dev, lower, nwarps=NWARP):
    """The level schedule's rules: in each slab, group gi (R consecutive
    positions, taken from the front for L and from the back for U) belongs
    to warp gi mod nwarps, which takes its groups in order; the rows of a
    group run in rounds (round[r]), a round when all its rows' entries are
    computed.  A row's entries are read as the kernel reads them: the
    2 * 32 / R prefetched ones, then the group's overflow steps of 32 / R
    (high byte of round[r]; 255: up to the slab's width); every entry past
    that must be padding."""
    npad = E["npad"]
    x = np.full(npad, np.nan)
    done = np.zeros(npad, bool)
    solved = np.zeros(npad, np.int64)
    b = np.zeros(npad)
    b[:n] = rhs_dev
    queues = []
    for s in range(E["ns"]):
        b0, b1 = s * bsize, min(npad, (s + 1) * bsize)
        ngrp = (b1 - b0) // R
        for w in range(nwarps):
            its = list(range(w, ngrp, nwarps))
            queues.append(dict(s=s, b0=b0, ngrp=ngrp, its=its, pos=0, rnd=0))
    while True:
        progress = False
        for qd in queues:
            while qd["pos"] < len(qd["its"]):
                it = qd["its"][qd["pos"]]
                gi = it if lower else qd["ngrp"] - 1 - it
                rows = [qd["b0"] + R * gi + q for q in range(R)]
                s = qd["s"]
                steps = int(E["round"][rows[0]]) >> 8
                assert all(int(E["round"][r]) >> 8 == steps for r in rows)
                wd = int(E["width"][s]) if steps == 255 else min(int(E["width"][s]), (2 + steps) * (32 // R))
                for r in rows:
                    e = E["off"][s] + (r - qd["b0"]) * int(E["width"][s])
                    assert np.all(E["col"][e + wd:e + int(E["width"][s])] == -1), "a real entry past the group's length"
                rounds = 1 + max(int(E["round"][r]) & 15 for r in rows)
                assert all(1 + ((int(E["round"][r]) >> 4) & 15) == rounds for r in rows)
                rd = qd["rnd"]
                act = [r for r in rows if (int(E["round"][r]) & 15) == rd]
                ready = True
                for r in act:
                    e = E["off"][s] + (r - qd["b0"]) * int(E["width"][s])
                    for k in range(wd):
                        c = E["col"][e + k]
                        if c >= 0 and not done[c]:
                            ready = False
                if not ready:
                    break
                for r in act:
                    e = E["off"][s] + (r - qd["b0"]) * int(E["width"][s])
                    acc = 0.0
                    for k in range(wd):
                        c = E["col"][e + k]
                        if c >= 0:
                            acc += E["val"][e + k] * x[c]
                    x[r] = (b[r] - acc) * E["rdiag"][r]
                    done[r] = True
                    solved[r] += 1
                progress = True
                if rd + 1 < rounds:
                    qd["rnd"] = rd + 1
                else:
                    qd["rnd"] = 0
                    qd["pos"] += 1
        if not progress:
            break
    return x, solved, all(qd["pos"] == len(qd["its"]) for qd in queues)


@pytest.mark.parametrize("R", [4, 2])
@pytest.mark.parametrize("lower", [True, False])
@pytest.mark.parametrize("name,lfil,tau", CASES)
def test_level_schedule_solves_and_never_stalls(shim, name, lfil, tau, lower, R):
    """The level layout (slab-major level-minor relabelling, per-slab ELL and
    rounds for groups of R = 4 or 2 rows) run by the level schedule's rules:
    every row solved once, no stall, and the triangular solve of the
    relabelled factor equals scipy's on the factor itself."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import spsolve_triangular

    import oracle as O

    A, _ = W.workload(name)
    n = A.n
    npad = (n + 127) // 128 * 128
    grid = 8
    bsize = (npad + ROWS * grid - 1) // (ROWS * grid) * ROWS
    E = level_layout(shim, A, lfil, tau, bsize, R, lower)
    perm = E["perm"]
    rhs = W.rng_for(13).standard_normal(n)
    x, solved, complete = simulate_level(E, n, bsize, R, rhs[perm], lower)
    assert complete, "the schedule stalled"
    assert np.all(solved == 1)
    ic = O.ic_factor(A, lfil, tau)
    L = sp.csr_matrix((ic.Lval, ic.Lcol, ic.Lrowptr), shape=(n, n))
    ref = spsolve_triangular(L, rhs, lower=True) if lower else spsolve_triangular(L.T.tocsr(), rhs, lower=False)
    np.testing.assert_allclose(x[:n], ref[perm], rtol=1e-10, atol=1e-12 * np.abs(ref).max())
