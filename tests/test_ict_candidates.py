"""The dependency rule of the device IC factor, checked on the CPU against
the oracle's factor (Section 2, IC(lfil, tau_IC) by left-looking columns).

The device kernel computes column j after the columns k < j with
L(j,k) != 0, which it discovers while it runs: it starts from the lower part
of row j of A and, for every column k' found to have L(j,k') != 0, adds the
rows of column k' between k' and j.  These tests check on the oracle's
factor that this candidate set holds every k with L(j,k) != 0 (so no update
is missed), and that the candidate sets, the accumulator rows and the
entries surviving the drop test fit the kernel's per-warp tables (256, 256
and 128) on the workloads the GPU tests factor on the device."""
import numpy as np
import pytest

import oracle as O
import workloads as W

SPA, CAND, KEEP = 256, 256, 128


def candidate_sets(A, F):
    """Per column j: (candidate columns, accumulator rows, entries before
    the drop test) exactly as the kernel builds them."""
    rp, ci = A.rowptr, A.col
    Lrp, Lci = F.Lrowptr, F.Lcol  # rows of L, diagonal last
    Urp, Uci = F.Urowptr, F.Ucol  # columns of L, diagonal first
    out = []
    for j in range(A.n):
        row = ci[rp[j]:rp[j + 1]]
        cand = set(row[row < j].tolist())
        spa = set(row[row >= j].tolist())
        for k in Lci[Lrp[j]:Lrp[j + 1] - 1]:
            colk = Uci[Urp[k] + 1:Urp[k + 1]]
            cand.update(colk[colk < j].tolist())
            spa.update(colk[colk >= j].tolist())
        out.append((cand, spa))
    return out


@pytest.mark.parametrize("name,lfil,tau", [("aniso2d_30x37", 5, 1e-2), ("diff3d7_24", 10, 1e-3),
                                           ("hex27_16", 20, 1e-4), ("rgg3000", 30, 1e-2),
                                           ("hex27_16", 31, 0.0), ("diff3d7_24", 31, 0.0)])
def test_candidates_hold_every_dependency_and_fit_the_tables(name, lfil, tau):
    A, _ = W.workload(name)
    F = O.ic_factor(A, lfil, tau)
    sets = candidate_sets(A, F)
    Lrp, Lci = F.Lrowptr, F.Lcol
    for j, (cand, spa) in enumerate(sets):
        deps = set(Lci[Lrp[j]:Lrp[j + 1] - 1].tolist())
        assert deps <= cand, (j, sorted(deps - cand))
        # the accumulator holds the diagonal and every entry kept in column j
        Urp, Uci = F.Urowptr, F.Ucol
        kept = set(Uci[Urp[j]:Urp[j + 1]].tolist())
        assert kept <= spa
        assert len(cand) <= CAND and len(spa) <= SPA and len(spa) - 1 <= KEEP


def test_a_dropped_dependency_is_caught():
    """Planted mistake: a candidate rule that forgets the fill candidates
    (only the lower part of row j of A) misses dependencies of a factor
    with fill, so the check above is not vacuous."""
    A, _ = W.workload("diff3d7_24")
    F = O.ic_factor(A, 10, 1e-3)
    missed = 0
    for j in range(A.n):
        row = A.col[A.rowptr[j]:A.rowptr[j + 1]]
        deps = set(F.Lcol[F.Lrowptr[j]:F.Lrowptr[j + 1] - 1].tolist())
        missed += len(deps - set(row[row < j].tolist()))
    assert missed > 0
