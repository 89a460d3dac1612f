"""Pins of the oracle against facts fixed by the paper and by the mathematics.

None of these re-types an oracle formula: each checks the oracle against a
closed form, a textbook brute force, a library routine for a special case,
or an identity that a dropped term, a wrong sign or a transposed operand
would break.  CPU only.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


# ---------------------------------------------------------------------------
# helpers written independently of the oracle
# ---------------------------------------------------------------------------

def jacobi_eigenvalues(M, sweeps=30, tol=1e-14):
    """Cyclic Jacobi eigenvalue method (textbook; Golub & Van Loan 8.5)."""
    A = np.array(M, dtype=np.float64, copy=True)
    n = A.shape[0]
    for _ in range(sweeps):
        off = math.sqrt(max(np.sum(A * A) - np.sum(np.diag(A) ** 2), 0.0))
        if off <= tol * np.linalg.norm(A):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = math.copysign(1.0, tau) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                rp = A[p, :].copy()
                rq = A[q, :].copy()
                A[p, :] = c * rp - s * rq
                A[q, :] = s * rp + c * rq
    return np.sort(np.diag(A))


def small_diffusion(nx=9, ny=11, seed=3):
    rng = W.rng_for(seed)
    return W.diffusion_2d_from_kappa(np.exp(0.5 * rng.standard_normal((ny, nx))))


def dense(A):
    return A.to_scipy().toarray()


# ---------------------------------------------------------------------------
# IC(lfil, tau) factor
# ---------------------------------------------------------------------------

def test_ict_exact_cholesky_when_nothing_dropped():
    A = small_diffusion(8, 9)
    ic = O.ic_factor(A, lfil=A.n, tau=0.0)
    Lref = np.linalg.cholesky(dense(A))
    L = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            L[i, ic.Lcol[e]] = ic.Lval[e]
    np.testing.assert_allclose(L, Lref, rtol=0, atol=1e-13 * np.abs(Lref).max())


def test_ict_tridiagonal_exact_for_any_lfil():
    A = W.tridiag(50, 2.5, -1.0)
    ic = O.ic_factor(A, lfil=1, tau=1e-2)
    assert ic.nnz == 2 * 50 - 1
    L = np.zeros((50, 50))
    for i in range(50):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            L[i, ic.Lcol[e]] = ic.Lval[e]
    np.testing.assert_allclose(L @ L.T, dense(A), atol=1e-14)


def test_ict_lfil0_is_diagonal_sqrt():
    A = small_diffusion()
    ic = O.ic_factor(A, lfil=0, tau=0.0)
    assert ic.nnz == A.n
    np.testing.assert_array_equal(ic.Lval, np.sqrt(A.to_scipy().diagonal()))


@pytest.mark.parametrize("lfil,tau", [(2, 1e-2), (5, 1e-3), (10, 0.0), (3, 0.2)])
def test_ict_matches_A_on_kept_pattern(lfil, tau):
    """Defining property of incomplete Cholesky: (L L^T)_ij = A_ij on every kept (i,j)."""
    A = small_diffusion(10, 12, seed=lfil)
    ic = O.ic_factor(A, lfil=lfil, tau=tau)
    L = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            L[i, ic.Lcol[e]] = ic.Lval[e]
    Ad = dense(A)
    LLt = L @ L.T
    mask = L != 0
    np.testing.assert_allclose(LLt[mask], Ad[mask], atol=1e-13 * np.abs(Ad).max())
    # lfil bound per column of L, diagonal always present
    counts = np.count_nonzero(L, axis=0)
    assert counts.max() <= lfil + 1 and np.all(np.diag(L) > 0)
    # the drop threshold: every kept off-diagonal clears tau * ||A(:,j)||
    cn = np.linalg.norm(Ad, axis=0)
    for j in range(A.n):
        off = np.abs(L[j + 1:, j])
        off = off[off != 0]
        assert np.all(off >= tau * cn[j])


def test_ict_keeps_largest_lfil_by_hand():
    """3x3 example worked by hand: column 0 has candidates 0.5 (row 1) and 0.25 (row 2)."""
    A = W.CSR(3, np.array([0, 3, 5, 7], np.int64), np.array([0, 1, 2, 0, 1, 0, 2], np.int32),
              np.array([4.0, 2.0, 1.0, 2.0, 5.0, 1.0, 6.0]))
    ic = O.ic_factor(A, lfil=1, tau=0.0)
    # L00 = 2, L10 = 1 (kept), L20 = 0.5 (dropped by lfil=1);
    # column 1: w1 = 5 - 1*1 = 4 -> L11 = 2; row 2 not touched -> L22 = sqrt(6)
    Lexp = {(0, 0): 2.0, (1, 0): 1.0, (1, 1): 2.0, (2, 2): math.sqrt(6.0)}
    got = {}
    for i in range(3):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            got[(i, int(ic.Lcol[e]))] = ic.Lval[e]
    assert got == Lexp
    # tau = 0.06: column 0 keeps L10 = 1 and L20 = 0.5 (threshold 0.06*sqrt(21) = 0.275);
    # column 1: w = (5 - 1, 0 - 0.5) -> L11 = 2, L21 = -0.25 < 0.06*sqrt(29) = 0.323 dropped;
    # column 2: w2 = 6 - 0.25 -> L22 = sqrt(5.75)
    ic2 = O.ic_factor(A, lfil=5, tau=0.06)
    got = {}
    for i in range(3):
        for e in range(ic2.Lrowptr[i], ic2.Lrowptr[i + 1]):
            got[(i, int(ic2.Lcol[e]))] = ic2.Lval[e]
    assert got == {(0, 0): 2.0, (1, 0): 1.0, (2, 0): 0.5, (1, 1): 2.0, (2, 2): math.sqrt(5.75)}


def test_ict_breakdown_reported():
    A = W.CSR(2, np.array([0, 2, 4], np.int64), np.array([0, 1, 0, 1], np.int32), np.array([1.0, 2.0, 2.0, 1.0]))
    with pytest.raises(O.ic.ICBreakdown):
        O.ic_factor(A, lfil=1, tau=0.0)


def test_levels_are_longest_paths():
    import networkx as nx

    A = small_diffusion(12, 10, seed=7)
    ic = O.ic_factor(A, lfil=4, tau=1e-3)
    G = nx.DiGraph()
    G.add_nodes_from(range(A.n))
    for i in range(A.n):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            j = int(ic.Lcol[e])
            if j < i:
                G.add_edge(j, i)
    lev = np.zeros(A.n, dtype=int)
    for v in nx.topological_sort(G):
        for w in G.successors(v):
            lev[w] = max(lev[w], lev[v] + 1)
    np.testing.assert_array_equal(ic.levL, lev)
    # upper factor: longest path to a sink of the same DAG
    levU = np.zeros(A.n, dtype=int)
    for v in reversed(list(nx.topological_sort(G))):
        for w in G.successors(v):
            levU[v] = max(levU[v], levU[w] + 1)
    np.testing.assert_array_equal(ic.levU, levU)
    lptr, rows = O.level_sets(ic.levL, ic.nlevL)
    for l in range(ic.nlevL):
        blk = rows[lptr[l]:lptr[l + 1]]
        assert np.all(np.diff(blk) > 0) and np.all(ic.levL[blk] == l)


def test_sparse_kernels_against_scipy():
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    A = small_diffusion(13, 7)
    ic = O.ic_factor(A, lfil=3, tau=1e-2)
    x = W.rng_for(1).standard_normal(A.n)
    np.testing.assert_allclose(O.spmv(A, x), A.to_scipy() @ x, rtol=1e-14, atol=1e-14)
    L = sp.csr_matrix((ic.Lval, ic.Lcol, ic.Lrowptr), shape=(A.n, A.n))
    U = sp.csr_matrix((ic.Uval, ic.Ucol, ic.Urowptr), shape=(A.n, A.n))
    np.testing.assert_allclose((L - U.T).toarray(), 0, atol=0)
    np.testing.assert_allclose(O.lsolve(ic, x), spl.spsolve_triangular(L, x, lower=True), rtol=1e-12)
    np.testing.assert_allclose(O.usolve(ic, x), spl.spsolve_triangular(U, x, lower=False), rtol=1e-12)


# ---------------------------------------------------------------------------
# Algorithm 3.1 (preconditioner application)
# ---------------------------------------------------------------------------

def _pairs(A, ic, k, seed=0):
    """k pairs with alpha_s = s^T r < 0, as produced by the Newton iteration
    (s solves the correction equation, so s^T r = -s^T J s < 0)."""
    rng = W.rng_for(seed)
    Ad = dense(A)
    S, R, al = [], [], []
    for _ in range(k):
        r = rng.standard_normal(A.n)
        s = -np.linalg.solve(Ad, r) + 0.1 * rng.standard_normal(A.n)
        if s @ r > 0:
            s = -s
        S.append(s)
        R.append(r)
        al.append(s @ r)
    return S, R, al


def test_bfgs_secant_identity_all_pairs():
    """P_{k}hat(-r_{k-1}) = s_{k-1} holds exactly for the newest pair (eq. lastprec)."""
    A = small_diffusion()
    ic = O.ic_factor(A, lfil=3, tau=1e-2)
    for k in (1, 2, 3, 5):
        S, R, al = _pairs(A, ic, k, seed=k)
        c = O.bfgs_apply(-R[-1], S, R, al, ic, None)
        np.testing.assert_allclose(c, S[-1], rtol=1e-10, atol=1e-10 * np.abs(S[-1]).max())
        # and for every older pair against the preconditioner built up to it
        for t in range(k - 1):
            c = O.bfgs_apply(-R[t], S[:t + 1], R[:t + 1], al[:t + 1], ic, None)
            np.testing.assert_allclose(c, S[t], rtol=1e-10, atol=1e-10 * np.abs(S[t]).max())


def _dense_op(fn, n):
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = fn(e)
    return M


def test_bfgs_symmetric_positive_definite():
    """Theorem 3.2: with alpha_s < 0 every P_khat is SPD (and symmetric)."""
    A = small_diffusion(7, 8)
    ic = O.ic_factor(A, lfil=3, tau=1e-2)
    S, R, al = _pairs(A, ic, 4, seed=11)
    assert all(a < 0 for a in al)
    P = _dense_op(lambda e: O.bfgs_apply(e, S, R, al, ic, None), A.n)
    np.testing.assert_allclose(P, P.T, atol=1e-10 * np.abs(P).max())
    assert np.linalg.eigvalsh(0.5 * (P + P.T)).min() > 0


def test_bfgs_k0_is_projected_ic():
    A = small_diffusion(7, 8)
    ic = O.ic_factor(A, lfil=2, tau=1e-2)
    L = np.zeros((A.n, A.n))
    for i in range(A.n):
        for e in range(ic.Lrowptr[i], ic.Lrowptr[i + 1]):
            L[i, ic.Lcol[e]] = ic.Lval[e]
    Q, _ = np.linalg.qr(W.rng_for(5).standard_normal((A.n, 3)))
    g = W.rng_for(6).standard_normal(A.n)
    g = g - Q @ (Q.T @ g)
    Pq = np.eye(A.n) - Q @ Q.T
    ref = Pq @ np.linalg.solve(L @ L.T, g)
    np.testing.assert_allclose(O.bfgs_apply(g, [], [], [], ic, Q), ref, rtol=1e-10, atol=1e-12)


def test_planted_mistakes_are_caught():
    """Mistakes planted in a copy of Algorithm 3.1 break the pins above: a sign
    error on b breaks symmetry, reversed pair nesting breaks the secant identity."""
    A = small_diffusion(6, 7)
    ic = O.ic_factor(A, lfil=3, tau=1e-2)
    S, R, al = _pairs(A, ic, 3, seed=2)

    def planted(g, sign_b=1.0, reverse=False):
        k = len(S)
        order = list(range(k))
        if reverse:
            order = order[::-1]
        w = g.copy()
        a = np.zeros(k)
        for s in reversed(order):
            a[s] = S[s] @ w / al[s]
            w = w - a[s] * R[s]
        c = O.solver.p0hat(ic, w)
        for s in order:
            b = R[s] @ c / al[s]
            c = c - (a[s] + sign_b * b) * S[s]
        return c

    # the unplanted copy passes both pins
    P = _dense_op(lambda e: planted(e), A.n)
    np.testing.assert_allclose(P, P.T, atol=1e-10 * np.abs(P).max())
    np.testing.assert_allclose(planted(-R[-1]), S[-1], atol=1e-10 * np.abs(S[-1]).max())
    Pbad = _dense_op(lambda e: planted(e, sign_b=-1.0), A.n)
    assert np.abs(Pbad - Pbad.T).max() > 1e-3 * np.abs(Pbad).max()
    c = planted(-R[-1], reverse=True)
    assert np.abs(c - S[-1]).max() > 1e-3 * np.abs(S[-1]).max()


# ---------------------------------------------------------------------------
# PCG on the correction equation
# ---------------------------------------------------------------------------

def _newton_state(A, j_conv=2, seed=0):
    """Converged eigenvectors v_1..v_j (dense eigh) and a perturbed u ~ v_{j+1}."""
    Ad = dense(A)
    lam, V = np.linalg.eigh(Ad)
    rng = W.rng_for(seed)
    Qt = V[:, :j_conv]
    d = rng.standard_normal(A.n)
    u = V[:, j_conv] + 0.05 * d / np.linalg.norm(d)
    u = u - Qt @ (Qt.T @ u)
    u /= np.linalg.norm(u)
    theta = u @ Ad @ u
    r = Ad @ u - theta * u
    return Ad, lam, V, Qt, u, theta, r


def test_pcg_solves_projected_system():
    A = small_diffusion(9, 10, seed=4)
    ic = O.ic_factor(A, lfil=4, tau=1e-3)
    Ad, lam, V, Qt, u, theta, r = _newton_state(A)
    Q = np.concatenate([Qt, u[:, None]], axis=1)
    opt = O.OracleOptions(tau_pcg=1e-13, max_pcg=400, exit_eigres=False, exit_stagnation=False)
    s, info = O.pcg_correction(A, theta, u, r, Q, [], [], [], ic, opt)
    # dense solution of the projected system on the complement of Q
    Z = np.linalg.svd(np.eye(A.n) - Q @ Q.T)[0][:, :A.n - Q.shape[1]]
    sref = Z @ np.linalg.solve(Z.T @ (Ad - theta * np.eye(A.n)) @ Z, -(Z.T @ r))
    np.testing.assert_allclose(s, sref, rtol=1e-8, atol=1e-9 * np.abs(sref).max())
    assert np.abs(Q.T @ s).max() < 1e-10 * np.linalg.norm(s)


def test_eigres_estimate_matches_exact():
    """The product-free exit (iii) value agrees with the exact ||A x - rho x||/||x||."""
    A = small_diffusion(10, 11, seed=9)
    ic = O.ic_factor(A, lfil=4, tau=1e-3)
    Ad, lam, V, Qt, u, theta, r = _newton_state(A, j_conv=3, seed=3)
    Q = np.concatenate([Qt, u[:, None]], axis=1)
    opt = O.OracleOptions(tau_pcg=1e-10, max_pcg=30, exit_eigres=False, exit_stagnation=False,
                          debug_exact_eigres=True)
    s, info = O.pcg_correction(A, theta, u, r, Q, [], [], [], ic, opt)
    est = np.array(info["eigres_est"])
    ex = np.array(info["eigres_exact"])
    np.testing.assert_allclose(est, ex, rtol=1e-6, atol=1e-12)


def test_lemma_notay_lower_bound():
    """Lemma 3.1 (general j, Section 3.2): z^T J_k z > (lambda_{j+1}-lambda_j)/2 for z perp Q."""
    A = small_diffusion(8, 9, seed=5)
    Ad, lam, V, Qt, u, theta, r = _newton_state(A, j_conv=2, seed=1)
    # u close to v_3: error small enough for the lemma's neighbourhood
    d = W.rng_for(2).standard_normal(A.n)
    u = V[:, 2] + 1e-3 * d / np.linalg.norm(d)
    u = u - Qt @ (Qt.T @ u)
    u /= np.linalg.norm(u)
    theta = u @ Ad @ u
    Q = np.concatenate([Qt, u[:, None]], axis=1)
    Z = np.linalg.svd(np.eye(A.n) - Q @ Q.T)[0][:, :A.n - 3]
    Jz = Z.T @ (Ad - theta * np.eye(A.n)) @ Z
    ev = np.linalg.eigvalsh(Jz)
    assert ev.min() > (lam[3] - lam[2]) / 2
    assert ev.max() < lam[-1]


# ---------------------------------------------------------------------------
# DACG line search
# ---------------------------------------------------------------------------

def test_line_search_minimises_rayleigh_quotient():
    from scipy.optimize import minimize_scalar

    A = small_diffusion()
    Ad = dense(A)
    rng = W.rng_for(4)
    for _ in range(5):
        x = rng.standard_normal(A.n)
        p = rng.standard_normal(A.n)

        def q(al):
            y = x + al * p
            return y @ Ad @ y / (y @ y)

        al = O.solver._line_search(p @ Ad @ p, x @ Ad @ p, x @ Ad @ x, p @ p, x @ p, x @ x)
        best = min((minimize_scalar(q, bracket=(b0, b0 + 1.0)) for b0 in (-10.0, -1.0, 0.0, 1.0, 10.0)),
                   key=lambda res: res.fun)
        assert q(al) <= best.fun + 1e-12 * abs(best.fun)


# ---------------------------------------------------------------------------
# Algorithm 3.2 end to end
# ---------------------------------------------------------------------------

def test_dacg_newton_closed_form_aniso_laplacian():
    A, st = W.workload("aniso2d_30x37")
    opt = O.OracleOptions(tol=1e-10, lfil=5, tau_ic=1e-2)
    X0 = W.start_vectors(A.n, 5, st["seed"])
    lam, V, stats = O.dacg_newton(A, 5, X0, opt)
    exact = W.laplacian_2d_aniso_eigs(30, 37, 1.0, 1.7)[:5]
    np.testing.assert_allclose(lam, exact, rtol=1e-12)
    assert stats["ascending"] and all(stats["converged"])
    # eigenvectors are the separable sines; the 5 smallest are (k,l) below
    kl = [(1, 1), (2, 1), (1, 2), (2, 2), (3, 1)]
    evs = {float(W.laplacian_2d_aniso_eigs(30, 37, 1, 1.7)[0]): None}
    del evs
    for j, (k, l) in enumerate(kl):
        v = W.laplacian_2d_aniso_eigvec(30, 37, k, l)
        assert abs(abs(v @ V[:, j]) - 1.0) < 1e-12
    np.testing.assert_allclose(V.T @ V, np.eye(5), atol=1e-12)
    Asp = A.to_scipy()
    for j in range(5):
        assert np.linalg.norm(Asp @ V[:, j] - lam[j] * V[:, j]) <= 1e-10 * lam[j]


@pytest.mark.parametrize("maker", ["diff", "rgg"])
def test_dacg_newton_against_jacobi_brute_force(maker):
    if maker == "diff":
        A = small_diffusion(9, 11, seed=21)
        p = 4
    else:
        A = W.geometric_graph_laplacian(140, seed=5)
        p = 3
    opt = O.OracleOptions(tol=1e-10, lfil=10, tau_ic=1e-3)
    X0 = W.start_vectors(A.n, p, 77)
    lam, V, stats = O.dacg_newton(A, p, X0, opt)
    ref = jacobi_eigenvalues(dense(A))
    np.testing.assert_allclose(ref, np.linalg.eigvalsh(dense(A)), rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(lam, ref[:p], rtol=1e-10)
    assert stats["ascending"]
    if maker == "rgg":
        assert abs(lam[0] - 1e-3) < 1e-13
        v1 = np.full(A.n, 1 / math.sqrt(A.n))
        assert abs(abs(V[:, 0] @ v1) - 1) < 1e-10


def test_bfgs_pairs_have_negative_alpha_and_help():
    """alpha_s = s^T r < 0 along the Newton iteration (Theorem 3.2), and k_max > 0
    needs no more inner iterations than k_max = 0 (Section 5.2 trend)."""
    A, st = W.workload("diff3d7_24")
    X0 = W.start_vectors(A.n, 3, st["seed"])
    tot = {}
    for kmax in (0, 5):
        opt = O.OracleOptions(tol=1e-8, lfil=10, tau_ic=1e-3, k_max=kmax)
        lam, V, stats = O.dacg_newton(A, 3, X0, opt)
        tot[kmax] = sum(sum(x) for x in stats["pcg_its"])
        assert all(stats["converged"])
    assert tot[5] <= tot[0]


def test_lemma3_step_bound():
    """Lemma 3.3: ||s|| <= 3 ||e_k|| near the solution (exact inner solve)."""
    A = small_diffusion(8, 9, seed=8)
    ic = O.ic_factor(A, lfil=4, tau=1e-3)
    Ad = dense(A)
    lam, Vv = np.linalg.eigh(Ad)
    v = Vv[:, 0]
    d = W.rng_for(3).standard_normal(A.n)
    u = v + 1e-2 * d / np.linalg.norm(d)
    u /= np.linalg.norm(u)
    if u @ v < 0:
        v = -v
    theta = u @ Ad @ u
    r = Ad @ u - theta * u
    opt = O.OracleOptions(tau_pcg=1e-14, max_pcg=500, exit_eigres=False, exit_stagnation=False)
    s, _ = O.pcg_correction(A, theta, u, r, u[:, None], [], [], [], ic, opt)
    assert np.linalg.norm(s) <= 3 * np.linalg.norm(u - v)


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------

def test_adjoint_eigenvalue_closed_form():
    """d lambda_{k,l} / d a = 2 - 2 cos(k pi/(nx+1)) for the anisotropic Laplacian."""
    nx, ny = 12, 15
    A = W.laplacian_2d_aniso(nx, ny, 1.0, 1.7)
    ic = O.ic_factor(A, 5, 1e-2)
    lam, Vv = np.linalg.eigh(dense(A))
    p = 3
    V = Vv[:, :p]
    grad = O.adjoint_grad(A, lam[:p], V, np.array([1.0, 0.0, 0.0]), None, ic)
    # dA/da has -1 on x-couplings and +2 on the diagonal
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    dA = np.where(rows == A.col, 2.0, np.where(np.abs(rows - A.col) == 1, -1.0, 0.0))
    assert abs(grad @ dA - (2 - 2 * math.cos(math.pi / (nx + 1)))) < 1e-12


def test_adjoint_eigenvector_finite_differences():
    A = small_diffusion(7, 8, seed=12)
    ic = O.ic_factor(A, 5, 1e-3)
    Ad = dense(A)
    p = 3
    rng = W.rng_for(13)
    wv = rng.random(A.n)

    def loss_of(M):
        lam, Vv = np.linalg.eigh(M)
        V = np.stack([O.fix_sign(Vv[:, j]) for j in range(p)], axis=1)
        return lam[:p].sum() + wv @ (V[:, 0] ** 2), lam[:p], V

    L0, lam, V = loss_of(Ad)
    gbar_V = np.zeros((A.n, p))
    gbar_V[:, 0] = 2 * wv * V[:, 0]
    grad = O.adjoint_grad(A, lam, V, np.ones(p), gbar_V, ic)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    for e in rng.choice(A.nnz, size=12, replace=False):
        h = 1e-6
        M1 = Ad.copy()
        M1[rows[e], A.col[e]] += h
        M2 = Ad.copy()
        M2[rows[e], A.col[e]] -= h
        # a one-sided (non-symmetric) perturbation: eigh reads the lower triangle,
        # so symmetrise explicitly the way the gradient convention defines it
        fd = (loss_of(0.5 * (M1 + M1.T))[0] - loss_of(0.5 * (M2 + M2.T))[0]) / (2 * h)
        e2 = np.flatnonzero((rows == A.col[e]) & (A.col == rows[e]))[0]
        sym = 0.5 * (grad[e] + grad[e2])
        assert abs(fd - sym) <= 1e-6 * max(1.0, abs(fd))


def test_torch_assembly_matches_numpy_assembly():
    """The differentiable assembly reproduces the stored values bit for bit
    (so gradients with respect to entries map onto cell coefficients)."""
    import torch

    A = W.diffusion_2d_lognormal(9, 7, seed=5)
    vals = W.diffusion_2d_values_torch(torch.tensor(A.meta["kappa"], dtype=torch.float64))
    np.testing.assert_array_equal(vals.numpy(), A.val)


def test_kappa_gradient_fd_and_euler_identity():
    """Cell-coefficient gradient of loss = sum lambda_j + sum_i w_i (v_1)_i^2:
    the oracle adjoint chained through the torch assembly against central
    differences of a dense eigendecomposition (step 1e-6 kappa_c), and the
    Euler identity for the degree-1 homogeneous assembly,
    sum_c kappa_c dL/dkappa_c = sum_j lambda_j."""
    import torch

    A = W.diffusion_2d_lognormal(9, 7, seed=21)
    kappa = A.meta["kappa"]
    w = A.meta["w"]
    p = 3

    def loss_of(kap):
        B = W.diffusion_2d_from_kappa(kap)
        lam, Vv = np.linalg.eigh(dense(B))
        V = np.stack([O.fix_sign(Vv[:, j]) for j in range(p)], axis=1)
        return lam[:p].sum() + w @ (V[:, 0] ** 2), lam[:p], V

    L0, lam, V = loss_of(kappa)
    ic = O.ic_factor(A, 5, 1e-3)
    gV = np.zeros((A.n, p))
    gV[:, 0] = 2 * w * V[:, 0]
    gA = O.adjoint_grad(A, lam, V, np.ones(p), gV, ic)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    (gk,) = torch.autograd.grad(W.diffusion_2d_values_torch(kt), kt, grad_outputs=torch.tensor(gA))
    gk = gk.numpy()
    assert abs((kappa * gk).sum() - lam.sum()) <= 1e-9 * lam.sum()
    scale = np.abs(gk).max()
    for c in range(A.n):
        h = 1e-6 * kappa.flat[c]
        kp = kappa.copy()
        kp.flat[c] += h
        km = kappa.copy()
        km.flat[c] -= h
        fd = (loss_of(kp)[0] - loss_of(km)[0]) / (2 * h)
        assert abs(fd - gk.flat[c]) <= 1e-6 * scale, (c, fd, gk.flat[c])


def test_hex_torch_assembly_matches_numpy_assembly():
    """The differentiable hex assembly reproduces the stored values of the
    27-point stiffness bit for bit (so gradients with respect to entries map
    onto element coefficients)."""
    import torch

    A = W.hex_poisson_27pt(5, seed=7)
    vals = W.hex_poisson_values_torch(torch.tensor(A.meta["kappa"], dtype=torch.float64))
    np.testing.assert_array_equal(vals.numpy(), A.val)


def test_hex_element_gradient_fd_and_euler_identity():
    """Element-coefficient gradient of loss = sum lambda_j for the hex
    stiffness: the oracle adjoint (d lambda_j / d A_ab = v_ja v_jb) chained
    through the torch assembly against central differences of a dense
    eigendecomposition (step 1e-6 kappa_e) at every element, and the Euler
    identity sum_e kappa_e dL/dkappa_e = sum_j lambda_j."""
    import torch

    A = W.hex_poisson_27pt(3, seed=31)  # 27 unknowns, 64 elements
    kappa = A.meta["kappa"]
    p = 4

    def loss_of(kap):
        lam = np.linalg.eigvalsh(dense(W.hex_poisson_from_kappa(kap)))
        return lam[:p].sum()

    lam, Vv = np.linalg.eigh(dense(A))
    V = np.stack([O.fix_sign(Vv[:, j]) for j in range(p)], axis=1)
    gA = O.adjoint_grad(A, lam[:p], V, np.ones(p), None, None)
    kt = torch.tensor(kappa, dtype=torch.float64, requires_grad=True)
    (gk,) = torch.autograd.grad(W.hex_poisson_values_torch(kt), kt, grad_outputs=torch.tensor(gA))
    gk = gk.numpy()
    assert abs((kappa * gk).sum() - lam[:p].sum()) <= 1e-12 * lam[:p].sum()
    scale = np.abs(gk).max()
    for e in range(kappa.size):
        h = 1e-6 * kappa.flat[e]
        kp = kappa.copy()
        kp.flat[e] += h
        km = kappa.copy()
        km.flat[e] -= h
        fd = (loss_of(kp) - loss_of(km)) / (2 * h)
        assert abs(fd - gk.flat[e]) <= 1e-6 * scale, (e, fd, gk.flat[e])


def test_count_sketch_estimates_vector_distance():
    """The CountSketch the full-size tests compare eigenvectors through:
    linear, and ||S x|| within 25 % of ||x|| for spread-out vectors at
    K = 256 (its relative spread is about sqrt(2/K) = 9 %)."""
    n, K = 200_000, 256
    bucket, sign = W.count_sketch_hash(n, K, 5)
    rng = W.rng_for(77)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    np.testing.assert_allclose(W.count_sketch(x + 2 * y, bucket, sign, K),
                               W.count_sketch(x, bucket, sign, K) + 2 * W.count_sketch(y, bucket, sign, K),
                               rtol=1e-12, atol=1e-9)
    for t in range(20):
        z = W.rng_for(100 + t).standard_normal(n) * np.exp(W.rng_for(200 + t).standard_normal(n))
        r = np.linalg.norm(W.count_sketch(z, bucket, sign, K)) / np.linalg.norm(z)
        assert 0.75 <= r <= 1.25, (t, r)


def test_full_bfgs_update_pairs_and_closed_form():
    """Section 3's full BFGS update (y_k = r_{k+1} - r_k): the method still
    reaches the closed-form spectrum of the anisotropic Laplacian; every
    stored pair has alpha = s^T w < 0 (Theorem 3.2, SPD update); and the
    preconditioner built from the stored pairs maps -w_k to s_k for the
    newest pair (the secant condition P_{k+1} y_k = s_k)."""
    A, st = W.workload("aniso2d_30x37")
    p = 3
    X0 = W.start_vectors(A.n, p, st["seed"])
    opt = O.OracleOptions(tol=1e-10, lfil=st["lfil"], tau_ic=st["tau_ic"], bfgs_full=True)
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    lam, V, stats = O.dacg_newton(A, p, X0, opt, ic=ic)
    exact = W.laplacian_2d_aniso_eigs(30, 37, 1.0, 1.7)[:p]
    np.testing.assert_allclose(lam, exact, rtol=1e-10)
    S, R = stats["last_pairs"]
    assert len(S) >= 1
    for s, w in zip(S, R):
        assert s @ w < 0
    # secant: the update that appended the newest pair maps -w to s
    alpha = [s @ w for s, w in zip(S, R)]
    c = O.bfgs_apply(-R[-1], S, R, alpha, ic, None)
    np.testing.assert_allclose(c, S[-1], rtol=1e-9, atol=1e-12 * np.linalg.norm(S[-1]))


def test_bfgs_pairs_raise_lambda_min_of_preconditioned_jacobian():
    """The effect of the BFGS update on the spectrum of P_k J_k restricted to
    the complement of u_k (the quantity of the paper's condition-number
    study, Section 5): along the Newton steps of the first eigenpair of the
    30 x 37 anisotropic Laplacian, every stored pair raises the smallest
    eigenvalue (the largest stays put), so the condition number falls;
    without pairs (k_max = 0) it stays at that of the projected IC
    preconditioner.  Dense eigenvalues, n = 1110."""
    A, st = W.workload("aniso2d_30x37")
    n = A.n
    Ad = dense(A)
    ic = O.ic_factor(A, st["lfil"], st["tau_ic"])
    x0 = W.start_vectors(n, 1, st["seed"])[0]
    result = {}
    for kmax in (0, 10):
        opt = O.OracleOptions(tol=1e-12, lfil=st["lfil"], tau_ic=st["tau_ic"], k_max=kmax)
        u, _, _ = O.solver.dacg(A, x0, np.zeros((n, 0)), ic, 1e-2, 5000)
        u = u / np.linalg.norm(u)
        theta = u @ Ad @ u
        r = Ad @ u - theta * u
        S, R, al = [], [], []
        spectra = []
        for step in range(5):
            Z = np.linalg.qr(np.concatenate([u[:, None], np.eye(n)], axis=1))[0][:, 1:n]
            K = Z.T @ (Ad - theta * np.eye(n)) @ Z
            M = Z.T @ np.stack([O.bfgs_apply(Z[:, i], S, R, al, ic, u[:, None]) for i in range(n - 1)], axis=1)
            ev = np.sort(np.linalg.eigvals(M @ K).real)
            spectra.append((len(S), ev[0], ev[-1]))
            s, _ = O.solver.pcg_correction(A, theta, u, r, u[:, None], S, R, al, ic, opt)
            if kmax > 0 and s @ r < 0:
                S.append(s)
                R.append(r)
                al.append(s @ r)
            t = u + s
            u = t / np.linalg.norm(t)
            theta = u @ Ad @ u
            r = Ad @ u - theta * u
        result[kmax] = spectra
    base = result[0]
    assert max(abs(b[1] / base[0][1] - 1) for b in base) < 1e-3  # no pairs: lambda_min unchanged
    bf = result[10]
    assert [b[0] for b in bf] == [0, 1, 2, 3, 4]
    lmin = [b[1] for b in bf]
    assert all(lmin[i + 1] >= lmin[i] * (1 - 1e-9) for i in range(4))
    assert lmin[-1] > 1.5 * lmin[0]
    assert abs(bf[-1][2] / bf[0][2] - 1) < 1e-3
