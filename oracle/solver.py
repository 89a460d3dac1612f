"""Oracle driver (test infrastructure): the DACG-Newton method in plain FP64 numpy.

Every function follows the paper's steps in the paper's order and notation;
the sparse kernels (SpMV, IC factor, triangular solves) come from the plain-C
file ``nle_oracle.c``.  Readings of points the paper leaves open are stated
where they are taken:

R-sign    The residual is r = A u - theta u and the correction equation is
          J_k s = -r (eq. "gras"); Section 2 writes r with the opposite sign
          once, which would make alpha = s^T r > 0 and break Theorem 3.2.
          With this sign alpha_s = s_s^T r_s < 0.
R-proj    Inside PCG the residual g is projected onto Q-perp after every
          update (g -= alpha y; g -= Q Q^T g).  Section 4.3 drops the
          projection of the Jacobian and Section 4.2 drops the right
          projection of the preconditioner; with both dropped the iteration
          would leave Q-perp because u^T (A - theta I) p = r^T p != 0.
R-exit    Inner exits (Section 4.3): (i) ||g_l|| <= tau_PCG ||g_0||;
          (ii) l = IMAX_PCG; (iii) eq. "residual" read as
          ||A x - rho x|| / ||x|| < tau rho with x = u + s, rho = q(x);
          (iv) for l >= 1, stop when ||r_{k,l}||/||r_{k,l-1}|| >
          ||g_l||/||g_{l-1}||.  ||r_{k,l}|| is evaluated without a product
          with A from the PCG scalars (formula in ``_eigres_estimate``).
R-ring    The k_max most recent pairs are applied in chronological order,
          the oldest innermost (Algorithm 3.1 with s = 0 the oldest).
R-reset   The pair buffer is empty at the start of every eigenpair j.
R-reorth  After u_{k+1} = (u_k+s_k)/||u_k+s_k|| the new iterate is
          re-orthogonalised once against the converged eigenvectors and
          normalised again (exact arithmetic needs no such step).
R-dacg    DACG (cited, not printed) is read as preconditioned nonlinear CG
          on the Rayleigh quotient restricted to the complement of the
          converged eigenvectors, with an exact line search.
R-full    The full BFGS update of Section 3 (option ``bfgs_full``) takes
          y_k = r_{k+1} - r_k in the same sign convention; the stored pair
          is (s_k, w_k = -y_k), which the simplified update (eq.
          "lastprec", the default) replaces by (s_k, r_k).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from . import ic as _ic


@dataclasses.dataclass
class OracleOptions:
    """Parameters of Algorithm 3.2 with the paper's defaults (Table "default")."""
    tol: float = 1e-8  # tau, outer tolerance ||A u - theta u|| <= tau theta
    max_newton: int = 100  # ITMAX
    tau_dacg: float = 1e-2
    max_dacg: int = 5000
    tau_pcg: float = 1e-2
    max_pcg: int = 20  # IMAX_PCG
    k_max: int = 5  # rank-two corrections kept (Section 4.4)
    lfil: int = 30
    tau_ic: float = 1e-2
    exit_eigres: bool = True  # exit (iii)
    exit_stagnation: bool = True  # exit (iv)
    # Section 3: the full BFGS update uses y_k = r_{k+1} - r_k; the default is
    # the simplified update (eq. "lastprec") with y_k replaced by -r_k.  Both
    # store the pair (s_k, w_k) with w_k = -y_k and apply Algorithm 3.1 to it.
    bfgs_full: bool = False
    debug_exact_eigres: bool = False  # also compute exit (iii) with an extra MVP


# ---------------------------------------------------------------------------
# Preconditioner
# ---------------------------------------------------------------------------

def p0hat(ic: _ic.ICFactor, w: np.ndarray) -> np.ndarray:
    """P0hat w = (L L^T)^{-1} w: forward then backward substitution (Section 2)."""
    return _ic.usolve(ic, _ic.lsolve(ic, w))


def bfgs_apply(g: np.ndarray, S: List[np.ndarray], R: List[np.ndarray], alpha: List[float],
               ic: _ic.ICFactor, Q: Optional[np.ndarray]) -> np.ndarray:
    """c = P_k g, Algorithm 3.1.

    S, R hold the stored pairs s_0..s_{k-1}, r_0..r_{k-1} oldest first (R-ring),
    alpha[s] = s_s^T r_s.  Q is n x m (columns orthonormal) or None.
    Pinned by: the secant identity P_{k+1}hat (-r_k) = s_k, symmetry and
    positive definiteness of P_khat (Theorem 3.2), k = 0 reducing to the
    projected IC preconditioner (tests/test_oracle_pins.py).
    """
    k = len(S)
    w = g.copy()
    a = np.zeros(k)
    for s in range(k - 1, -1, -1):
        a[s] = S[s] @ w / alpha[s]
        w = w - a[s] * R[s]
    c = p0hat(ic, w)
    for s in range(k):
        b = R[s] @ c / alpha[s]
        c = c - (a[s] + b) * S[s]
    if Q is not None and Q.shape[1] > 0:
        z = Q.T @ c
        c = c - Q @ z
    return c


# ---------------------------------------------------------------------------
# PCG on the correction equation (Section 4.3)
# ---------------------------------------------------------------------------

def _eigres_estimate(theta, gnorm, rs, sg, ss):
    """||A x - rho x|| / ||x|| and rho for x = u + s, without a product with A.

    From J s = -r - g, s perp Q, (A - theta I) u = r and neglecting the
    residuals of the converged eigenvectors:
      (A - theta I) x = -g + u (r^T s)  =>  ||(A - theta I) x||^2 = ||g||^2 + (r^T s)^2
      x^T (A - theta I) x = r^T s - s^T g,   ||x||^2 = 1 + ||s||^2
      rho - theta = (r^T s - s^T g) / (1 + ||s||^2)
      ||A x - rho x||^2 = ||(A - theta I) x||^2 - (rho - theta)^2 ||x||^2
    Pinned by tests comparing it with the exact value (debug_exact_eigres).
    """
    x2 = 1.0 + ss
    d = (rs - sg) / x2
    e2 = gnorm * gnorm + rs * rs - d * d * x2
    return math.sqrt(max(e2, 0.0) / x2), theta + d


def pcg_correction(A, theta: float, u: np.ndarray, r: np.ndarray, Q: np.ndarray, S, R, alpha, ic,
                   opt: OracleOptions, A_for_debug=None):
    """Solve J_k s = -r_k, s perp Q, by PCG with preconditioner P_k (Section 4.3).

    J_k = (I - Q Q^T)(A - theta I)(I - Q Q^T); P_k applied by Algorithm 3.1.
    Returns (s, info) with info = dict(its, exit, mvp, eigres_est, eigres_exact).
    Exits and projection placement follow R-exit and R-proj.
    """
    n = len(r)
    s = np.zeros(n)
    g = -r.copy()
    g = g - Q @ (Q.T @ g)
    c = bfgs_apply(g, S, R, alpha, ic, Q)
    p = c.copy()
    gamma = g @ c
    g0 = np.linalg.norm(g)
    info = dict(its=0, exit="maxit", mvp=0, eigres_est=[], eigres_exact=[])
    gprev = g0
    eprev = None
    for l in range(opt.max_pcg):
        y = _ic.spmv(A, p) - theta * p
        info["mvp"] += 1
        delta = p @ y
        info["its"] = l + 1
        if not (delta > 0.0):
            info["exit"] = "breakdown"
            info["its"] = l
            break
        a = gamma / delta
        s = s + a * p
        g = g - a * y
        g = g - Q @ (Q.T @ g)
        gn = np.linalg.norm(g)
        eres, rho = _eigres_estimate(theta, gn, r @ s, s @ g, s @ s)
        info["eigres_est"].append(eres)
        if opt.debug_exact_eigres:
            x = u + s
            Ax = _ic.spmv(A, x)
            rq = x @ Ax / (x @ x)
            info["eigres_exact"].append(np.linalg.norm(Ax - rq * x) / np.linalg.norm(x))
        if gn <= opt.tau_pcg * g0:
            info["exit"] = "tol"
            break
        if opt.exit_eigres and eres < opt.tol * rho:
            info["exit"] = "eigres"
            break
        if opt.exit_stagnation and l >= 1 and eres / eprev > gn / gprev:
            info["exit"] = "stagnation"
            break
        if l + 1 == opt.max_pcg:
            info["exit"] = "maxit"
            break
        c = bfgs_apply(g, S, R, alpha, ic, Q)
        gamma_new = g @ c
        beta = gamma_new / gamma
        p = c + beta * p
        gamma = gamma_new
        gprev = gn
        eprev = eres
    return s, info


# ---------------------------------------------------------------------------
# DACG initial guess (Section 4.1, R-dacg)
# ---------------------------------------------------------------------------

def _line_search(a, b, c, d, e, f):
    """Minimiser over alpha of q(x + alpha p) = (c + 2 alpha b + alpha^2 a) / (f + 2 alpha e + alpha^2 d).

    a = p^T A p, b = x^T A p, c = x^T A x, d = p^T p, e = x^T p, f = x^T x.
    dq/dalpha = 0  <=>  (a e - b d) alpha^2 + (a f - c d) alpha + (b f - c e) = 0;
    of the two roots the one with the smaller q is taken (stable formula).
    """
    A2 = a * e - b * d
    B2 = a * f - c * d
    C2 = b * f - c * e

    def q(al):
        return (c + 2 * al * b + al * al * a) / (f + 2 * al * e + al * al * d)

    if A2 == 0.0:
        return -C2 / B2 if B2 != 0.0 else 0.0
    disc = max(B2 * B2 - 4.0 * A2 * C2, 0.0)
    t = -0.5 * (B2 + math.copysign(math.sqrt(disc), B2))
    roots = [t / A2]
    if t != 0.0:
        roots.append(C2 / t)
    return min(roots, key=q)


def dacg(A, x0: np.ndarray, Qt: np.ndarray, ic, tau: float, maxit: int, recompute_every: int = 50):
    """Preconditioned conjugate-gradient minimisation of q(x) on Qt-perp (Section 4.1).

    x0 is projected on Qt-perp (classical Gram-Schmidt, twice) and normalised.
    Each iteration: q = x^T A x, g = A x - q x; stop when ||g|| <= tau q;
    gt = (I - Qt Qt^T) P0hat g; beta = g^T gt / (g_prev^T gt_prev); p = -gt + beta p;
    exact line search for alpha; x += alpha p, A x += alpha A p; normalise.
    Returns (x, its, mvp).  Pinned by the eigenvalue it leads Newton to
    (tests compare with the closed-form and brute-force spectra).
    """
    m = Qt.shape[1]
    x = x0.copy()
    for _ in range(2):
        if m:
            x = x - Qt @ (Qt.T @ x)
    x = x / np.linalg.norm(x)
    Ax = _ic.spmv(A, x)
    mvp = 1
    p = np.zeros_like(x)
    gg_prev = None
    its = 0
    for it in range(maxit):
        q = x @ Ax
        g = Ax - q * x
        if np.linalg.norm(g) <= tau * q:
            break
        gt = p0hat(ic, g)
        if m:
            gt = gt - Qt @ (Qt.T @ gt)
        gg = g @ gt
        beta = 0.0 if gg_prev is None else gg / gg_prev
        p = -gt + beta * p
        Ap = _ic.spmv(A, p)
        mvp += 1
        al = _line_search(p @ Ap, x @ Ap, x @ Ax, p @ p, x @ p, x @ x)
        x = x + al * p
        Ax = Ax + al * Ap
        its = it + 1
        if its % recompute_every == 0:
            Ax = _ic.spmv(A, x)
            mvp += 1
        nx = np.linalg.norm(x)
        x = x / nx
        Ax = Ax / nx
        gg_prev = gg
    return x, its, mvp


# ---------------------------------------------------------------------------
# Algorithm 3.2: DACG-Newton
# ---------------------------------------------------------------------------

def fix_sign(v: np.ndarray) -> np.ndarray:
    """Sign convention: the entry of largest modulus is positive (lowest index on ties)."""
    i = int(np.argmax(np.abs(v)))
    return -v if v[i] < 0 else v


def dacg_newton(A, p: int, X0: np.ndarray, opt: OracleOptions, ic=None):
    """Leftmost p eigenpairs of SPD A by Algorithm 3.2.

    X0 is (p, n): the seeded start vector x_0 of each eigenpair j.
    Returns (lam (p,), V (n, p), stats).  Eigenvalues are returned in the
    order they were found, which must be ascending (stats["ascending"]).
    """
    n = A.n
    if ic is None:
        ic = _ic.ic_factor(A, opt.lfil, opt.tau_ic)
    Qt = np.zeros((n, 0))
    lam = np.zeros(p)
    stats = dict(dacg_its=[], dacg_mvp=[], outer_its=[], pcg_its=[], newton_mvp=[], converged=[],
                 exits=[], final_res=[])
    for j in range(p):
        u, its, mvp_d = dacg(A, X0[j], Qt, ic, opt.tau_dacg, opt.max_dacg)
        stats["dacg_its"].append(its)
        stats["dacg_mvp"].append(mvp_d)
        k = 0
        u = u / np.linalg.norm(u)
        Au = _ic.spmv(A, u)
        mvp_n = 1
        theta = u @ Au
        r = Au - theta * u
        S, R, alpha = [], [], []
        pcg_its = []
        exits = []
        while np.linalg.norm(r) > opt.tol * theta and k < opt.max_newton:
            Q = np.concatenate([Qt, u[:, None]], axis=1)
            s, info = pcg_correction(A, theta, u, r, Q, S, R, alpha, ic, opt)
            mvp_n += info["mvp"]
            pcg_its.append(info["its"])
            exits.append(info["exit"])
            t = u + s
            u_new = t / np.linalg.norm(t)
            if Qt.shape[1]:
                u_new = u_new - Qt @ (Qt.T @ u_new)
                u_new = u_new / np.linalg.norm(u_new)
            u = u_new
            Au = _ic.spmv(A, u)
            mvp_n += 1
            theta = u @ Au
            r_new = Au - theta * u
            # the pair's second vector: w = -y with y = r_{k+1} - r_k (full
            # update) or y ~ -r_k (simplified, eq. "lastprec")
            w = r - r_new if opt.bfgs_full else r
            # Theorem 3.2: the update keeps Phat SPD when alpha = s^T w < 0
            # (s^T y > 0), which holds when the correction equation is
            # solved; a pair with alpha >= 0 (e.g. s = 0 after an immediate
            # PCG breakdown) defines no SPD update and is not stored.
            if opt.k_max > 0 and s @ w < 0:
                if len(S) == opt.k_max:
                    S.pop(0)
                    R.pop(0)
                    alpha.pop(0)
                S.append(s)
                R.append(w)
                alpha.append(s @ w)
            r = r_new
            k += 1
        lam[j] = theta
        stats["outer_its"].append(k)
        stats["pcg_its"].append(pcg_its)
        stats["exits"].append(exits)
        stats["newton_mvp"].append(mvp_n)
        stats["converged"].append(bool(np.linalg.norm(r) <= opt.tol * theta))
        stats["final_res"].append(float(np.linalg.norm(r) / theta))
        stats["last_pairs"] = (list(S), list(R))
        Qt = np.concatenate([Qt, u[:, None]], axis=1)
    V = np.stack([fix_sign(Qt[:, j]) for j in range(p)], axis=1)
    stats["ascending"] = bool(np.all(np.diff(lam) > 0))
    stats["nnz_L"] = ic.nnz
    stats["sigma"] = ic.nnz / ((A.nnz + n) // 2)
    return lam, V, stats


# ---------------------------------------------------------------------------
# Adjoint of the eigenpairs (not in the paper)
# ---------------------------------------------------------------------------

def projected_solve(A, shift: float, Q: np.ndarray, b: np.ndarray, ic, tol: float = 1e-12, maxit: int = 5000):
    """y perp Q solving (I - Q Q^T)(A - shift I)(I - Q Q^T) y = (I - Q Q^T) b.

    The same projected PCG as the correction equation, with the fixed
    preconditioner (I - Q Q^T) P0hat (I - Q Q^T) and a relative-residual exit.
    Returns (y, its).
    """
    y = np.zeros_like(b)
    g = b - Q @ (Q.T @ b)
    g0 = np.linalg.norm(g)
    if g0 == 0.0:
        return y, 0
    c = bfgs_apply(g, [], [], [], ic, Q)
    p = c.copy()
    gamma = g @ c
    for it in range(maxit):
        w = _ic.spmv(A, p) - shift * p
        delta = p @ w
        a = gamma / delta
        y = y + a * p
        g = g - a * w
        g = g - Q @ (Q.T @ g)
        if np.linalg.norm(g) <= tol * g0:
            return y, it + 1
        c = bfgs_apply(g, [], [], [], ic, Q)
        gamma_new = g @ c
        p = c + (gamma_new / gamma) * p
        gamma = gamma_new
    return y, maxit


def adjoint_grad(A, lam: np.ndarray, V: np.ndarray, gbar_lam: Optional[np.ndarray],
                 gbar_V: Optional[np.ndarray], ic, tol: float = 1e-12):
    """d loss / d A_ab for every stored entry (a, b) of A (A_ab and A_ba independent).

    Eigenvalues: d lambda_j / d A_ab = v_ja v_jb.
    Eigenvectors (unit norm, fixed sign): with xi_j = -(A - lambda_j I)^+ gbar_vj,
      xi_j = -sum_{i<=p, i!=j} v_i (v_i^T gbar_vj)/(lambda_i - lambda_j) - y_j,
      y_j perp V solving (I-VV^T)(A - lambda_j I)(I-VV^T) y_j = (I-VV^T) gbar_vj,
    and d loss / d A_ab += xi_ja v_jb.
    Pinned by central finite differences and by d lambda / d a for the
    anisotropic Laplacian (closed form).
    """
    n, p = V.shape
    rows = np.repeat(np.arange(n), np.diff(A.rowptr))
    cols = A.col.astype(np.int64)
    grad = np.zeros(A.nnz)
    if gbar_lam is not None:
        for j in range(p):
            if gbar_lam[j] != 0.0:
                grad += gbar_lam[j] * V[rows, j] * V[cols, j]
    if gbar_V is not None:
        for j in range(p):
            gv = gbar_V[:, j]
            if not np.any(gv):
                continue
            xi = np.zeros(n)
            for i in range(p):
                if i != j:
                    xi -= V[:, i] * (V[:, i] @ gv) / (lam[i] - lam[j])
            y, _ = projected_solve(A, lam[j], V, gv, ic, tol=tol)
            xi -= y
            grad += xi[rows] * V[cols, j]
    return grad
