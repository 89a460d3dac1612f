"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module builds matrices and start vectors only.  It holds none of the
eigensolver's arithmetic (no IC factor, no preconditioner, no Newton or PCG
step), so both sides of every parity test can take their inputs from here
without sharing solver code.

The paper's own test matrices (trino, hyb2d, monte-carlo, emilia-923, dblp;
Section 5, Table "list") are not available, so each workload below stands in
for one class of them with the same structure: finite-difference and finite-
element stiffness matrices of elliptic operators (SPD M-matrices, 5/7/27
entries per row) and grounded graph Laplacians (irregular degree).

Every generator is deterministic for a given seed: numpy's PCG64 bit stream
is platform independent, so the same arrays come out on x86_64 and aarch64
(floating-point post-processing may differ in the last bit across platforms,
which changes eigenvalues by ~1e-16 relative).

CSR convention used everywhere: ``rowptr`` int64 (n+1), ``col`` int32 sorted
ascending within each row, ``val`` float64; the pattern is symmetric and the
values are symmetric.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

BASE_SEED = 13121553


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray  # int64, n+1
    col: np.ndarray  # int32, nnz
    val: np.ndarray  # float64, nnz
    name: str = ""
    # Optional metadata (grid shape, coefficient fields, closed-form data).
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))

    def dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        for i in range(self.n):
            for e in range(self.rowptr[i], self.rowptr[i + 1]):
                d[i, self.col[e]] += self.val[e]
        return d


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# Generic structured-grid stencil assembly
# ---------------------------------------------------------------------------

def _stencil_csr(shape, offsets, coefs, name="", meta=None) -> CSR:
    """Assemble a CSR matrix from a structured stencil.

    ``shape`` is the grid shape in (z, y, x) order (x fastest in the natural
    numbering).  ``offsets`` is a list of (dz, dy, dx) tuples and ``coefs`` a
    list of arrays of ``shape`` holding the coefficient that couples node c
    with node c+offset.  Couplings that leave the grid are dropped (Dirichlet
    elimination).  Columns come out sorted because offsets are sorted by their
    linear displacement.
    """
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[d + 1:])) for d in range(nd)]
    lin = [sum(o[d] * strides[d] for d in range(nd)) for o in offsets]
    order = np.argsort(lin, kind="stable")
    idx = np.indices(shape).reshape(nd, -1)
    cols = []
    vals = []
    masks = []
    node = np.arange(n, dtype=np.int64)
    for t in order:
        o = offsets[t]
        ok = np.ones(n, dtype=bool)
        for d in range(nd):
            q = idx[d] + o[d]
            ok &= (q >= 0) & (q < shape[d])
        masks.append(ok)
        cols.append(node + lin[t])
        vals.append(np.asarray(coefs[t], dtype=np.float64).reshape(-1))
    M = np.stack(masks, axis=1)  # n x s
    C = np.stack(cols, axis=1)
    V = np.stack(vals, axis=1)
    counts = M.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    col = C[M].astype(np.int32)
    val = V[M]
    return CSR(n, rowptr, col, val, name=name, meta=dict(meta or {}))


# ---------------------------------------------------------------------------
# Workload 1: 2D anisotropic Dirichlet Laplacian (closed-form spectrum)
# ---------------------------------------------------------------------------

def laplacian_2d_aniso(nx: int = 30, ny: int = 37, a: float = 1.0, b: float = 1.7) -> CSR:
    """5-point stencil a*(-u_xx) + b*(-u_yy) on an nx x ny grid, h = 1.

    Its eigenvalues are a(2-2cos(k pi/(nx+1))) + b(2-2cos(l pi/(ny+1))),
    k=1..nx, l=1..ny, with separable sine eigenvectors (stored in ``meta``
    as the data needed to evaluate them).
    """
    shape = (ny, nx)
    one = np.ones(shape)
    offsets = [(0, 0), (0, -1), (0, 1), (-1, 0), (1, 0)]
    coefs = [(2 * a + 2 * b) * one, -a * one, -a * one, -b * one, -b * one]
    return _stencil_csr(shape, offsets, coefs, name=f"aniso2d_{nx}x{ny}",
                        meta=dict(nx=nx, ny=ny, a=a, b=b))


def laplacian_2d_aniso_eigs(nx: int, ny: int, a: float, b: float) -> np.ndarray:
    k = np.arange(1, nx + 1)
    l = np.arange(1, ny + 1)
    ex = a * (2 - 2 * np.cos(k * np.pi / (nx + 1)))
    ey = b * (2 - 2 * np.cos(l * np.pi / (ny + 1)))
    return np.sort((ex[:, None] + ey[None, :]).ravel())


def laplacian_2d_aniso_eigvec(nx: int, ny: int, k: int, l: int) -> np.ndarray:
    """Unit eigenvector sin(k pi x/(nx+1)) sin(l pi y/(ny+1)), x fastest."""
    x = np.arange(1, nx + 1)
    y = np.arange(1, ny + 1)
    v = np.outer(np.sin(l * np.pi * y / (ny + 1)), np.sin(k * np.pi * x / (nx + 1))).ravel()
    return v / np.linalg.norm(v)


def tridiag(n: int, d: float = 2.0, o: float = -1.0) -> CSR:
    one = np.ones((n,))
    return _stencil_csr((n,), [(0,), (-1,), (1,)], [d * one, o * one, o * one], name=f"tridiag{n}")


# ---------------------------------------------------------------------------
# Workload 2: 3D 7-point variable-coefficient diffusion, Gaussian log-field
# ---------------------------------------------------------------------------

def gaussian_field(shape, corr_len: float, rng: np.random.Generator) -> np.ndarray:
    """Zero-mean, unit sample-std Gaussian random field on cells.

    White noise on a padded grid is convolved with exp(-d^2/l^2) along each
    axis; the result has squared-exponential covariance exp(-d^2/(2 l^2)).
    """
    from scipy.ndimage import convolve1d

    pad = int(np.ceil(4 * corr_len))
    big = tuple(s + 2 * pad for s in shape)
    w = rng.standard_normal(big)
    d = np.arange(-pad, pad + 1, dtype=np.float64)
    ker = np.exp(-(d * d) / (corr_len * corr_len))
    for ax in range(len(shape)):
        w = convolve1d(w, ker, axis=ax, mode="constant")
    sl = tuple(slice(pad, pad + s) for s in shape)
    g = w[sl]
    g = g - g.mean()
    g = g / g.std()
    return np.ascontiguousarray(g)


def diffusion_3d_7pt(nx: int = 100, ny: Optional[int] = None, nz: Optional[int] = None,
                     corr_len: float = 8.0, sigma: float = 1.0, seed: int = BASE_SEED + 2) -> CSR:
    """Cell-centred 7-point diffusion with face coefficients exp(mean of g).

    g is a Gaussian field (std ``sigma``, correlation length ``corr_len``
    cells).  An interior face between cells c and c' gets exp((g_c+g_c')/2);
    a Dirichlet boundary face of cell c gets exp(g_c).
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    shape = (nz, ny, nx)
    rng = rng_for(seed)
    g = sigma * gaussian_field(shape, corr_len, rng)
    eg = np.exp(g)
    diag = np.zeros(shape)
    offsets = [(0, 0, 0)]
    coefs = [diag]
    for ax in range(3):
        for sgn in (-1, 1):
            o = [0, 0, 0]
            o[ax] = sgn
            # neighbour g (clamped at the boundary; boundary couplings are
            # dropped by the assembler but their face still enters the diagonal)
            nb = np.roll(g, -sgn, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = -1 if sgn == 1 else 0
            face = np.exp(0.5 * (g + nb))
            face[tuple(edge)] = eg[tuple(edge)]
            diag += face
            offsets.append(tuple(o))
            coefs.append(-face)
    return _stencil_csr(shape, offsets, coefs, name=f"diff3d7_{nx}x{ny}x{nz}",
                        meta=dict(shape=shape, g=g))


# ---------------------------------------------------------------------------
# Workload 3: 2D 5-point diffusion with log-normal cell coefficients
# ---------------------------------------------------------------------------

def diffusion_2d_faces(kappa: np.ndarray):
    """Face coefficients of the two-point flux scheme on cells (ny, nx).

    Interior face: harmonic mean 2 k1 k2/(k1+k2).  Boundary face: k_c.
    Returns (fx, fy): fx[j, i] couples cell (j,i) with (j,i+1) for
    i < nx-1; fx[:, -1] is the right boundary face.  Likewise fy.  Left and
    bottom boundary faces are kappa[:, 0] and kappa[0, :].
    """
    k1 = kappa[:, :-1]
    k2 = kappa[:, 1:]
    fx = 2 * k1 * k2 / (k1 + k2)
    k1 = kappa[:-1, :]
    k2 = kappa[1:, :]
    fy = 2 * k1 * k2 / (k1 + k2)
    return fx, fy


def diffusion_2d_from_kappa(kappa: np.ndarray, name: str = "") -> CSR:
    ny, nx = kappa.shape
    fx, fy = diffusion_2d_faces(kappa)
    west = np.empty_like(kappa)
    east = np.empty_like(kappa)
    south = np.empty_like(kappa)
    north = np.empty_like(kappa)
    west[:, 1:] = fx
    west[:, 0] = kappa[:, 0]
    east[:, :-1] = fx
    east[:, -1] = kappa[:, -1]
    south[1:, :] = fy
    south[0, :] = kappa[0, :]
    north[:-1, :] = fy
    north[-1, :] = kappa[-1, :]
    diag = west + east + south + north
    offsets = [(0, 0), (0, -1), (0, 1), (-1, 0), (1, 0)]
    coefs = [diag, -west, -east, -south, -north]
    return _stencil_csr((ny, nx), offsets, coefs, name=name or f"diff2d5_{nx}x{ny}",
                        meta=dict(shape=(ny, nx), kappa=kappa))


def diffusion_2d_values_torch(kappa):
    """The stored values of diffusion_2d_from_kappa(kappa), in its CSR order,
    as a differentiable function of the torch tensor kappa (ny, nx).

    Used to carry gradients with respect to the matrix entries over to the
    cell coefficients (chain rule through the harmonic-mean faces)."""
    import torch

    ny, nx = kappa.shape
    fx = 2 * kappa[:, :-1] * kappa[:, 1:] / (kappa[:, :-1] + kappa[:, 1:])
    fy = 2 * kappa[:-1, :] * kappa[1:, :] / (kappa[:-1, :] + kappa[1:, :])
    west = torch.cat([kappa[:, :1], fx], dim=1)
    east = torch.cat([fx, kappa[:, -1:]], dim=1)
    south = torch.cat([kappa[:1, :], fy], dim=0)
    north = torch.cat([fy, kappa[-1:, :]], dim=0)
    diag = west + east + south + north
    # entries per row in the assembler's order: south, west, diagonal, east, north
    jj, ii = torch.meshgrid(torch.arange(ny), torch.arange(nx), indexing="ij")
    cols = [(-south, jj > 0), (-west, ii > 0), (diag, torch.ones_like(ii, dtype=torch.bool)),
            (-east, ii < nx - 1), (-north, jj < ny - 1)]
    V = torch.stack([c.reshape(-1) for c, _ in cols], dim=1)
    M = torch.stack([m.reshape(-1) for _, m in cols], dim=1)
    return V[M]


def diffusion_2d_lognormal(nx: int = 600, ny: int = 700, sigma: float = 0.5,
                           seed: int = BASE_SEED + 3) -> CSR:
    rng = rng_for(seed)
    kappa = np.exp(sigma * rng.standard_normal((ny, nx)))
    A = diffusion_2d_from_kappa(kappa, name=f"diff2d5_{nx}x{ny}")
    # loss weights w ~ U[0,1] for the eigenvector term of the loss
    A.meta["w"] = rng.random(nx * ny)
    return A


# ---------------------------------------------------------------------------
# Workload 4: grounded random geometric graph Laplacians
# ---------------------------------------------------------------------------

def geometric_graph_laplacian(n: int, seed: int, shift: float = 1e-3, avg_degree: float = 10.0) -> CSR:
    """L + shift*I for a random geometric graph in the unit square.

    Points are uniform, edges join pairs closer than sqrt(avg_degree/(pi n)),
    weights are U[0.5, 2].  Only the largest connected component is kept, so
    the smallest eigenvalue is exactly ``shift`` with the constant vector.
    """
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    from scipy.spatial import cKDTree

    rng = rng_for(seed)
    pts = rng.random((n, 2))
    radius = np.sqrt(avg_degree / (np.pi * n))
    pairs = cKDTree(pts).query_pairs(radius, output_type="ndarray")
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    w = rng.uniform(0.5, 2.0, size=len(pairs))
    W = sp.coo_matrix((w, (pairs[:, 0], pairs[:, 1])), shape=(n, n)).tocsr()
    W = W + W.T
    ncomp, lab = connected_components(W, directed=False)
    big = np.argmax(np.bincount(lab))
    keep = np.flatnonzero(lab == big)
    W = W[keep][:, keep].tocsr()
    m = W.shape[0]
    deg = np.asarray(W.sum(axis=1)).ravel()
    L = sp.diags(deg + shift) - W
    L = L.tocsr()
    L.sort_indices()
    return CSR(m, L.indptr.astype(np.int64), L.indices.astype(np.int32), L.data.astype(np.float64),
               name=f"rgg{n}_s{seed}", meta=dict(shift=shift, n_points=n))


def graph_batch(count: int = 256, nmin: int = 2000, nmax: int = 60000, seed: int = BASE_SEED + 4):
    rng = rng_for(seed)
    sizes = rng.integers(nmin, nmax + 1, size=count)
    return [geometric_graph_laplacian(int(sizes[b]), seed * 1000 + b) for b in range(count)]


def graph_batch_problem(b: int, count: int = 256, nmin: int = 2000, nmax: int = 60000,
                        seed: int = BASE_SEED + 4) -> CSR:
    """Problem b of graph_batch(count, ...), built alone."""
    sizes = rng_for(seed).integers(nmin, nmax + 1, size=count)
    return geometric_graph_laplacian(int(sizes[b]), seed * 1000 + b)


def graph_batch_start(A: CSR, b: int, p: int = 4) -> np.ndarray:
    """Start vectors of problem b of the batched workload (p per problem)."""
    return start_vectors(A.n, p, BASE_SEED + 400 + b)


# ---------------------------------------------------------------------------
# Workload 5: trilinear hexahedral Poisson stiffness, 27-point
# ---------------------------------------------------------------------------

def hex8_reference_stiffness() -> np.ndarray:
    """8x8 stiffness of grad(phi_a).grad(phi_b) on the unit cube.

    Trilinear shape functions, exact 2x2x2 Gauss quadrature.  Local node
    index a = ax + 2 ay + 4 az with corner (ax, ay, az) in {0,1}^3.
    """
    gp = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    K = np.zeros((8, 8))
    corners = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]

    def phi1(c, t):
        return t if c else 1.0 - t

    def dphi1(c):
        return 1.0 if c else -1.0

    for x in gp:
        for y in gp:
            for z in gp:
                G = np.zeros((8, 3))
                for a, (cx, cy, cz) in enumerate(corners):
                    G[a, 0] = dphi1(cx) * phi1(cy, y) * phi1(cz, z)
                    G[a, 1] = phi1(cx, x) * dphi1(cy) * phi1(cz, z)
                    G[a, 2] = phi1(cx, x) * phi1(cy, y) * dphi1(cz)
                K += 0.125 * G @ G.T
    return K


def _hex_coefs(kappa, zeros):
    """Stencil coefficients of the hex stiffness, one (m, m, m) array per
    offset (dz, dy, dx) in lexicographic order, from the element
    coefficients kappa ((m+1)^3, numpy or torch: the same operations in the
    same order, so both give identical values)."""
    ne = kappa.shape[0]
    m = ne - 1
    Kr = hex8_reference_stiffness()
    h = 1.0 / ne
    offsets = []
    coefs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                c = zeros((m, m, m))
                # elements around node N = (K, J, I) in 1..m: e = N - a, a in {0,1}^3
                for az in (0, 1):
                    for ay in (0, 1):
                        for ax in (0, 1):
                            bz, by, bx = az + dz, ay + dy, ax + dx
                            if not (0 <= bz <= 1 and 0 <= by <= 1 and 0 <= bx <= 1):
                                continue
                            la = ax + 2 * ay + 4 * az
                            lb = bx + 2 * by + 4 * bz
                            ke = kappa[1 - az:ne - az, 1 - ay:ne - ay, 1 - ax:ne - ax]
                            c = c + ke * float(h * Kr[la, lb])
                offsets.append((dz, dy, dx))
                coefs.append(c)
    return offsets, coefs, h


def hex_poisson_from_kappa(kappa: np.ndarray, name: str = "") -> CSR:
    """27-point stiffness on the m^3 interior nodes of an (m+1)^3 hex mesh
    with element coefficients kappa (shape (m+1)^3, index (ez, ey, ex)).

    Mesh width h = 1/(m+1), so the element matrix is h*kappa_e*K_ref;
    boundary nodes are eliminated (homogeneous Dirichlet).  All 27 couplings
    are kept in the pattern even where the assembled value is (numerically)
    zero.
    """
    m = kappa.shape[0] - 1
    offsets, coefs, h = _hex_coefs(kappa, np.zeros)
    return _stencil_csr((m, m, m), offsets, coefs, name=name or f"hex27_{m}",
                        meta=dict(shape=(m, m, m), kappa=kappa, h=h))


def hex_poisson_values_torch(kappa):
    """The stored values of hex_poisson_from_kappa(kappa), in its CSR order,
    as a differentiable function of the torch tensor kappa ((m+1)^3).

    Used to carry gradients with respect to the matrix entries over to the
    element coefficients (chain rule through the assembly)."""
    import torch

    m = kappa.shape[0] - 1
    offsets, coefs, _ = _hex_coefs(kappa, lambda s: torch.zeros(s, dtype=kappa.dtype))
    idx = np.indices((m, m, m)).reshape(3, -1)
    masks = []
    for o in offsets:
        ok = np.ones(m ** 3, dtype=bool)
        for d in range(3):
            q = idx[d] + o[d]
            ok &= (q >= 0) & (q < m)
        masks.append(ok)
    V = torch.stack([c.reshape(-1) for c in coefs], dim=1)
    M = torch.from_numpy(np.stack(masks, axis=1))
    return V[M]


def hex_poisson_27pt(m: int = 96, sigma: float = 1.0, seed: int = BASE_SEED + 5) -> CSR:
    """hex_poisson_from_kappa with element coefficients kappa_e =
    exp(sigma N(0,1)) on an (m+1)^3 element grid (m^3 unknowns)."""
    rng = rng_for(seed)
    ne = m + 1
    kappa = np.exp(sigma * rng.standard_normal((ne, ne, ne)))  # (ez, ey, ex)
    return hex_poisson_from_kappa(kappa, name=f"hex27_{m}")


# ---------------------------------------------------------------------------
# Start vectors and the named workloads
# ---------------------------------------------------------------------------

# ---------------------------------------------------------------------------
# Symmetric reorderings (inputs to both sides: the oracle factors the
# permuted matrix P A P^T that the library builds from the same definition)
# ---------------------------------------------------------------------------

def multicolor_order(A: CSR, distance: int = 2, return_colors: bool = False):
    """Greedy colouring in natural order: row i takes the smallest colour not
    held by an already coloured row j != i with A_ij != 0 (distance 1) or
    reachable through one such row (distance 2).  Returns (perm, ncolors),
    perm listing the rows by colour, ascending row inside a colour (and the
    colour of every row when return_colors)."""
    n = A.n
    rp, ci = A.rowptr, A.col
    color = np.full(n, -1, np.int64)
    for i in range(n):
        nb = ci[rp[i]:rp[i + 1]]
        if distance == 2:
            nb = np.concatenate([nb] + [ci[rp[j]:rp[j + 1]] for j in nb])
        cs = color[nb[nb != i]]
        used = set(cs[cs >= 0].tolist())
        c = 0
        while c in used:
            c += 1
        color[i] = c
    perm = np.argsort(color, kind="stable").astype(np.int32)
    if return_colors:
        return perm, int(color.max()) + 1, color
    return perm, int(color.max()) + 1


def permute(A: CSR, perm) -> CSR:
    """P A P^T with row k = row perm[k] of A, columns ascending."""
    import scipy.sparse as sp

    S = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.n, A.n))
    B = S[perm][:, perm].tocsr()
    B.sort_indices()
    return CSR(A.n, B.indptr.astype(np.int64), B.indices.astype(np.int32), B.data.copy(),
               name=A.name + "_perm", meta=dict(A.meta))


def count_sketch_hash(n: int, K: int, seed: int):
    """Seeded CountSketch of R^n into R^K: a bucket in [0, K) and a sign
    +-1 for every coordinate.  Used to compare long vectors (eigenvectors
    at n ~ 1e6) through K numbers: for x in R^n the sketch S x has
    E ||S x||^2 = ||x||^2, with relative spread about sqrt(2/K) for vectors
    whose mass is spread over many coordinates."""
    rng = rng_for(seed + 9_000_000)
    bucket = rng.integers(0, K, size=n)
    sign = rng.integers(0, 2, size=n).astype(np.float64) * 2.0 - 1.0
    return bucket, sign


def count_sketch(x: np.ndarray, bucket: np.ndarray, sign: np.ndarray, K: int) -> np.ndarray:
    """S x for the hash of count_sketch_hash: y[b] = sum over i with
    bucket[i] = b of sign[i] x[i]."""
    return np.bincount(bucket, weights=sign * np.asarray(x, dtype=np.float64), minlength=K)


def start_vectors(n: int, p: int, seed: int) -> np.ndarray:
    """p seeded N(0,1) start vectors, shape (p, n), one per wanted eigenpair."""
    return rng_for(seed + 7_000_000).standard_normal((p, n))


WORKLOADS = {
    # name: (builder, solver settings)
    "aniso2d_30x37": dict(build=lambda: laplacian_2d_aniso(30, 37, 1.0, 1.7), p=5, lfil=5, tau_ic=1e-2,
                          tol=1e-10, seed=BASE_SEED + 1),
    "diff3d7_100": dict(build=lambda: diffusion_3d_7pt(100), p=10, lfil=10, tau_ic=1e-3, tol=1e-8,
                        seed=BASE_SEED + 2),
    # the oracle needs up to 99 Newton steps here (eigenpair 6), the mixed
    # GPU run a few more
    "diff2d5_600x700": dict(build=lambda: diffusion_2d_lognormal(600, 700), p=8, lfil=30, tau_ic=1e-2,
                            tol=1e-8, seed=BASE_SEED + 3, max_newton=200),
    # eigenpairs 18-20 form a cluster (relative gaps 6e-4 and 1.3e-3) that
    # needs more than the default 100 Newton steps
    "hex27_96": dict(build=lambda: hex_poisson_27pt(96), p=20, lfil=20, tau_ic=1e-4, tol=1e-8,
                     seed=BASE_SEED + 5, max_newton=400),
    # reduced sizes of the same recipes (tests)
    "diff3d7_24": dict(build=lambda: diffusion_3d_7pt(24, corr_len=8.0), p=4, lfil=10, tau_ic=1e-3,
                       tol=1e-8, seed=BASE_SEED + 12),
    "diff2d5_60x70": dict(build=lambda: diffusion_2d_lognormal(60, 70), p=4, lfil=30, tau_ic=1e-2,
                          tol=1e-8, seed=BASE_SEED + 13),
    "hex27_16": dict(build=lambda: hex_poisson_27pt(16), p=5, lfil=20, tau_ic=1e-4, tol=1e-8,
                     seed=BASE_SEED + 15),
    "rgg3000": dict(build=lambda: geometric_graph_laplacian(3000, BASE_SEED + 14), p=4, lfil=30, tau_ic=1e-2,
                    tol=1e-8, seed=BASE_SEED + 14),
}


def workload(name: str):
    """Return (A, settings dict) for a named workload."""
    w = WORKLOADS[name]
    A = w["build"]()
    settings = {k: v for k, v in w.items() if k != "build"}
    return A, settings
