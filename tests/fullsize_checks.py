"""Shared checks of the full-size parity tests (not a test module).

Eigenvectors at n ~ 1e6 are compared with the stored oracle run through a
seeded CountSketch (workloads.count_sketch, K numbers per vector; its
E ||S x||^2 = ||x||^2 and, for vectors spread over many entries, ||S x||
stays within 25 % of ||x|| at K = 256: tests/test_oracle_pins.py), which
estimates ||v - v_oracle|| = 2 sin(angle / 2) without storing the vectors.

Bound on the angle between the two sides: each side's unit vector v with
Rayleigh quotient theta and residual ||A v - theta v|| = res * theta has
sin angle(v, true eigenvector) <= res * theta / delta, delta the distance
from theta to the rest of the spectrum (Davis-Kahan); the two angles add.
delta is taken from the computed eigenvalues, a lower bound for every pair
but the last (whose gap to lambda_{p+1} is not known; there the bound uses
lambda_p - lambda_{p-1} only)."""
import numpy as np

import workloads as W

SKETCH_SLACK = 1.25


def sketch_angles(A, V, gold):
    K = gold["sketch_K"]
    bucket, sign = W.count_sketch_hash(A.n, K, gold["sketch_seed"])
    out = []
    for j in range(len(gold["lam"])):
        sk = W.count_sketch(V[j], bucket, sign, K)
        ref = np.array(gold["sketch_V"][j])
        out.append(float(min(np.linalg.norm(sk - ref), np.linalg.norm(sk + ref))))
    return np.array(out)


def angle_bounds(gold, res_gpu):
    glam = np.array(gold["lam"])
    res_or = np.array(gold["oracle_stats"]["final_res"])
    p = len(glam)
    b = np.zeros(p)
    for j in range(p):
        gap = np.min(np.abs(np.delete(glam, j) - glam[j]))
        b[j] = (res_gpu[j] + res_or[j]) * glam[j] / gap
    return b


def check_eigenvectors(A, V, gold, res_gpu, label):
    """Assert every sketched distance within its bound (with the sketch's
    slack); print the table.  Returns (angles, bounds)."""
    ang = sketch_angles(A, V, gold)
    bnd = angle_bounds(gold, res_gpu)
    print(f"\n{label}: eigenvector distance to the oracle (CountSketch) and its residual bound")
    for j, (a, b) in enumerate(zip(ang, bnd)):
        print(f"  pair {j + 1:2d}  angle ~ {a:.2e}  bound {b:.2e}")
    assert np.all(ang <= SKETCH_SLACK * bnd), (ang, bnd)
    return ang, bnd


def cluster_subspace_angles(A, V, gold, res_gpu, rel_gap=0.02):
    """Eigenvalue clusters (maximal runs of computed eigenvalues whose
    consecutive relative gaps are below rel_gap): the distance between the
    spans of the GPU's and the oracle's eigenvectors of each cluster, as the
    sketched residual of the best rotation (orthogonal Procrustes) of the
    oracle's onto the GPU's, and its bound (res_gpu + res_oracle) lambda_max
    / delta, delta the distance from the cluster to the other computed
    eigenvalues (the subspace is well conditioned when an individual
    eigenvector of the cluster is not).  Returns [(pairs, angle, bound)]."""
    K = gold["sketch_K"]
    bucket, sign = W.count_sketch_hash(A.n, K, gold["sketch_seed"])
    glam = np.array(gold["lam"])
    res_or = np.array(gold["oracle_stats"]["final_res"])
    p = len(glam)
    out = []
    j = 0
    while j < p:
        e = j + 1
        while e < p and (glam[e] - glam[e - 1]) / glam[e] < rel_gap:
            e += 1
        if e - j >= 2:
            idx = list(range(j, e))
            Yg = np.stack([W.count_sketch(V[i], bucket, sign, K) for i in idx], axis=1)
            Yo = np.stack([np.array(gold["sketch_V"][i]) for i in idx], axis=1)
            U, _, Vt = np.linalg.svd(Yo.T @ Yg)
            ang = float(np.linalg.norm(Yg - Yo @ (U @ Vt)))
            rest = np.delete(glam, idx)
            delta = float(np.min(np.abs(rest[:, None] - glam[idx][None, :]))) if len(rest) else np.inf
            bnd = float(np.sqrt(len(idx)) * max(res_gpu[i] + res_or[i] for i in idx) * glam[e - 1] / delta)
            out.append(([i + 1 for i in idx], ang, bnd))
        j = e
    return out


def check_clusters(A, V, gold, res_gpu, label):
    """Assert each cluster's subspace distance within its bound (sketch
    slack included) and within 1e-6 wherever that bound allows; print."""
    rows = cluster_subspace_angles(A, V, gold, res_gpu)
    print(f"\n{label}: eigenvalue clusters, subspace distance to the oracle's (CountSketch) and its bound")
    for pairs, a, b in rows:
        print(f"  pairs {pairs[0]}-{pairs[-1]}  distance ~ {a:.2e}  bound {b:.2e}")
        assert a <= SKETCH_SLACK * b, (pairs, a, b)
        if b <= 1e-6:
            assert a <= 1e-6, (pairs, a)
    return rows
