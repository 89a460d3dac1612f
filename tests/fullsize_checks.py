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
