"""Write the stored expected values used by the full-size parity tests.

Every value comes from the oracle (``oracle/``) run on the seeded workloads
of ``workloads/``; nothing here calls the CUDA library.  Usage:

    python tests/golden/make_golden.py [--threads T] [--out DIR] diff3d7_100 [more workload names]

--threads fixes the BLAS thread count of the oracle's dot products (the
summation order, hence the last bits, depends on it; on the 27-point
workload's eigenvalue cluster 18-20 that changes the Newton path); the count
used is stored in the file.

Each run writes tests/golden/<name>.json with the eigenvalues, the oracle's
iteration counts, a seeded sample of eigenvector entries and a seeded
CountSketch (workloads.count_sketch) of every eigenvector (sign convention:
entry of largest modulus positive), plus the loss gradient with respect to
the cell or element coefficients for the 2D diffusion and hex workloads.
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def kappa_gradient(A, lam, V, opt):
    """Gradient of loss = sum lambda_j + sum_i w_i (v_1)_i^2 with respect to the
    cell coefficients, by the oracle's adjoint and the chain rule through
    the assembly (torch CPU autograd), sampled at 64 seeded cells."""
    import torch

    p = len(lam)
    ic = O.ic_factor(A, opt.lfil, opt.tau_ic)
    w = A.meta["w"]
    gl = np.ones(p)
    gV = np.zeros((A.n, p))
    gV[:, 0] = 2 * w * V[:, 0]
    gA = O.adjoint_grad(A, lam, V, gl, gV, ic)
    kappa = torch.tensor(A.meta["kappa"], dtype=torch.float64, requires_grad=True)
    vals = W.diffusion_2d_values_torch(kappa)
    (gk,) = torch.autograd.grad(vals, kappa, grad_outputs=torch.tensor(gA))
    gk = gk.numpy().ravel()
    rng = W.rng_for(4242)
    cells = np.sort(rng.choice(A.n, size=64, replace=False))
    loss = float(lam.sum() + w @ (V[:, 0] ** 2))
    return dict(loss=loss, grad_cells=[int(c) for c in cells], grad_kappa=[float(gk[c]) for c in cells],
                grad_kappa_norm=float(np.linalg.norm(gk)))


def hex_kappa_gradient(A, lam, V):
    """Gradient of loss = sum lambda_j with respect to the element
    coefficients of the hex stiffness: d lambda_j / d A_ab = v_ja v_jb (the
    oracle's adjoint with no eigenvector term), carried through the assembly
    by torch CPU autograd; sampled at 64 seeded elements."""
    import torch

    p = len(lam)
    gA = O.adjoint_grad(A, lam, V, np.ones(p), None, None)
    kappa = torch.tensor(A.meta["kappa"], dtype=torch.float64, requires_grad=True)
    vals = W.hex_poisson_values_torch(kappa)
    (gk,) = torch.autograd.grad(vals, kappa, grad_outputs=torch.tensor(gA))
    gk = gk.numpy().ravel()
    rng = W.rng_for(5252)
    elems = np.sort(rng.choice(gk.size, size=64, replace=False))
    return dict(loss=float(lam.sum()), grad_elems=[int(e) for e in elems], grad_kappa=[float(gk[e]) for e in elems],
                grad_kappa_norm=float(np.linalg.norm(gk)),
                grad_kappa_euler=float(A.meta["kappa"].ravel() @ gk))


SKETCH_K = 256


def main(names, threads=None, out_dir=HERE):
    if threads:
        from threadpoolctl import threadpool_limits

        threadpool_limits(limits=threads, user_api="blas")
    for name in names:
        if name.startswith("graph_batch_"):
            # problem b of the batched workload, its own start vectors
            b = int(name.rsplit("_", 1)[1])
            A = W.graph_batch_problem(b)
            st = dict(p=4, lfil=30, tau_ic=1e-2, tol=1e-8, max_newton=400, seed=W.BASE_SEED + 400 + b)
            X0 = W.graph_batch_start(A, b, 4)
        else:
            A, st = W.workload(name)
            X0 = W.start_vectors(A.n, st["p"], st["seed"])
        p = st["p"]
        opt = O.OracleOptions(tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"],
                              max_newton=st.get("max_newton", 100))
        t0 = time.time()
        lam, V, stats = O.dacg_newton(A, p, X0, opt)
        sec = time.time() - t0
        rng = W.rng_for(st["seed"] + 99)
        idx = np.sort(rng.choice(A.n, size=64, replace=False))
        out = dict(workload=name, n=A.n, nnz=A.nnz, p=p, tol=st["tol"], lfil=st["lfil"], tau_ic=st["tau_ic"],
                   lam=[float(x) for x in lam], sample_index=[int(i) for i in idx],
                   sample_V=[[float(V[i, j]) for i in idx] for j in range(p)],
                   oracle_seconds=sec, oracle_stats={k: stats[k] for k in
                                                     ("dacg_its", "outer_its", "pcg_its", "converged", "final_res",
                                                      "ascending", "nnz_L", "sigma")},
                   blas_threads=threads)
        if name.startswith("graph_batch_"):
            out.update(max_newton=st["max_newton"])
        # CountSketch of every eigenvector (sign convention applied): the
        # full-size tests compare sketches, which estimate ||v_gpu - v_oracle||
        bucket, sign = W.count_sketch_hash(A.n, SKETCH_K, st["seed"])
        out.update(sketch_K=SKETCH_K, sketch_seed=st["seed"],
                   sketch_V=[[float(x) for x in W.count_sketch(V[:, j], bucket, sign, SKETCH_K)] for j in range(p)])
        if name.startswith("diff2d5"):
            out.update(kappa_gradient(A, lam, V, opt))
        if name.startswith("hex27"):
            out.update(hex_kappa_gradient(A, lam, V))
        with open(os.path.join(out_dir, f"{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print(name, sec, lam)


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--out", default=HERE)
    ap.add_argument("names", nargs="+")
    a = ap.parse_args()
    main(a.names, a.threads, a.out)
