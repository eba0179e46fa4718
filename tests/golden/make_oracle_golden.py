"""Write tests/golden/*_oracle.json: FP64 oracle results on the full-size
synthetic workloads, for the GPU tests and the benchmark's CPU baseline.

Calls only oracle/ (and the seeded generators in workloads/).  Usage:
    python tests/golden/make_oracle_golden.py c2     # 128^3 27-point mesh
    python tests/golden/make_oracle_golden.py c1     # 64 x 64 5-point mesh
    python tests/golden/make_oracle_golden.py c3     # R-MAT scale 22, largest component
    python tests/golden/make_oracle_golden.py amg    # 128^3 27-point mesh, multigrid preconditioner
    python tests/golden/make_oracle_golden.py c4 [i ...]  # graphs i of the 2000-graph RGG batch
                                                          # (default: the largest, median and smallest)
"""

from __future__ import annotations

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402

CASES = {
    "c1": dict(graph=lambda: workloads.grid2d(64, 64), K=4, problem="combinatorial", precond="jacobi",
               tol=1e-2, seed=1, poly_degree=25, desc="2D 5-point 64x64, combinatorial, Jacobi, K=4, tol 1e-2"),
    "c2": dict(graph=lambda: workloads.grid3d(128, 128, 128, 27), K=64, problem="generalized", precond="poly",
               tol=1e-3, seed=2, poly_degree=25,
               desc="3D 27-point 128^3, generalized, polynomial degree 25, K=64, tol 1e-3"),
    "c3": dict(graph=lambda: workloads.rmat(22, 16, 0.57, 0.19, 0.19, seed=3), K=256, problem="normalized",
               precond="jacobi", tol=1e-2, seed=3, poly_degree=25,
               desc="R-MAT scale 22 (a,b,c = .57,.19,.19), largest component, normalized, Jacobi, K=256, tol 1e-2"),
    "amg": dict(graph=lambda: workloads.grid3d(128, 128, 128, 27), K=64, problem="combinatorial", precond="amg",
                tol=1e-2, seed=2, poly_degree=25,
                desc="3D 27-point 128^3, combinatorial, aggregation multigrid, K=64, tol 1e-2"),
}


# the 2000-graph batch: the three largest graphs, three of median size and two
# of the smallest, each partitioned alone by the oracle with the batch's options
C4 = dict(K=8, problem="combinatorial", precond="poly", poly_degree=25, tol=1e-3, seed=4, count=2000, maxit=3000)


def c4_sizes() -> np.ndarray:
    """n_i of the batch (workloads.rgg_batch's rule), without drawing the graphs."""
    u = workloads.graphs.uniform01(4, 61, C4["count"])
    return np.floor(np.exp(np.log(1e3) + u * np.log(200.0))).astype(np.int64)


def c4_indices() -> list:
    order = [int(i) for i in np.argsort(c4_sizes(), kind="stable")]
    mid = len(order) // 2
    return order[-3:] + order[mid - 1:mid + 2] + order[:2]


def run_c4(indices=None) -> dict:
    """The oracle on graphs `indices` of the batch (default: c4_indices()),
    each merged into c4_oracle.json as soon as it finishes (under a file lock,
    so that several processes can share the list)."""
    import fcntl
    sizes = c4_sizes()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c4_oracle.json")
    out = None
    for i in (indices if indices else c4_indices()):
        g = workloads.rgg(int(sizes[i]), seed=4 + i)
        t0 = time.time()
        r = oracle.partition(g, C4["K"], problem=C4["problem"], precond=C4["precond"], tol=C4["tol"],
                             seed=C4["seed"], poly_degree=C4["poly_degree"], maxit=C4["maxit"])
        entry = {"index": i, "n_drawn": int(sizes[i]), "n": g.n, "nnz": g.nnz,
                 "eigenvalues": [float(v) for v in r.eigenvalues], "iterations": int(r.iterations),
                 "status": r.status, "cut": float(r.cut), "imbalance": float(r.imbalance),
                 "oracle_seconds": round(time.time() - t0, 2)}
        print(i, g.n, r.iterations, r.status, r.cut, entry["oracle_seconds"], flush=True)
        with open(path + ".lock", "w") as lk:
            fcntl.flock(lk, fcntl.LOCK_EX)
            out = {"workload": "2000 RGGs (workloads.rgg_batch), combinatorial, polynomial degree 25, K=8, tol 1e-3",
                   **C4, "graphs": []}
            if os.path.exists(path):
                with open(path) as f:
                    out["graphs"] = [e for e in json.load(f)["graphs"] if e["index"] != i]
            out["graphs"] = sorted(out["graphs"] + [entry], key=lambda e: -e["n"])
            with open(path, "w") as f:
                json.dump(out, f, indent=1)
    return out


def run(name: str) -> dict:
    c = CASES[name]
    g = c["graph"]()
    t0 = time.time()
    r = oracle.partition(g, c["K"], problem=c["problem"], precond=c["precond"], tol=c["tol"], seed=c["seed"],
                         poly_degree=c["poly_degree"])
    dt = time.time() - t0
    out = {
        "workload": c["desc"], "n": g.n, "nnz": g.nnz, "K": c["K"], "seed": c["seed"],
        "eigenvalues": [float(v) for v in r.eigenvalues], "resnorm": [float(v) for v in r.resnorm],
        "iterations": int(r.iterations), "status": r.status, "cut": float(r.cut), "cut_twice": float(r.cut_twice),
        "imbalance": float(r.imbalance), "poly_roots": [float(v) for v in r.roots],
        "oracle_seconds": round(dt, 2),
        "part_weights": [int(v) for v in np.bincount(r.parts, minlength=c["K"])],
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return out


if __name__ == "__main__":
    for name in sys.argv[1:] or ["c1", "c2"]:
        if name == "c4":
            run_c4([int(v) for v in sys.argv[2:]])
            break
        res = run(name)
        print(name, res["iterations"], res["eigenvalues"], res["cut"], res["oracle_seconds"])
