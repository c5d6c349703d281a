"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Every value in these files comes from ``oracle/`` (and the seeded inputs of
``fieldgen/``), never from the CUDA path. Run from the repository root:

    python tests/golden/make_golden.py

tiny_4x4x4x4_fgmresdr.json — the tiny workload (4^4 lattice, eps 0.3, seed 0,
m0 = -0.5, 2^4 domains, SAP 4 cycles x 4 MR steps, FGMRES-DR m = 20, k = 5,
tol 1e-10, Gaussian right-hand side seed 1), solved by the oracle's
Algorithm 4 with the refinement of Sec. 5.7: Arnoldi steps, cycles, clean
restarts, the per-cycle (steps, implicit, explicit) relative residuals, the
harmonic Ritz values kept at each deflated restart (Lemma 1a), the norm of
the solution and its first components; and D = Eq. "Dw" applied to the
right-hand side at the first sites.

wilson_16x16x16x32_oracle.json -- the benchmark workload (16^3 x 32, eps 0.5,
seed 0, bare mass from the stored spectral edge, 4^4 domains, SAP 5 x 4,
FGMRES-DR m = 30, k = 10, tol 1e-10, Gaussian right-hand side seed 1) solved
completely by the oracle: Arnoldi steps, cycles, clean restarts, the
per-cycle residuals and the final true residual. Written again whenever the
bare mass changes (the file records it).
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fieldgen as fg  # noqa: E402
import oracle  # noqa: E402


def cplx(a):
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    return [[float(v.real), float(v.imag)] for v in a]


def main():
    cfg = fg.lattice_configs()["tiny_4x4x4x4"]
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(dims, 1)
    res = oracle.solve(U, b, dims, cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"], cfg["k"],
                       cfg["tol"])
    Db = oracle.dw(U, b, dims, cfg["m0"])
    out = {
        "workload": "tiny_4x4x4x4",
        "source": "oracle (FP64 CPU): Algorithm 4 with the refinement of Sec. 5.7; Eq. \"Dw\"",
        "config": {"dims": list(dims), "block": list(cfg["block"]), "eps": cfg["eps"], "seed": cfg["seed"],
                   "m0": cfg["m0"], "sap_cycles": cfg["sap_cycles"], "mr_steps": cfg["mr_steps"], "m": cfg["m"],
                   "k": cfg["k"], "tol": cfg["tol"], "rhs_seed": 1},
        "iterations": int(res.iterations),
        "cycles": int(res.cycles),
        "clean_restarts": int(res.clean_restarts),
        "true_rel_res": float(res.true_rel_res),
        "history": [[int(h[0]), float(h[1]), float(h[2])] for h in res.history],
        "ritz": [cplx(r) for r in res.ritz],
        "x_norm": float(np.linalg.norm(res.x)),
        "x_head": cplx(np.asarray(res.x).reshape(-1)[:24]),
        "Db_head": cplx(np.asarray(Db).reshape(-1)[:24]),
    }
    path = os.path.join(HERE, "tiny_4x4x4x4_fgmresdr.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)
    if "--tiny-only" not in sys.argv:
        bench_workload()


def bench_workload():
    name = "wilson_16x16x16x32"
    cfg = fg.lattice_configs()[name]
    dims = cfg["dims"]
    U = fg.gauge_field(dims, cfg["eps"], cfg["seed"])
    b = fg.gaussian_source(dims, 1)
    res = oracle.solve(U, b, dims, cfg["block"], cfg["m0"], cfg["sap_cycles"], cfg["mr_steps"], cfg["m"], cfg["k"],
                       cfg["tol"])
    out = {
        "workload": name,
        "source": "oracle (FP64 CPU): Algorithm 4 with the refinement of Sec. 5.7, SAP (Algorithm 2) with MR",
        "config": {"dims": list(dims), "block": list(cfg["block"]), "eps": cfg["eps"], "seed": cfg["seed"],
                   "m0": cfg["m0"], "sap_cycles": cfg["sap_cycles"], "mr_steps": cfg["mr_steps"], "m": cfg["m"],
                   "k": cfg["k"], "tol": cfg["tol"], "rhs_seed": 1},
        "iterations": int(res.iterations),
        "cycles": int(res.cycles),
        "clean_restarts": int(res.clean_restarts),
        "true_rel_res": float(res.true_rel_res),
        "history": [[int(h[0]), float(h[1]), float(h[2])] for h in res.history],
    }
    path = os.path.join(HERE, name + "_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
