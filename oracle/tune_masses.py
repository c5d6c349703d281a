"""Writes fieldgen/spectral_edges.json: the left spectral edge of D (at m0 = 0)
for every synthetic gauge field the workloads use, from the oracle only.

The edge is the leftmost Ritz value of a thick-restarted Arnoldi process
(Krylov-Schur, ``oracle.tune_m0_schur``) on the oracle's D, run until the
residual norm of its Ritz pair is at most ``tol``. Since
spec(D_m0) = spec(D_0) + m0, a workload that wants the leftmost eigenvalue of
D at real part delta takes m0 = delta - Re(edge) (fieldgen.lattice_configs
does this); ``tol`` is a tenth of the smallest delta the field is used with.

Usage: python -m oracle.tune_masses [--only KEY] [--max-matvecs N]
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import fieldgen as fg  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(ROOT, "fieldgen", "spectral_edges.json")

# (dims, eps, seed, c_sw, residual tolerance), cheapest first. The tolerance is
# a tenth of the smallest delta the field serves: 1e-2 for the 16^3 x 32 bench
# and clover workloads, 5e-3 for the batched 24^3 x 48 one, 1e-3 for the mixed
# 32^3 x 64 one and for the served requests (delta in [1e-3, 1e-2]).
FIELDS = [
    ((8, 8, 8, 16), 0.3, 0, 0.0, 1e-4),
    ((8, 8, 8, 16), 0.6, 0, 0.0, 1e-4),
    ((16, 16, 16, 32), 0.5, 0, 0.0, 1e-3),
    ((16, 16, 16, 32), 0.5, 0, 1.91, 1e-3),
    ((16, 16, 16, 32), 0.3, 0, 0.0, 1e-4),
    ((16, 16, 16, 32), 0.6, 0, 0.0, 1e-4),
    ((24, 24, 24, 48), 0.5, 0, 0.0, 5e-4),
    ((32, 32, 32, 64), 0.6, 0, 0.0, 1e-4),
    ((24, 24, 24, 48), 0.3, 0, 0.0, 1e-4),
    ((24, 24, 24, 48), 0.6, 0, 0.0, 1e-4),
]
M, K = 60, 20


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    ap.add_argument("--max-matvecs", type=int, default=8000)
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for dims, eps, seed, csw, tol in FIELDS:
        k = fg.edge_key(dims, eps, seed, csw)
        if args.only and args.only != k:
            continue
        old = data.get(k, {})
        if old.get("method") == "krylov_schur" and old.get("tol") == tol and old.get("converged"):
            continue
        t0 = time.time()
        U = fg.gauge_field(dims, eps, seed)
        A = oracle.clover(U, dims, csw) if csw else None

        def log(restart, mv, theta, res):
            print(f"{k} restart {restart} matvecs {mv} theta {theta.real:.9f}{theta.imag:+.6f}i residual {res:.3e} "
                  f"{time.time() - t0:.0f}s", flush=True)

        max_restarts = max(1, (args.max_matvecs - M) // (M - K) + 1)
        _, theta, res, mv, secs = oracle.tune_m0_schur(U, dims, 0.0, m=M, k=K, tol=tol, clov=A,
                                                       max_restarts=max_restarts, log=log)
        data[k] = {"dims": list(dims), "eps": eps, "seed": seed, "method": "krylov_schur", "m": M, "k": K,
                   "tol": tol, "matvecs": mv, "converged": bool(res < tol),
                   "edge_re": float(theta.real), "edge_im": float(theta.imag), "ritz_residual": float(res),
                   "seconds": round(time.time() - t0, 1)}
        if csw:
            data[k]["csw"] = csw
        print(k, data[k], flush=True)
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        del U, A


if __name__ == "__main__":
    main()
