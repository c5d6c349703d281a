"""Writes fieldgen/spectral_edges.json: the left spectral edge of D (at m0 = 0)
for every synthetic gauge field the workloads use, from the oracle only.

The edge is the Ritz value of smallest real part of an m-step Arnoldi process
on the oracle's D (oracle.tune_m0_arnoldi). Since spec(D_m0) = spec(D_0) + m0,
a workload that wants its smallest |eigenvalue| near delta takes
m0 = delta - Re(edge) (fieldgen.lattice_configs does this).

Usage: python -m oracle.tune_masses [--only NAME]
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

# (dims, eps, seed, Arnoldi steps); 0 steps selects the thick-restarted
# (Krylov-Schur) variant, which keeps 61 basis vectors for the 32^3 x 64 field.
FIELDS = [
    ((16, 16, 16, 32), 0.5, 0, 200),
    ((24, 24, 24, 48), 0.5, 0, 200),
    ((32, 32, 32, 64), 0.6, 0, 0),
] + [((8, 8, 8, 16), e, 0, 200) for e in (0.3, 0.45, 0.6)] \
  + [((16, 16, 16, 32), e, 0, 200) for e in (0.3, 0.45, 0.6)] \
  + [((24, 24, 24, 48), e, 0, 160) for e in (0.3, 0.45, 0.6)]


# clover-improved operators: (dims, eps, seed, Arnoldi steps, c_sw)
CLOVER_FIELDS = [((16, 16, 16, 32), 0.5, 0, 0, 1.91)]


def key(dims, eps, seed, csw=0.0):
    k = f"{'x'.join(map(str, dims))}_eps{eps}_seed{seed}"
    return k + (f"_csw{csw}" if csw else "")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for dims, eps, seed, m, csw in [f + (0.0,) for f in FIELDS] + CLOVER_FIELDS:
        k = key(dims, eps, seed, csw)
        if args.only and args.only != k:
            continue
        if k in data and data[k].get("arnoldi_steps") == m:
            continue
        t0 = time.time()
        U = fg.gauge_field(dims, eps, seed)
        A = oracle.clover(U, dims, csw) if csw else None
        if m > 0:
            _, theta, bound, secs = oracle.tune_m0_arnoldi(U, dims, 0.0, m=m, clov=A)
            how = {"arnoldi_steps": m}
        else:
            _, theta, bound, mv, secs = oracle.tune_m0_schur(U, dims, 0.0, m=60, k=20, tol=2e-3, clov=A)
            how = {"arnoldi_steps": 0, "krylov_schur": {"m": 60, "k": 20, "tol": 2e-3, "matvecs": mv}}
        if csw:
            how["csw"] = csw
        data[k] = {"dims": list(dims), "eps": eps, "seed": seed, **how,
                   "edge_re": float(theta.real), "edge_im": float(theta.imag), "ritz_residual_bound": float(bound),
                   "seconds": round(time.time() - t0, 1)}
        print(k, data[k], flush=True)
        with open(OUT + ".tmp", "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(OUT + ".tmp", OUT)
        del U


if __name__ == "__main__":
    main()
