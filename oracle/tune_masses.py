"""Writes fieldgen/spectral_edges.json: the left spectral edge of D (at m0 = 0)
for every synthetic gauge field the workloads use, and the eigenvalues of the
workload's D_m0 nearest the origin, from the oracle only.

spec(D_m0) = spec(D_0) + m0 exactly, so a workload that wants the leftmost
eigenvalue of D at real part delta takes m0 = delta - edge. For each field:

1. start from a rough edge e0 (a stored value, else 300 products of the
   thick-restarted Arnoldi process ``oracle.krylov_schur_edge``); on lattices
   of at most 8192 sites run that process to a residual below delta_ref / 10
   as well (the leftmost eigenvalue there can have an imaginary part large
   enough to miss the set of step 2);
2. compute the eigenvalues of D_{m1}, m1 = delta_ref - e0, nearest the origin
   by harmonic Ritz extraction with thick restarts
   (``oracle.harmonic_ritz_nearest``, Lemma 1a), until each of the ten
   nearest that lies within twice the smallest modulus has a residual
   ||D u - theta u|| below delta_ref / 10 (the cluster that sets the
   conditioning; the farther ones are kept with their residuals);
3. edge = min Re(theta) - m1 (the leftmost of them, as an eigenvalue of D_0),
   or the converged Krylov-Schur value of step 1 where that lies further left;
   at the workload's m0 = delta_ref - edge its eigenvalues nearest the origin
   are theta + (m0 - m1), so the stored min |lambda| is that of the workload's
   operator (the verification asked for by reading R16).

delta_ref is the smallest delta the field serves (1e-2 for the 16^3 x 32 bench
and clover workloads, 5e-3 for the batched 24^3 x 48 one, 1e-3 for the mixed
32^3 x 64 one and for the served requests).

Usage: python -m oracle.tune_masses [--only KEY] [--max-restarts N] [--force]
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import fieldgen as fg  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(ROOT, "fieldgen", "spectral_edges.json")

# (dims, eps, seed, c_sw, delta_ref, basis m, kept k), in the order they run
FIELDS = [
    ((16, 16, 16, 32), 0.5, 0, 0.0, 1e-2, 60, 20),
    ((16, 16, 16, 32), 0.5, 0, 1.91, 1e-2, 60, 20),
    ((8, 8, 8, 16), 0.3, 0, 0.0, 1e-3, 60, 20),
    ((8, 8, 8, 16), 0.6, 0, 0.0, 1e-3, 60, 20),
    ((24, 24, 24, 48), 0.5, 0, 0.0, 5e-3, 60, 20),
    ((16, 16, 16, 32), 0.3, 0, 0.0, 1e-3, 60, 20),
    ((16, 16, 16, 32), 0.6, 0, 0.0, 1e-3, 60, 20),
    ((32, 32, 32, 64), 0.6, 0, 0.0, 1e-3, 48, 16),
    ((24, 24, 24, 48), 0.3, 0, 0.0, 1e-3, 60, 20),
    ((24, 24, 24, 48), 0.6, 0, 0.0, 1e-3, 60, 20),
]
NEV = 10


def fg_edges_path():
    return os.path.join(ROOT, "fieldgen", "spectral_edges.json")
SMALL = 8192  # sites: the leftmost Ritz value is also converged directly


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default=None)
    ap.add_argument("--max-restarts", type=int, default=200)
    ap.add_argument("--force", action="store_true", help="recompute fields that are already stored")
    ap.add_argument("--out", default=OUT, help="file to merge the results into")
    ap.add_argument("--max-seconds", type=float, default=None,
                    help="stop the harmonic Ritz run after this long and store its values as not converged")
    args = ap.parse_args()
    out_path = args.out
    data = {}
    if os.path.exists(fg_edges_path()):
        with open(fg_edges_path()) as f:
            data = json.load(f)
    for dims, eps, seed, csw, delta, m, k in FIELDS:
        key = fg.edge_key(dims, eps, seed, csw)
        if args.only and args.only != key:
            continue
        old = data.get(key, {})
        V = fg.volume(dims)
        if (not args.force and old.get("method") == "harmonic_ritz" and old.get("delta_ref") == delta
                and old.get("converged") and old.get("tol", 1.0) <= delta / 10
                and (V > SMALL or old.get("krylov_schur"))):
            continue  # a stored result at least as tight as this run's
        t0 = time.time()
        U = fg.gauge_field(dims, eps, seed)
        A = oracle.clover(U, dims, csw) if csw else None

        def op(m0):
            return lambda v: oracle.dw(U, np.asarray(v).reshape(V, 4, 3), dims, m0, A=A).reshape(-1)

        e0 = old.get("edge_re")
        ks = None
        if V <= SMALL:
            th, res_ks, mv_ks = oracle.krylov_schur_edge(op(0.0), 12 * V, 60, 20, max_restarts=200, tol=delta / 10)
            ks = {"edge_re": float(th.real), "edge_im": float(th.imag), "residual": float(res_ks), "matvecs": mv_ks,
                  "converged": bool(res_ks < delta / 10)}
            e0 = ks["edge_re"]
        elif e0 is None:
            theta, _, _ = oracle.krylov_schur_edge(op(0.0), 12 * V, 60, 20, max_restarts=7, tol=0.0)
            e0 = float(theta.real)
        m1 = delta - e0

        def log(restart, mv, th, res):
            print(f"{key} restart {restart} matvecs {mv} nearest "
                  + " ".join(f"{t.real:+.6f}{t.imag:+.6f}i({r:.1e})" for t, r in zip(th, res))
                  + f" {time.time() - t0:.0f}s", flush=True)

        theta, res, mv = oracle.harmonic_ritz_nearest(op(m1), 12 * V, m=m, k=k, max_restarts=args.max_restarts,
                                                      tol=delta / 10, nev=NEV, log=log, near_factor=2.0,
                                                      stop=(lambda: time.time() - t0 > args.max_seconds)
                                                      if args.max_seconds else None)
        lead = int(np.argmin(theta.real))
        edge, edge_im = float(theta.real.min()) - m1, float(theta[lead].imag)
        if ks and ks["converged"] and ks["edge_re"] < edge:
            edge, edge_im = ks["edge_re"], ks["edge_im"]
        m0 = delta - edge
        at_m0 = theta + (m0 - m1)
        near = np.abs(at_m0).min()
        if ks and ks["converged"]:
            near = min(near, abs(complex(ks["edge_re"] + m0, ks["edge_im"])))
        data[key] = {"dims": list(dims), "eps": eps, "seed": seed, "method": "harmonic_ritz", "m": m, "k": k, "nev": NEV,
                     "delta_ref": delta, "tol": delta / 10, "matvecs": mv,
                     "converged": bool(res[np.abs(theta) <= 2.0 * np.abs(theta).min()].max() < delta / 10),
                     "edge_re": edge, "edge_im": edge_im, "start_edge_re": e0, "krylov_schur": ks,
                     "m0_ref": m0, "min_abs_eig_at_m0_ref": float(near),
                     "nearest_at_m0_ref": [[float(t.real), float(t.imag), float(r)] for t, r in zip(at_m0, res)],
                     "seconds": round(time.time() - t0, 1)}
        if csw:
            data[key]["csw"] = csw
        print(key, data[key], flush=True)
        # merge into the file as it is now (other runs may have added fields)
        cur = {}
        if os.path.exists(out_path):
            with open(out_path) as f:
                cur = json.load(f)
        cur[key] = data[key]
        with open(out_path + ".tmp", "w") as f:
            json.dump(cur, f, indent=1, sort_keys=True)
        os.replace(out_path + ".tmp", out_path)
        del U, A


if __name__ == "__main__":
    main()
