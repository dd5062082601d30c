"""Writes tests/golden/audit12_oracle.json: the FP64 oracle's 12-geometry
rank audit (Sec. 6.2-6.3) on the oracle's own ray tables, for the GPU parity
test of rtt_rank_audit.  Calls only oracle/ and the seeded input module.

For every geometry (spins {0, 0.5, 0.75, 0.94} x inclinations {20, 50, 75}
deg, kerr256 sizes) and both arms (direct n = 0, resolved n = 0..2):
  * the restricted Gram of the S224 class, G = (s A Q)^T (s A Q), formed as
    Q^T (A^T (A Q)) column block by column block with the oracle's applies
    (the definition of G; P = s A Q itself would not fit in memory), its
    eigenvalues (numpy eigvalsh), sigma = sqrt(max(lambda, 0)), the
    operational rank #{sigma >= rho} (Eq. 31) and the margin
    min |sigma - rho| / rho;
  * the probe information at the 64 ages, the anchor-connected reach
    L_anchor (Eq. 30, 33), A_{0,0.999} (Sec. 4.5) and J_old (Eq. 35).
Two samplings: the workload list's 256 frames at 1 M, and the paper's audit
sampling of eight frames 2.5 M apart (inputs.audit12_paper_sampling).

Usage: python tests/golden/make_audit12.py [--sampling frames256|paper8|both]
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "oracle"))

import oracle as O  # noqa: E402
from paper_2609_05528_b300 import inputs as I  # noqa: E402

OUT = os.path.join(HERE, "audit12_oracle.json")
RHO = 1.0
CHUNK = 16


def workload_key(w) -> str:
    """Hash of everything that defines the oracle's tables and operator."""
    return hashlib.sha256(repr(w).encode()).hexdigest()[:16]


def gram_normal(w, tab, Q, scl):
    S, K = w.grid.n_nodes, w.time.n_hats
    d = Q.shape[1]
    G = np.zeros((d, d))
    for c0 in range(0, d, CHUNK):
        c1 = min(d, c0 + CHUNK)
        xc = np.ascontiguousarray(Q[:, c0:c1]).reshape(S, K, c1 - c0)
        y = O.apply_A(w, tab, xc, scl)
        z = O.apply_AT(w, tab, y, scl).reshape(S * K, c1 - c0)
        G[:, c0:c1] = Q.T @ z
    return 0.5 * (G + G.T)


def audit_cell(w):
    tab = O.build_table(w, I.screen_samples(w))
    scl = O.scale(tab)
    Q = O.synth_class(w, "S224")
    a0 = O.a0999(w, tab)
    rec = {"name": w.name, "key": workload_key(w), "n_rays": tab.n_rays, "n_rows": tab.n_rows,
           "A0999": a0, "arms": {}}
    for arm, orders in (("direct", (0,)), ("resolved", (0, 1, 2))):
        sub = tab.select(orders)
        G = gram_normal(w, sub, Q, scl)
        ev = np.linalg.eigvalsh(G)
        sig = np.sort(np.sqrt(np.maximum(ev, 0.0)))[::-1]
        info = O.probe_info(w, sub, scl)
        r = O.reach(w, sub, info, orders, rho=RHO)
        rec["arms"][arm] = {
            "rank": int(np.count_nonzero(sig >= RHO)),
            "margin": float(np.min(np.abs(sig - RHO)) / RHO),
            "sigma_max": float(sig[0]),
            "sigma_min": float(sig[-1]),
            "L_anchor": float(r.L_anchor),
            "anchor": None if r.anchor is None else float(r.anchor),
            "J_old": float(O.j_old(info, a0)),
        }
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sampling", default="both", choices=["frames256", "paper8", "both"])
    args = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            out = json.load(fh)
    todo = []
    if args.sampling in ("paper8", "both"):
        todo.append(("paper8", I.audit12_paper_sampling()))
    if args.sampling in ("frames256", "both"):
        todo.append(("frames256", I.audit12()))
    for name, cells in todo:
        recs = out.get(name, {}).get("cells", [])
        done = {r["key"] for r in recs}
        for w in cells:
            if workload_key(w) in done:
                continue
            t = time.perf_counter()
            recs.append(audit_cell(w))
            print(f"{name} {w.name}: {time.perf_counter() - t:.1f} s", flush=True)
            out[name] = {"rho": RHO, "snr0": 100.0, "class": "S224", "cells": recs}
            with open(OUT, "w") as fh:
                json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
