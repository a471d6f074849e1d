"""Error of the four-step fast product against the direct product for the
Helmholtz double layer (op A) at higher wavenumbers, on the level-4 geodesic
sphere of 6-node triangles (5,120 elements, 10,242 nodes), over the
wavenumber, the separation factor and the expansion order.

Test infrastructure: it runs the CPU oracle only (the same quadrature, tree
and truncation as the library, Sections 3.1-3.6) and writes
tests/golden/highk_sweep.json, which tests/test_oracle_highk.py reads.  Run
from the repository root:  python -m oracle.highk_sweep   (about 15 minutes
on 8 cores).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_0908_0673_gb300 import inputs as I  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "highk_sweep.json")
KA = (2.0, 8.0, 16.0)
ETA = (2.0, 3.0)
ORDERS = (8, 10, 12, 16)
LEAF = 128


def main():
    O.build()
    m = I.icosphere(4, I.TRI6)
    ci, n_chi = O.chi_index(m.nodes, m.elems)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(m.n_nodes) + 1j * rng.standard_normal(m.n_nodes)
    _, _, d0 = O.assemble(m.nodes, m.elems, ci, n_chi, rows=np.arange(m.n_nodes))
    out = {"mesh": "icosphere level 4, 6-node triangles", "elements": int(m.n_elems), "nodes": int(m.n_nodes),
           "leaf_size": LEAF, "operator": "A (C - D), Helmholtz double layer", "vector": "complex normal, seed 0",
           "error": "relative L2 of the four-step product against the direct product", "runs": []}
    for ka in KA:
        t0 = time.time()
        ref = O.apply_rows(m.nodes, m.elems, ci, O.OP_A, x, None, green=O.HELMHOLTZ, k=ka)
        corr = O.correction(m.nodes, m.elems, ci, green=O.HELMHOLTZ, k=ka)
        print(f"ka {ka}: direct product and correction {time.time() - t0:.1f} s", flush=True)
        for eta in ETA:
            T = O.Tree(m.nodes, m.elems, B=LEAF, eta=eta)
            for p in ORDERS:
                t0 = time.time()
                y = O.fmm_apply(T, ci, O.OP_A, x, d0, corr, p, green=O.HELMHOLTZ, k=ka)
                err = float(np.linalg.norm(y - ref) / np.linalg.norm(ref))
                out["runs"].append({"ka": ka, "eta": eta, "p": p, "rel_err": err,
                                    "interaction_pairs": int(T.inter_idx.shape[0]), "seconds": time.time() - t0})
                print(f"  eta {eta} p {p}: {err:.3e} ({time.time() - t0:.1f} s)", flush=True)
                with open(OUT, "w") as f:
                    json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
