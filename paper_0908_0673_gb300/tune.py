"""Autotuner for the plan's leaf size.

The leaf size B (vertices per leaf box) sets the balance between the near
field (grows with B) and the expansions and translations (grow with the box
count): the fastest B depends on the mesh size, the Green's function and the
precision.  The tuner times, on this GPU, plan set-up plus an expected number
of products for every candidate B on a representative mesh of each size
class, and keeps the cheapest.  Accuracy parameters (expansion order,
separation factor, quadrature) are not tuned: they fix the stated errors.

    table = tune(green, precision)          # measure (needs a GPU)
    save(table, path); table = load(path)
    params = choose(n_elems, green, precision, table)   # fmm parameters for a mesh
"""
from __future__ import annotations

import json
import math
import os
import time

from . import bem
from . import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuned_leaf_size.json")

# size classes by element count (upper bounds) and the leaf sizes tried
CLASSES = (4_000, 15_000, 60_000, 250_000)
CANDIDATES = (24, 32, 48, 64, 96, 128)
DEFAULT_LEAF = 64
ITERS = 15                                # products per solve assumed by the cost


def _key(green: int, precision: int) -> str:
    return f"{'helmholtz' if green == bem.BEM_HELMHOLTZ else 'laplace'}-{'mixed' if precision == bem.BEM_MIXED else 'f64'}"


def _representative(hi: int):
    """Geodesic sphere of 6-node triangles near the geometric middle of a class."""
    lo = 1_000 if hi == CLASSES[0] else CLASSES[CLASSES.index(hi) - 1]
    target = math.sqrt(lo * hi)
    return I.geodesic(max(2, int(round(math.sqrt(target / 20.0)))), I.TRI6)


def measure(mesh, green: int, k: float, precision: int, leaf: int, reps: int = 5, p: int = 10, eta: float = 2.0):
    """(set-up ms, product ms) of one plan on this GPU."""
    import torch
    ctx = bem.bem_ctx_create(0)
    mh = bem.bem_mesh_create(ctx, mesh.nodes, mesh.elems, mesh.elem_type)
    try:
        n_phi, _ = bem.bem_mesh_sizes(mh)
        prm = bem.bem_fmm_params_default(p=p, leaf_size=leaf, eta=eta, precision=precision)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = bem.bem_plan_create(mh, green, k, prm)
        setup_ms = (time.perf_counter() - t0) * 1e3
        try:
            dt = torch.complex128 if green == bem.BEM_HELMHOLTZ else torch.float64
            x = torch.ones(n_phi, device="cuda", dtype=dt)
            y = torch.empty_like(x)
            for _ in range(2):
                bem.bem_matvec(plan, bem.BEM_OP_A, x, y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                bem.bem_matvec(plan, bem.BEM_OP_A, x, y)
            e1.record()
            e1.synchronize()
            return setup_ms, e0.elapsed_time(e1) / reps
        finally:
            bem.bem_plan_destroy(plan)
    finally:
        bem.bem_mesh_destroy(mh)
        bem.bem_ctx_destroy(ctx)


def tune(green: int = bem.BEM_LAPLACE, precision: int = bem.BEM_MIXED, k: float = 2.0, classes=CLASSES,
         candidates=CANDIDATES, iters: int = ITERS, table: dict | None = None) -> dict:
    """Measures every candidate leaf size on each class's representative mesh
    and records the cheapest (set-up + iters products) in the table."""
    table = dict(table or {})
    key = _key(green, precision)
    rows = []
    for hi in classes:
        mesh = _representative(hi)
        costs = {}
        for leaf in candidates:
            setup_ms, prod_ms = measure(mesh, green, k if green == bem.BEM_HELMHOLTZ else 0.0, precision, leaf)
            costs[leaf] = {"setup_ms": setup_ms, "product_ms": prod_ms, "cost_ms": setup_ms + iters * prod_ms}
        best = min(costs, key=lambda b: costs[b]["cost_ms"])
        rows.append({"max_elems": hi, "mesh_elems": int(mesh.n_elems), "leaf_size": int(best),
                     "measured": {str(b): v for b, v in costs.items()}})
    table[key] = rows
    return table


def save(table: dict, path: str = TABLE) -> None:
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def load(path: str = TABLE) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def choose(n_elems: int, green: int = bem.BEM_LAPLACE, precision: int = bem.BEM_MIXED, table: dict | None = None,
           p: int = 10, eta: float = 2.0) -> dict:
    """fmm parameters for a mesh of n_elems elements: the tuned leaf size of
    its class (the largest class for bigger meshes), else the default."""
    table = load() if table is None else table
    rows = table.get(_key(green, precision), [])
    leaf = DEFAULT_LEAF
    for row in sorted(rows, key=lambda r: r["max_elems"]):
        leaf = row["leaf_size"]
        if n_elems <= row["max_elems"]:
            break
    return {"p": p, "leaf_size": int(leaf), "eta": eta, "precision": precision}


if __name__ == "__main__":
    t = load()
    for green in (bem.BEM_LAPLACE, bem.BEM_HELMHOLTZ):
        for precision in (bem.BEM_MIXED, bem.BEM_F64):
            t = tune(green, precision, table=t)
            print(_key(green, precision), [(r["max_elems"], r["leaf_size"]) for r in t[_key(green, precision)]],
                  flush=True)
    save(t)
