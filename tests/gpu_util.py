"""Helpers for the GPU parity tests: build a plan through the C ABI, run
products on torch CUDA tensors, canonicalise trees for bit-exact comparison."""
import numpy as np

from paper_0908_0673_gb300 import bem


class Plan:
    def __init__(self, m, green=bem.BEM_LAPLACE, k=0.0, **prm):
        import torch
        self.torch = torch
        self.m = m
        self.ctx = bem.bem_ctx_create(0)
        self.mesh = bem.bem_mesh_create(self.ctx, m.nodes, m.elems, m.elem_type)
        self.n_phi, self.n_chi = bem.bem_mesh_sizes(self.mesh)
        self.chi_idx = bem.bem_mesh_chi_index(self.mesh, m.n_elems, m.npe)
        self.params = bem.bem_fmm_params_default(**prm)
        self.green, self.k = green, k
        self.plan = bem.bem_plan_create(self.mesh, green, k, self.params)
        self.complex = green == bem.BEM_HELMHOLTZ

    def _dev(self, x):
        t = self.torch
        dt = t.complex128 if self.complex else t.float64
        return t.tensor(np.asarray(x), device="cuda", dtype=dt)

    def matvec(self, op, x):
        t = self.torch
        xd = self._dev(x)
        yd = t.empty(self.n_phi, device="cuda", dtype=xd.dtype)
        bem.bem_matvec(self.plan, op, xd, yd)
        t.cuda.synchronize()
        return yd.cpu().numpy()

    def solve(self, chi, **sp):
        t = self.torch
        cd = self._dev(chi)
        pd = t.empty(self.n_phi, device="cuda", dtype=cd.dtype)
        code, info = bem.bem_solve(self.plan, cd, pd, 1, bem.bem_solve_params_default(**sp))
        t.cuda.synchronize()
        return pd.cpu().numpy(), code, info[0]

    def stats(self):
        return bem.bem_plan_stats(self.plan)

    def close(self):
        bem.bem_plan_destroy(self.plan)
        bem.bem_mesh_destroy(self.mesh)
        bem.bem_ctx_destroy(self.ctx)


def canon_tree(level, ijk, parent, leaf, centre, radius, near_ptr, near_idx, inter_ptr, inter_idx,
               leaf_of_node, owner):
    """Tree as a dict keyed by (level, ix, iy, iz): every field that must be
    bit-exact, with box references replaced by keys and lists by sets."""
    key = [(int(level[b]),) + tuple(int(v) for v in ijk[b]) for b in range(len(level))]
    nodes = {}
    for i, b in enumerate(leaf_of_node):
        nodes.setdefault(key[b], []).append(i)
    elems = {}
    for e, b in enumerate(owner):
        elems.setdefault(key[b], []).append(e)
    out = {}
    for b in range(len(level)):
        out[key[b]] = dict(
            parent=key[parent[b]] if parent[b] >= 0 else None,
            leaf=int(leaf[b]),
            centre=tuple(np.asarray(centre[b]).view(np.uint64).tolist()),
            radius=int(np.asarray(radius[b]).view(np.uint64)),
            near=frozenset(key[j] for j in near_idx[near_ptr[b]:near_ptr[b + 1]]),
            inter=frozenset(key[j] for j in inter_idx[inter_ptr[b]:inter_ptr[b + 1]]),
            nodes=tuple(sorted(nodes.get(key[b], []))),
            elems=tuple(sorted(elems.get(key[b], []))))
    return out


def canon_oracle(T):
    return canon_tree(T.level, T.ijk, T.parent, T.leaf, T.centre, T.radius, T.near_ptr, T.near_idx,
                      T.inter_ptr, T.inter_idx, T.leaf_of_node, T.owner)


def canon_export(d):
    return canon_tree(d["level"], d["ijk"], d["parent"], d["leaf"], d["centre"], d["radius"], d["near_ptr"],
                      d["near_idx"], d["inter_ptr"], d["inter_idx"], d["leaf_of_node"], d["owner"])


def coo_sum(rows, cols, vals):
    out = {}
    for r, c, v in zip(rows.tolist(), cols.tolist(), vals.tolist()):
        out[(r, c)] = out.get((r, c), 0.0) + v
    return out


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
