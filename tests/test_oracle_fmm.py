"""Pins for the oracle's tree, lists and fast matrix multiplication
(Sections 3.1, 3.4, 3.6).

* tree invariants: every vertex in exactly one leaf; a leaf holds fewer than
  B vertices (unless at the level cap); children nest in their parents;
  every radius covers the points it must (Eq. 12 bound included);
* list invariants: for every leaf target box the sources are covered exactly
  once by the interaction lists of its ancestors (and itself) plus its near
  list, and every interaction pair is well separated (Eq. 13);
* the four-step matrix multiplication converges to the dense operator as the
  order p and the separation factor eta grow;
* locals coarser than the coarsest interaction-list target are exactly zero
  (what lets the product skip the coarse levels of both passes);
* the oracle's GMRES agrees with the LU solve.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import inputs as I


def _subtree_leaves(T, b, children):
    out, stack = [], [b]
    while stack:
        x = stack.pop()
        if T.leaf[x]:
            out.append(x)
        else:
            stack += children[x]
    return out


@pytest.mark.parametrize("mesh,B,eta,ld", [
    (lambda: I.icosphere(3), 16, 1.0, 1), (lambda: I.icosphere(3), 32, 2.0, 0),
    (lambda: I.cube(6, I.TRI6), 24, 1.5, 1), (lambda: I.cube(6, I.TRI6), 24, 1.5, 0)])
def test_tree_and_list_invariants(oracle_lib, mesh, B, eta, ld):
    O = oracle_lib
    m = mesh()
    T = O.Tree(m.nodes, m.elems, B=B, eta=eta, leaf_descend=ld)
    nb = T.n_boxes
    children = {b: [] for b in range(nb)}
    for b in range(nb):
        if T.parent[b] >= 0:
            children[int(T.parent[b])].append(b)
            p = T.parent[b]
            assert T.level[b] == T.level[p] + 1
            assert np.all(T.ijk[b] // 2 == T.ijk[p])
    # leaves partition the vertices; fewer than B per leaf
    counts = np.bincount(T.leaf_of_node, minlength=nb)
    assert np.all(T.leaf[T.leaf_of_node] == 1)
    assert np.all(counts[T.leaf == 1] < B)
    # each vertex lies in its leaf's cube
    h = T.side / 2.0 ** T.level[T.leaf_of_node]
    lo = T.lo + T.ijk[T.leaf_of_node] * h[:, None]
    assert np.all(m.nodes >= lo) and np.all(m.nodes <= lo + h[:, None])
    # radii cover vertices and the element points of the subtree
    qx, _, _, _ = O.quad_points(m.nodes, m.elems)
    for b in range(nb):
        lv = _subtree_leaves(T, b, children)
        els = np.nonzero(np.isin(T.owner, lv))[0]
        pts = [m.nodes[np.isin(T.leaf_of_node, lv)]]
        if len(els):
            pts += [m.nodes[m.elems[els].ravel()], qx.reshape(-1, 7, 3)[els].reshape(-1, 3)]
        d = np.linalg.norm(np.vstack(pts) - T.centre[b], axis=1)
        assert d.max() <= T.radius[b] * (1 + 1e-14)
    # interaction pairs are separated; sources covered exactly once per leaf
    for t in range(nb):
        for s in T.inter_idx[T.inter_ptr[t]:T.inter_ptr[t + 1]]:
            d = np.linalg.norm(T.centre[t] - T.centre[s])
            assert d > eta * (T.radius[t] + T.radius[s])
    nleaf_total = int(T.leaf.sum())
    for t in np.nonzero(T.leaf)[0]:
        cover = []
        a = t
        while a >= 0:
            for s in T.inter_idx[T.inter_ptr[a]:T.inter_ptr[a + 1]]:
                cover += _subtree_leaves(T, int(s), children)
            a = T.parent[a]
        for s in T.near_idx[T.near_ptr[t]:T.near_ptr[t + 1]]:
            if ld:
                assert T.leaf[s]
            cover += _subtree_leaves(T, int(s), children)
        assert len(cover) == nleaf_total and len(set(cover)) == nleaf_total


def test_fmm_converges_to_dense(oracle_lib):
    O = oracle_lib
    m = I.icosphere(3)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    A, B, d0 = O.operators(m.nodes, m.elems, ci, nchi)
    corr = O.correction(m.nodes, m.elems, ci)
    x = I.random_vector(m.n_nodes, 1)
    xs = I.random_vector(nchi, 2)
    yA, yB = A @ x, B @ xs
    prev = None
    for p in (4, 8):
        T = O.Tree(m.nodes, m.elems, B=16, eta=2.0)
        eA = np.linalg.norm(O.fmm_apply(T, ci, O.OP_A, x, d0, corr, p).real - yA) / np.linalg.norm(yA)
        eB = np.linalg.norm(O.fmm_apply(T, ci, O.OP_B, xs, d0, corr, p).real - yB) / np.linalg.norm(yB)
        if prev is not None:
            assert eA < prev[0] / 10 and eB < prev[1] / 10
        prev = (eA, eB)
    assert prev[0] < 1e-6 and prev[1] < 1e-6


def test_fmm_helmholtz_converges(oracle_lib):
    O = oracle_lib
    m = I.icosphere(2, I.TRI6)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    A, B, d0 = O.operators(m.nodes, m.elems, ci, nchi, O.HELMHOLTZ, 2.0)
    corr = O.correction(m.nodes, m.elems, ci, O.HELMHOLTZ, 2.0)
    x = I.random_vector(m.n_nodes, 3, complex_=True)
    T = O.Tree(m.nodes, m.elems, B=16, eta=2.0)
    e = []
    for p in (4, 10):
        y = O.fmm_apply(T, ci, O.OP_A, x, d0, corr, p, O.HELMHOLTZ, 2.0)
        e.append(np.linalg.norm(y - A @ x) / np.linalg.norm(A @ x))
    assert e[1] < e[0] / 10 and e[1] < 1e-6


def test_gmres_matches_lu(oracle_lib):
    O = oracle_lib
    m = I.cube(4, I.TRI6)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    A, B, d0 = O.operators(m.nodes, m.elems, ci, nchi)
    _, chi_e = I.point_source(m, (0.2, -0.1, 0.3))
    b = B @ O.chi_from_elem(ci, nchi, chi_e)
    x_lu = O.solve_dense(A, b)
    x, it, rel = O.gmres(lambda v: A @ v, b, restart=30, tol=1e-10)
    assert rel <= 1e-10
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) < 1e-8


@pytest.mark.parametrize("mesh,B,eta", [
    (lambda: I.icosphere(3), 16, 2.0),
    (lambda: I.cube(6, I.TRI6), 24, 2.0),
    (lambda: I.geodesic(8, I.TRI6, axes=(0.6, 1.0, 1.7)), 32, 2.0),
    (lambda: I.icosphere(3), 16, 1.0),
])
def test_coarse_expansions_never_reach_the_product(oracle_lib, mesh, B, eta):
    """Section 3.6 as the product uses it: moments are read only by the
    interaction lists, and a box's local is its parent's shifted local plus
    its own list terms, so every local coarser than the coarsest box with a
    nonempty interaction list is exactly zero, and the product can stop the
    upward pass at the coarsest source level and start the downward pass
    below the coarsest target level.  At eta = 2 neither level 0 nor level 1
    interacts on these meshes."""
    O = oracle_lib
    m = mesh()
    ci, nchi = O.chi_index(m.nodes, m.elems)
    T = O.Tree(m.nodes, m.elems, B=B, eta=eta)
    ip, lev = T.inter_ptr, T.level
    assert len(T.inter_idx) > 0
    src_lmin = int(lev[T.inter_idx].min())
    tgt_lmin = int(lev[np.flatnonzero(ip[1:] > ip[:-1])].min())
    if eta >= 2.0:
        assert src_lmin >= 2 and tgt_lmin >= 2
    corr = dict(row=np.zeros(0, np.int64), col_phi=np.zeros(0, np.int32), col_chi=np.zeros(0, np.int32),
                D=np.zeros(0, complex), S=np.zeros(0, complex))
    x = I.random_vector(m.n_nodes, 12)
    _, mom, loc = O.fmm_apply(T, ci, O.OP_A, x, np.zeros(m.n_nodes), corr, 6, want_expansions=True)
    coarse = lev < tgt_lmin
    assert np.all(np.asarray(loc)[coarse] == 0)
    assert np.any(np.asarray(loc)[~coarse] != 0)
    assert np.any(np.asarray(mom)[lev < src_lmin] != 0) or src_lmin == 0   # formed by the oracle, unused
