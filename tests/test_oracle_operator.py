"""Pins for the oracle's discrete operators (Section 2.1, Eq. 1-3).

* Gauss solid-angle identity: sum_j D0_ij = -Omega_i / (4 pi), Omega_i the
  interior solid angle at node i.  On flat-faceted meshes Omega follows in
  closed form from the dihedral angles (spherical excess); on cube faces,
  edges and corners it is 2 pi, pi and pi / 2.
* Point-source test of Section 4: the solved surface potential matches the
  source potential with the rms error the paper prints for the same mesh
  family and size (tests/golden/paper_errors.json): at most 3x worse, and
  not more than 10x better (the paper gives neither source position nor
  mesh details, so only the order of magnitude is fixed).
* The sign reading of Eq. 1: with the printed sign the point-source test
  fails outright.
* Sharp-edge multi-indexing (Section 2.3): 1, 2 and 3 indices at cube face,
  edge and corner nodes; one per node on the sphere.
* Helmholtz: the exterior point-source test at k = 2 (Table 3) and the
  rigid-sphere Mie series.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_0908_0673_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_errors.json")))


def _solid_angles_flat(nodes, elems):
    """Interior solid angle at every vertex of a closed convex flat-faceted
    surface: sum of interior dihedral angles - (n - 2) pi."""
    tri = elems[:, :3]
    X = nodes[tri]
    fn = np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0])
    fn /= np.linalg.norm(fn, axis=1, keepdims=True)
    edge_faces = {}
    for f, (a, b, c) in enumerate(tri):
        for u, v in ((a, b), (b, c), (c, a)):
            edge_faces.setdefault((min(u, v), max(u, v)), []).append(f)
    omega = np.zeros(len(nodes))
    deg = np.zeros(len(nodes), int)
    for (u, v), fs in edge_faces.items():
        assert len(fs) == 2
        dih = math.pi - math.acos(max(-1.0, min(1.0, float(np.dot(fn[fs[0]], fn[fs[1]])))))
        for w in (u, v):
            omega[w] += dih
            deg[w] += 1
    return omega - (deg - 2) * math.pi


def test_gauss_identity_flat_sphere(oracle_lib):
    O = oracle_lib
    m = I.icosphere(3)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    rows = np.arange(0, m.n_nodes, 7)
    _, _, d0 = O.assemble(m.nodes, m.elems, ci, nchi, rows=rows)
    omega = _solid_angles_flat(m.nodes, m.elems)[rows]
    assert np.max(np.abs(d0 + omega / (4 * math.pi))) < 2e-6


@pytest.mark.parametrize("elem_type", [I.TRI3, I.TRI6])
def test_gauss_identity_cube_faces_edges_corners(oracle_lib, elem_type):
    O = oracle_lib
    m = I.cube(4, elem_type)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    _, _, d0 = O.assemble(m.nodes, m.elems, ci, nchi)
    on = np.isclose(np.abs(m.nodes), 1.0).sum(axis=1)     # 1 face, 2 edge, 3 corner
    want = {1: -0.5, 2: -0.25, 3: -0.125}
    for c, w in want.items():
        assert np.max(np.abs(d0[on == c] - w)) < 2e-6, c


def test_gauss_identity_curved_sphere_converges(oracle_lib):
    O = oracle_lib
    errs = []
    for lev in (1, 2):
        m = I.icosphere(lev, I.TRI6)
        ci, nchi = O.chi_index(m.nodes, m.elems)
        _, _, d0 = O.assemble(m.nodes, m.elems, ci, nchi)
        errs.append(np.max(np.abs(d0 + 0.5)))
    assert errs[1] < errs[0] / 3 and errs[1] < 5e-3


def _point_source_error(O, m, xs, green=0, k=0.0, sign=-1):
    ci, nchi = O.chi_index(m.nodes, m.elems)
    D, S, d0 = O.assemble(m.nodes, m.elems, ci, nchi, green, k)
    if green == 0:
        phi_ex, chi_e = I.point_source(m, xs)
        D, S = D.real, S.real
    else:
        phi_ex, chi_e = I.helmholtz_point_source(m, xs, k)
    chi = O.chi_from_elem(ci, nchi, chi_e)
    A = np.diag(1.0 + d0) + sign * D
    phi = O.solve_dense(A, -S @ chi)
    err = phi - phi_ex
    return math.sqrt(np.mean(np.abs(err) ** 2))


SPHERE_SRC = (0.1, 0.2, -0.15)
CUBE_SRC = (0.2, -0.1, 0.3)


@pytest.mark.parametrize("table,level,etype", [
    ("sphere_laplace_tri3", 2, I.TRI3), ("sphere_laplace_tri3", 3, I.TRI3),
    ("sphere_laplace_tri6", 1, I.TRI6), ("sphere_laplace_tri6", 2, I.TRI6)])
def test_point_source_sphere_matches_paper_error(oracle_lib, table, level, etype):
    O = oracle_lib
    m = I.icosphere(level, etype)
    eps = _point_source_error(O, m, SPHERE_SRC)
    row = [r for r in GOLD[table]["rows"] if r["N"] == m.n_nodes][0]
    assert row["eps_direct"] / 10 < eps < 3 * row["eps_direct"], (eps, row)


@pytest.mark.parametrize("table,n,etype,N", [
    ("cube_laplace_tri3", 8, I.TRI3, 431), ("cube_laplace_tri6", 4, I.TRI6, 378)])
def test_point_source_cube_matches_paper_error(oracle_lib, table, n, etype, N):
    """The paper's cubes are unstructured GMSH meshes; ours have the nearest
    vertex count (386 vs 431 and 378)."""
    O = oracle_lib
    m = I.cube(n, etype)
    eps = _point_source_error(O, m, CUBE_SRC)
    row = [r for r in GOLD[table]["rows"] if r["N"] == N][0]
    assert row["eps_direct"] / 10 < eps < 3 * row["eps_direct"], (eps, row)


def test_printed_sign_fails_point_source(oracle_lib):
    """Eq. 1 printed as  C phi = int (G dphi/dn - phi dG/dn)  with the
    exterior C of Eq. 2 cannot reproduce the exterior point-source field;
    A = C - D, B = -S can."""
    O = oracle_lib
    m = I.icosphere(2, I.TRI6)
    good = _point_source_error(O, m, SPHERE_SRC, sign=-1)
    bad = _point_source_error(O, m, SPHERE_SRC, sign=+1)
    assert good < 1e-3 and bad > 100 * good


def test_chi_multi_index_cube_and_sphere(oracle_lib):
    O = oracle_lib
    m = I.cube(3, I.TRI3)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    on = np.isclose(np.abs(m.nodes), 1.0).sum(axis=1)
    per_node = {}
    for e in range(m.n_elems):
        for a in range(3):
            per_node.setdefault(int(m.elems[e, a]), set()).add(int(ci[e, a]))
    for node, s in per_node.items():
        assert len(s) == on[node]
    assert nchi == int(on.sum())
    s = I.icosphere(2, I.TRI6)
    ci, nchi = O.chi_index(s.nodes, s.elems)
    assert nchi == s.n_nodes


def test_helmholtz_point_source_matches_paper_error(oracle_lib):
    O = oracle_lib
    m = I.icosphere(3)
    eps = _point_source_error(O, m, SPHERE_SRC, green=1, k=2.0)
    row = GOLD["sphere_helmholtz_k2_tri3"]["rows"][0]
    assert row["eps_direct"] / 3 < eps < 3 * row["eps_direct"], eps


def test_mie_low_frequency_and_bem(oracle_lib):
    """The series tends to a uniform unit field as ka -> 0, and the BEM
    scattered field on a level-2 6-node sphere matches it at ka = 1."""
    O = oracle_lib
    ct = np.linspace(-1, 1, 7)
    assert np.max(np.abs(O.mie_rigid_sphere_total(1e-4, ct) - 1.0)) < 1e-3
    ka = 1.0
    m = I.icosphere(2, I.TRI6)
    ci, nchi = O.chi_index(m.nodes, m.elems)
    A, B, d0 = O.operators(m.nodes, m.elems, ci, nchi, O.HELMHOLTZ, ka)
    chi = O.chi_from_elem(ci, nchi, I.plane_wave_rigid(m, ka))
    phi = O.solve_dense(A, B @ chi)
    mie = O.mie_rigid_sphere_scattered(ka, m.nodes[:, 2])
    assert np.linalg.norm(phi - mie) / np.linalg.norm(mie) < 5e-3
