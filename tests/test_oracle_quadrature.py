"""Pins for the oracle's quadrature (not the oracle checked against itself).

* the 7-point rule integrates every monomial of degree <= 5 on the reference
  triangle exactly and fails at degree 6 (closed form a! b! / (a+b+2)!);
* the Duffy self rule reproduces the analytic integral of 1/R over a flat
  triangle seen from a vertex or an edge midpoint;
* the near-singular subdivision rule agrees with a brute-force uniformly
  refined rule written here in numpy.
"""
import math

import numpy as np
import pytest

from paper_0908_0673_gb300 import inputs as I


def test_rule7_degree5_exact_degree6_not(oracle_lib):
    O = oracle_lib
    s, t, w = O.rule7()
    assert abs(w.sum() - 0.5) < 1e-15
    assert np.all(s > 0) and np.all(t > 0) and np.all(s + t < 1)
    worst6 = 0.0
    for deg in range(7):
        for a in range(deg + 1):
            b = deg - a
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = float(np.sum(w * s ** a * t ** b))
            if deg <= 5:
                assert abs(got - exact) < 1e-15, (a, b)
            else:
                worst6 = max(worst6, abs(got - exact) / exact)
    assert worst6 > 1e-4


def _flat_vertex_integral(P, A, B):
    """int over triangle PAB of 1/|x - P| dS = h (asinh(tB/h) - asinh(tA/h)),
    h the distance from P to line AB, tA, tB the signed positions of A, B
    along AB measured from the foot of the perpendicular."""
    P, A, B = map(np.asarray, (P, A, B))
    u = (B - A) / np.linalg.norm(B - A)
    F = A + np.dot(P - A, u) * u
    h = np.linalg.norm(P - F)
    tA, tB = np.dot(A - F, u), np.dot(B - F, u)
    return h * (math.asinh(tB / h) - math.asinh(tA / h))


@pytest.mark.parametrize("npe,n_duffy,tol", [(3, 12, 1e-7), (6, 12, 1e-7), (3, 20, 1e-12), (6, 20, 1e-12)])
def test_duffy_self_integral_flat_triangle(oracle_lib, npe, n_duffy, tol):
    O = oracle_lib
    st = O.Settings(n_duffy=n_duffy)
    X = np.array([[0.0, 0.0, 0.0], [1.3, 0.2, 0.0], [0.3, 0.9, 0.0]])
    if npe == 6:
        X = np.vstack([X, 0.5 * (X[0] + X[1]), 0.5 * (X[1] + X[2]), 0.5 * (X[2] + X[0])])
    elems = np.arange(npe, dtype=np.int32)[None, :]
    ci = np.arange(npe, dtype=np.int32)[None, :]
    D, S, d0 = O.assemble(X, elems, ci, npe, st=st)
    for i in range(npe):
        got = S[i].real.sum() * 4.0 * math.pi           # int G dS * 4 pi = int 1/R dS
        if i < 3:
            P, A, B = X[i], X[(i + 1) % 3], X[(i + 2) % 3]
            exact = _flat_vertex_integral(P, A, B)
        else:
            M = X[i]
            u, v = [(0, 1), (1, 2), (2, 0)][i - 3]
            w = 3 - u - v
            exact = _flat_vertex_integral(M, X[v], X[w]) + _flat_vertex_integral(M, X[w], X[u])
        assert abs(got - exact) < tol * exact, (i, got, exact)
        # the double layer of a flat element seen from its own plane vanishes
        assert np.all(np.abs(D[i]) < 1e-14)


def _brute(X, npe, xi, level):
    """Uniformly refined 7-point rule (4^level pieces), numpy, independent of
    the oracle's code: returns (int L_a G dS, int L_a dG/dn dS) for one flat or
    curved triangle and target xi (Laplace)."""
    s7, t7, w7 = (np.array(v) for v in zip(*[
        (1 / 3, 1 / 3, 9 / 80)] + [(a, b, wgt) for (a, b, wgt) in _orbit()]))
    tris = [np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])]
    for _ in range(level):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(v) for v in ([a, ab, ca], [ab, b, bc], [ca, bc, c], [ab, bc, ca])]
        tris = nxt
    T = np.array(tris)                                   # [n, 3, 2]
    det = np.abs((T[:, 1, 0] - T[:, 0, 0]) * (T[:, 2, 1] - T[:, 0, 1])
                 - (T[:, 1, 1] - T[:, 0, 1]) * (T[:, 2, 0] - T[:, 0, 0]))
    ps = T[:, 0, 0][:, None] + s7 * (T[:, 1, 0] - T[:, 0, 0])[:, None] + t7 * (T[:, 2, 0] - T[:, 0, 0])[:, None]
    pt = T[:, 0, 1][:, None] + s7 * (T[:, 1, 1] - T[:, 0, 1])[:, None] + t7 * (T[:, 2, 1] - T[:, 0, 1])[:, None]
    wq = (w7[None, :] * det[:, None]).ravel()
    s, t = ps.ravel(), pt.ravel()
    L0, L1, L2 = 1 - s - t, s, t
    if npe == 3:
        N = np.stack([L0, L1, L2], 1)
        Ns = np.tile([-1.0, 1.0, 0.0], (len(s), 1))
        Nt = np.tile([-1.0, 0.0, 1.0], (len(s), 1))
    else:
        N = np.stack([L0 * (2 * L0 - 1), L1 * (2 * L1 - 1), L2 * (2 * L2 - 1), 4 * L0 * L1, 4 * L1 * L2, 4 * L2 * L0], 1)
        Ns = np.stack([-(4 * L0 - 1), 4 * L1 - 1, 0 * s, 4 * (L0 - L1), 4 * L2, -4 * L2], 1)
        Nt = np.stack([-(4 * L0 - 1), 0 * s, 4 * L2 - 1, -4 * L1, 4 * L1, 4 * (L0 - L2)], 1)
    x = N @ X
    n = np.cross(Ns @ X, Nt @ X)
    J = np.linalg.norm(n, axis=1)
    n /= J[:, None]
    r = xi - x
    R = np.linalg.norm(r, axis=1)
    G = 1 / (4 * np.pi * R)
    dG = np.sum(r * n, 1) / (4 * np.pi * R ** 3)
    return (wq * J * G) @ N, (wq * J * dG) @ N


def _orbit():
    r15 = math.sqrt(15.0)
    a, b = (6 - r15) / 21, (9 + 2 * r15) / 21
    c, d = (6 + r15) / 21, (9 - 2 * r15) / 21
    wa, wc = (155 - r15) / 2400, (155 + r15) / 2400
    return [(a, a, wa), (b, a, wa), (a, b, wa), (c, c, wc), (d, c, wc), (c, d, wc)]


@pytest.mark.parametrize("npe", [3, 6])
@pytest.mark.parametrize("tau,depth,tolS,tolD", [(2.0, 6, 2e-7, 1e-5), (6.0, 10, 1e-9, 3e-8)])
def test_near_singular_rule_vs_brute_force(oracle_lib, npe, tau, depth, tolS, tolD):
    """Target 0.15 below an edge of a flat or curved element: the subdivided
    rule matches a uniformly 4^8-refined rule, and converges as tau grows."""
    O = oracle_lib
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.0]])
    if npe == 6:   # curved: lift the mid-side nodes
        X = np.vstack([X, 0.5 * (X[0] + X[1]) + [0, 0, 0.05], 0.5 * (X[1] + X[2]) + [0, 0, 0.04],
                       0.5 * (X[2] + X[0]) + [0, 0, 0.03]])
    tgt = np.array([0.5, -0.15, 0.07])
    nodes = np.vstack([X, tgt])
    elems = np.arange(npe, dtype=np.int32)[None, :]
    D, S, d0 = O.assemble(nodes, elems, elems.copy(), npe, rows=[npe], st=O.Settings(tau, depth))
    Sb, Db = _brute(X, npe, tgt, 8)
    assert np.max(np.abs(S[0, :npe].real - Sb)) < tolS * np.max(np.abs(Sb))
    assert np.max(np.abs(D[0, :npe].real - Db)) < tolD * np.max(np.abs(Db))


def test_regular_rule_matches_brute_force_far(oracle_lib):
    O = oracle_lib
    m = I.icosphere(1, I.TRI6)
    X = m.nodes[m.elems[0]]
    tgt = m.nodes[m.elems[40][0]]
    # pick an element far from the target: the regular rule is in use
    D, S, d0 = O.assemble(np.vstack([X, tgt]), np.arange(6, dtype=np.int32)[None, :],
                          np.arange(6, dtype=np.int32)[None, :], 6, rows=[6])
    Sb, Db = _brute(X, 6, tgt, 5)
    assert np.max(np.abs(S[0, :6].real - Sb)) < 1e-4 * np.max(np.abs(Sb))
