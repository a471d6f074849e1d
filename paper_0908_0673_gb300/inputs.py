"""Seeded synthetic inputs shaped like the paper's test cases (Section 4).

The paper tests on a unit sphere made by successive refinement of an initial
surface and on a cube of edge 2 centred on the origin, with first- and
second-order triangles, and drives both with the field of a point source
placed inside the surface (Section 4).  This module generates those meshes and
that boundary data.  It holds none of the method's arithmetic: no shape-function
geometry, no quadrature, no Green's-function integrals.  Both the oracle and
the CUDA path take its arrays as plain inputs.

Conventions shared by every generator:

* ``nodes``  float64 [n_nodes, 3]
* ``elems``  int32 [n_elems, npe]; npe = 3 (flat 3-node triangle) or 6
  (6-node triangle: corners 0, 1, 2, then mid-sides 3 (0-1), 4 (1-2), 5 (2-0)).
  Corners run counter-clockwise seen from outside, so the normal is outward.
* ``normals`` float64 [n_elems, npe, 3]: the exact outward normal of the
  *true* surface (sphere, cube face, ellipsoid) at each element node.  It is
  used only to build Neumann data; the method computes its own element normals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TRI3 = 1
TRI6 = 2


@dataclass
class Mesh:
    name: str
    nodes: np.ndarray          # float64 [n_nodes, 3]
    elems: np.ndarray          # int32 [n_elems, npe]
    elem_type: int             # TRI3 or TRI6
    normals: np.ndarray        # float64 [n_elems, npe, 3], exact surface normals
    info: dict = field(default_factory=dict)

    @property
    def npe(self) -> int:
        return self.elems.shape[1]

    @property
    def n_nodes(self) -> int:
        return self.nodes.shape[0]

    @property
    def n_elems(self) -> int:
        return self.elems.shape[0]


# ----------------------------------------------------------------------------
# Sphere: subdivided icosahedron
# ----------------------------------------------------------------------------

def _icosahedron():
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, g, 0], [1, g, 0], [-1, -g, 0], [1, -g, 0],
        [0, -1, g], [0, 1, g], [0, -1, -g], [0, 1, -g],
        [g, 0, -1], [g, 0, 1], [-g, 0, -1], [-g, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    # orient every face outward
    for t in range(len(f)):
        a, b, c = v[f[t]]
        if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
            f[t, 1], f[t, 2] = f[t, 2], f[t, 1]
    return v, f


def _subdivide(verts, faces):
    verts = list(map(tuple, verts))
    cache = {}

    def mid(i, j):
        key = (min(i, j), max(i, j))
        if key not in cache:
            m = np.add(verts[i], verts[j])
            m = m / np.linalg.norm(m)
            cache[key] = len(verts)
            verts.append(tuple(m))
        return cache[key]

    out = []
    for a, b, c in faces:
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    return np.array(verts, dtype=np.float64), np.array(out, dtype=np.int64)


def _add_midside_nodes(verts, faces, project):
    """Turn a 3-node mesh into 6-node triangles; ``project`` maps each new
    mid-side point (the chord midpoint) onto the true surface."""
    verts = [np.asarray(p) for p in verts]
    cache = {}

    def mid(i, j):
        key = (min(i, j), max(i, j))
        if key not in cache:
            cache[key] = len(verts)
            verts.append(project(0.5 * (verts[i] + verts[j])))
        return cache[key]

    el = []
    for a, b, c in faces:
        el.append((a, b, c, mid(a, b), mid(b, c), mid(c, a)))
    return np.array(verts, dtype=np.float64), np.array(el, dtype=np.int64)


def icosphere(level: int, elem_type: int = TRI3, radius: float = 1.0) -> Mesh:
    """Icosahedron subdivided ``level`` times, vertices projected onto the
    sphere.  Level 3 gives 1280 triangles and 642 vertices; level 6 with
    6-node triangles gives 81,920 elements and 163,842 nodes."""
    v, f = _icosahedron()
    for _ in range(level):
        v, f = _subdivide(v, f)
    if elem_type == TRI6:
        v, f = _add_midside_nodes(v, f, lambda p: p / np.linalg.norm(p))
    v = v * radius
    nrm = v[f] / np.linalg.norm(v[f], axis=2, keepdims=True)
    return Mesh(f"icosphere{level}-{'tri6' if elem_type == TRI6 else 'tri3'}",
                v, f.astype(np.int32), elem_type, nrm,
                {"level": level, "radius": radius})


def geodesic(freq: int, elem_type: int = TRI6, axes=(1.0, 1.0, 1.0)) -> Mesh:
    """Frequency-``freq`` geodesic sphere: every icosahedron face cut into
    freq^2 triangles on a barycentric grid, points projected onto the unit
    sphere, then scaled by the semi-axes ``axes`` (an ellipsoid unless all are
    1).  20 freq^2 elements; 10 freq^2 + 2 nodes (tri3) or 40 freq^2 + 2
    (tri6, whose mid-side nodes are the odd points of the grid of frequency
    2 freq, so they lie on the surface).  Points on an icosahedron edge are
    computed once, from the edge's lower-numbered vertex, so neighbouring faces
    share them exactly."""
    if freq < 1:
        raise ValueError("freq must be >= 1")
    V, Fc = _icosahedron()
    F = freq * (2 if elem_type == TRI6 else 1)          # grid frequency
    edges = {}
    for a, b, c in Fc:
        for u, v in ((a, b), (b, c), (c, a)):
            edges.setdefault((min(u, v), max(u, v)), len(edges))
    n_int = (F - 1) * (F - 2) // 2                      # interior points per face
    base_e, base_f = 12, 12 + 30 * (F - 1)
    pts = np.zeros((base_f + 20 * n_int, 3))
    pts[:12] = V
    t = np.arange(1, F)[:, None] / F
    for (lo, hi), e in edges.items():
        pts[base_e + e * (F - 1): base_e + (e + 1) * (F - 1)] = V[lo] + (V[hi] - V[lo]) * t
    ii, jj = np.meshgrid(np.arange(F + 1), np.arange(F + 1), indexing="ij")
    keep = ii + jj <= F
    ii, jj = ii[keep], jj[keep]
    kk = F - ii - jj
    interior = (ii > 0) & (jj > 0) & (kk > 0)
    gidx = np.empty((20, F + 1, F + 1), np.int64)
    for f, (a, b, c) in enumerate(Fc):
        w = np.stack([kk, ii, jj], 1)                    # weights of a, b, c
        ids = np.array([a, b, c])
        g = np.empty(len(ii), np.int64)
        nz = (w > 0).sum(1)
        vert = nz == 1
        g[vert] = ids[np.argmax(w[vert], 1)]
        edge = nz == 2
        for r in np.nonzero(edge)[0]:
            (p, q), = [tuple(ids[w[r] > 0])]
            lo, hi = min(p, q), max(p, q)
            s = w[r][ids == hi][0]                      # steps from lo toward hi
            g[r] = base_e + edges[(lo, hi)] * (F - 1) + s - 1
        first = base_f + f * n_int
        g[interior] = first + np.arange(n_int)
        pts[first: first + n_int] = (V[a] * kk[interior, None] + V[b] * ii[interior, None]
                                     + V[c] * jj[interior, None]) / F
        gidx[f][ii, jj] = g
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    s = 2 if elem_type == TRI6 else 1
    el = []
    i, j = np.meshgrid(np.arange(freq), np.arange(freq), indexing="ij")
    up = (i + j) <= freq - 1
    dn = (i + j) <= freq - 2
    for f in range(20):
        G = gidx[f]
        for msk, corners in ((up, ((0, 0), (1, 0), (0, 1))), (dn, ((1, 0), (1, 1), (0, 1)))):
            I0, J0 = s * i[msk], s * j[msk]
            cs = [(I0 + s * di, J0 + s * dj) for di, dj in corners]
            cols = [G[ci, cj] for ci, cj in cs]
            if elem_type == TRI6:
                for p, q in ((0, 1), (1, 2), (2, 0)):
                    cols.append(G[(cs[p][0] + cs[q][0]) // 2, (cs[p][1] + cs[q][1]) // 2])
            el.append(np.stack(cols, 1))
    elems = np.concatenate(el).astype(np.int32)
    a = np.asarray(axes, dtype=np.float64)
    nodes = pts * a
    g = nodes[elems] / (a * a)
    nrm = g / np.linalg.norm(g, axis=2, keepdims=True)
    kind = "sphere" if np.all(a == 1.0) else "ellipsoid"
    return Mesh(f"geodesic{freq}-{kind}-{'tri6' if elem_type == TRI6 else 'tri3'}", nodes, elems,
                elem_type, nrm, {"freq": freq, "axes": a.tolist()})


def ellipsoid(level: int, axes, elem_type: int = TRI6) -> Mesh:
    """Sphere mesh scaled by semi-axes ``axes``; mid-side nodes are placed on
    the ellipsoid by scaling the sphere-projected chord midpoints."""
    a = np.asarray(axes, dtype=np.float64)
    base = icosphere(level, elem_type)
    v = base.nodes * a
    g = v[base.elems] / (a * a)
    nrm = g / np.linalg.norm(g, axis=2, keepdims=True)
    return Mesh(f"ellipsoid{level}-{a.tolist()}", v, base.elems.copy(), elem_type, nrm,
                {"level": level, "axes": a.tolist()})


# ----------------------------------------------------------------------------
# Cube [-1, 1]^3, faces graded toward the edges, seeded diagonal split
# ----------------------------------------------------------------------------

# (normal axis, side) -> in-plane axes (u, v) with e_u x e_v = outward normal
_CUBE_FACES = [
    (0, 1, (1, 2)), (0, 0, (2, 1)),
    (1, 1, (2, 0)), (1, 0, (0, 2)),
    (2, 1, (0, 1)), (2, 0, (1, 0)),
]


def graded_coords(n: int, grade: float) -> np.ndarray:
    """n+1 points on [-1, 1] clustered toward both ends by a tanh map."""
    u = np.linspace(-1.0, 1.0, n + 1)
    if grade <= 0.0:
        return u
    t = np.tanh(grade * u) / math.tanh(grade)
    t[0], t[-1] = -1.0, 1.0
    return t


def cube(n: int, elem_type: int = TRI6, grade: float = 1.2, seed: int = 0) -> Mesh:
    """Cube of edge 2 centred on the origin.  Each face is an n x n grid of
    quads (1-D coordinates graded toward the edges, identical on every face so
    the mesh is conforming), each quad split along a diagonal chosen by a
    seeded coin.  6-node triangles put their mid-side nodes at the midpoints of
    the straight edges.  Gives 12 n^2 elements."""
    even = graded_coords(n, grade)
    if elem_type == TRI6:
        c = np.empty(2 * n + 1)
        c[0::2] = even
        c[1::2] = 0.5 * (even[:-1] + even[1:])
        step = 2
    else:
        c = even
        step = 1
    T = len(c)
    rng = np.random.default_rng(seed)
    index = {}
    nodes = []

    def node(ijk):
        if ijk not in index:
            index[ijk] = len(nodes)
            nodes.append((c[ijk[0]], c[ijk[1]], c[ijk[2]]))
        return index[ijk]

    elems, nrms, faces = [], [], []
    for fid, (ax, side, (ua, va)) in enumerate(_CUBE_FACES):
        fixed = T - 1 if side == 1 else 0
        nvec = np.zeros(3)
        nvec[ax] = 1.0 if side == 1 else -1.0

        def gid(u, v):
            ijk = [0, 0, 0]
            ijk[ax] = fixed
            ijk[ua] = u
            ijk[va] = v
            return node(tuple(ijk))

        flips = rng.integers(0, 2, size=(n, n))
        for i in range(n):
            for j in range(n):
                u0, v0 = i * step, j * step
                u1, v1 = u0 + step, v0 + step
                p00, p10, p11, p01 = (u0, v0), (u1, v0), (u1, v1), (u0, v1)
                if flips[i, j] == 0:
                    tris = [(p00, p10, p11), (p00, p11, p01)]
                else:
                    tris = [(p00, p10, p01), (p10, p11, p01)]
                for a, b, d in tris:
                    corner = [gid(*a), gid(*b), gid(*d)]
                    if elem_type == TRI6:
                        def m(p, q):
                            return gid((p[0] + q[0]) // 2, (p[1] + q[1]) // 2)
                        corner += [m(a, b), m(b, d), m(d, a)]
                    elems.append(corner)
                    nrms.append(np.tile(nvec, (len(corner), 1)))
                    faces.append(fid)
    nodes = np.array(nodes, dtype=np.float64)
    return Mesh(f"cube{n}-{'tri6' if elem_type == TRI6 else 'tri3'}", nodes,
                np.array(elems, dtype=np.int32), elem_type, np.array(nrms),
                {"n": n, "grade": grade, "seed": seed, "face": np.array(faces, dtype=np.int32)})


# ----------------------------------------------------------------------------
# Boundary data
# ----------------------------------------------------------------------------

def point_source(mesh: Mesh, xs):
    """Unit Laplace point source at ``xs`` inside the surface (Section 4):
    returns (phi at every node, dphi/dn at every element node [E, npe]) using
    the exact surface normals."""
    xs = np.asarray(xs, dtype=np.float64)
    d = mesh.nodes - xs
    r = np.linalg.norm(d, axis=1)
    phi = 1.0 / (4.0 * math.pi * r)
    de = mesh.nodes[mesh.elems] - xs                      # [E, npe, 3]
    re = np.linalg.norm(de, axis=2)
    grad = -de / (4.0 * math.pi * re[..., None] ** 3)
    chi = np.sum(grad * mesh.normals, axis=2)
    return phi, chi


def helmholtz_point_source(mesh: Mesh, xs, k: float):
    """Outgoing Helmholtz point source exp(jkR)/(4 pi R) at ``xs`` (time
    factor exp(-j omega t)): (phi at nodes, dphi/dn at element nodes)."""
    xs = np.asarray(xs, dtype=np.float64)
    r = np.linalg.norm(mesh.nodes - xs, axis=1)
    phi = np.exp(1j * k * r) / (4.0 * math.pi * r)
    de = mesh.nodes[mesh.elems] - xs
    re = np.linalg.norm(de, axis=2)
    dGdr = np.exp(1j * k * re) * (1j * k * re - 1.0) / (4.0 * math.pi * re ** 2)
    chi = dGdr * np.sum(de * mesh.normals, axis=2) / re
    return phi, chi


def plane_wave_rigid(mesh: Mesh, k: float, direction=(0.0, 0.0, 1.0)):
    """Scattered-field Neumann data for a rigid body hit by exp(jk d.x):
    dphi_s/dn = -d(phi_inc)/dn at every element node [E, npe]."""
    d = np.asarray(direction, dtype=np.float64)
    x = mesh.nodes[mesh.elems]
    inc = np.exp(1j * k * (x @ d))
    return -1j * k * inc * (mesh.normals @ d)


def random_vector(n: int, seed: int, complex_: bool = False) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n)
    if complex_:
        v = v + 1j * rng.standard_normal(n)
    return v
