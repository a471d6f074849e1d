"""The synthetic mesh generators: closed, consistently oriented outward,
conforming, nodes on the true surface, and of the stated sizes."""
import numpy as np
import pytest

from paper_0908_0673_gb300 import inputs as I


def _closed_oriented(m):
    c = m.elems[:, :3]
    de = np.concatenate([c[:, [0, 1]], c[:, [1, 2]], c[:, [2, 0]]])
    s = set(map(tuple, de.tolist()))
    return len(s) == len(de) and all((b, a) in s for a, b in s)


def _outward(m):
    x = m.nodes[m.elems[:, :3]]
    n = np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    return bool(np.all(np.einsum("ij,ij->i", n, x.mean(1)) > 0))


@pytest.mark.parametrize("freq,et", [(1, I.TRI3), (3, I.TRI3), (2, I.TRI6), (7, I.TRI6)])
def test_geodesic_sphere(freq, et):
    m = I.geodesic(freq, et)
    assert m.n_elems == 20 * freq * freq
    assert m.n_nodes == (10 if et == I.TRI3 else 40) * freq * freq + 2
    assert np.unique(m.elems).size == m.n_nodes             # no unused or duplicated node
    assert _closed_oriented(m) and _outward(m)
    assert np.abs(np.linalg.norm(m.nodes, axis=1) - 1.0).max() < 1e-14
    if et == I.TRI6:                                         # each mid-side node is shared by the two
        mids = np.concatenate([m.elems[:, 3], m.elems[:, 4], m.elems[:, 5]])   # elements on its edge
        assert np.all(np.bincount(mids, minlength=m.n_nodes)[np.unique(mids)] == 2)


def test_geodesic_matches_icosphere_counts():
    for lev in range(4):
        a, b = I.geodesic(2 ** lev, I.TRI3), I.icosphere(lev, I.TRI3)
        assert (a.n_elems, a.n_nodes) == (b.n_elems, b.n_nodes)


def test_geodesic_ellipsoid():
    ax = np.array([0.5, 1.0, 2.0])
    m = I.geodesic(4, I.TRI6, axes=ax)
    assert np.abs(np.sum((m.nodes / ax) ** 2, axis=1) - 1.0).max() < 1e-13
    assert _closed_oriented(m) and _outward(m)
    g = m.nodes[m.elems] / ax ** 2                           # exact normals along the gradient
    cosang = np.einsum("eij,eij->ei", m.normals, g / np.linalg.norm(g, axis=2, keepdims=True))
    assert np.allclose(cosang, 1.0)


def test_cube_sizes_and_orientation():
    for n, et in [(3, I.TRI3), (4, I.TRI6)]:
        m = I.cube(n, et)
        assert m.n_elems == 12 * n * n
        assert _closed_oriented(m) and _outward(m)
        assert np.allclose(np.abs(m.nodes).max(axis=1), 1.0)
