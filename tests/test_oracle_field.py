"""The oracle's off-surface field (the representation of Eq. 1 evaluated from
surface data) pinned against closed forms, with the exact surface data of
known exterior solutions:

* Laplace: the field of an interior unit point source is reproduced outside
  the sphere and the representation vanishes inside (C(x) = 0 there);
* Helmholtz: the Mie series for the field scattered by a rigid sphere;
* the error falls at the rate of 6-node triangles (x8 or more per refinement),
  so a dropped term, a sign error or a transposed operand cannot hide below it.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import inputs as I

XS = np.array([0.1, 0.2, -0.15])


def _dirs(n, seed):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def _laplace_errors(O, level):
    m = I.icosphere(level, I.TRI6)
    idx, nchi = O.chi_index(m.nodes, m.elems)
    phi, chi_e = I.point_source(m, XS)
    chi = O.chi_from_elem(idx, nchi, chi_e)
    d = _dirs(40, 0)
    errs = {}
    for R in (1.2, 2.0, 5.0, 0.5):
        pts = d * R
        ref_mag = np.linalg.norm(1.0 / (4 * np.pi * np.linalg.norm(pts - XS, axis=1)))
        exact = 1.0 / (4 * np.pi * np.linalg.norm(pts - XS, axis=1)) if R > 1 else 0.0
        u = O.field(m.nodes, m.elems, idx, phi, chi, pts)
        errs[R] = np.linalg.norm(u - exact) / ref_mag
    return errs


def test_laplace_point_source_field(oracle_lib):
    e2, e3 = _laplace_errors(oracle_lib, 2), _laplace_errors(oracle_lib, 3)
    for R in (1.2, 2.0, 5.0):
        assert e3[R] <= 2e-5, (R, e3[R])
        assert e2[R] / e3[R] >= 8.0
    assert e3[0.5] <= 5e-6 and e2[0.5] / e3[0.5] >= 8.0        # zero inside the body


def test_helmholtz_mie_field(oracle_lib):
    O, k = oracle_lib, 2.0
    d = _dirs(40, 1)
    errs = []
    for level in (2, 3):
        m = I.icosphere(level, I.TRI6)
        idx, nchi = O.chi_index(m.nodes, m.elems)
        chi = O.chi_from_elem(idx, nchi, I.plane_wave_rigid(m, k))
        phi = O.mie_rigid_sphere_scattered(k, m.nodes[:, 2])
        e = []
        for R in (1.3, 3.0):
            u = O.field(m.nodes, m.elems, idx, phi, chi, d * R, O.HELMHOLTZ, k)
            ex = O.mie_rigid_sphere_field(k, 1.0, R, d[:, 2])
            e.append(np.linalg.norm(u - ex) / np.linalg.norm(ex))
        errs.append(max(e))
    assert errs[1] <= 5e-5 and errs[0] / errs[1] >= 8.0


def test_mie_field_on_the_surface(oracle_lib):
    ct = np.linspace(-1, 1, 9)
    a = oracle_lib.mie_rigid_sphere_field(3.0, 1.0, 1.0, ct)
    b = oracle_lib.mie_rigid_sphere_scattered(3.0, ct)
    assert np.max(np.abs(a - b)) < 1e-12
