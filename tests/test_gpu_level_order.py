"""Level-dependent expansion order (Section 3.6, end: L_l = min(L_max,
L_min + l_max - l)) through the C ABI (bem_fmm_params.p_min).

* p_min = 0 and p_min = p give the uniform product bit for bit;
* Laplace: the product with orders p_min..p lies between the uniform
  products at p_min and at p against the dense oracle operator;
* Helmholtz at k = 8: the error falls from uniform order 10 through the
  level-dependent orders 10..16 and 13..16 to uniform order 16 (the large
  boxes, where k h is large, get the high orders);
* the mixed form with level-dependent orders against its float64 twin, and
  a solve against the Mie series."""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu


def _prod(m, green, k, x, **prm):
    P = Plan(m, green, k, **prm)
    try:
        return P.matvec(bem.BEM_OP_A, x), P
    finally:
        P.close()


def test_uniform_equivalence():
    m = I.icosphere(3)
    x = I.random_vector(m.n_nodes, 3)
    y0, _ = _prod(m, bem.BEM_LAPLACE, 0.0, x, p=8, leaf_size=16, eta=2.0)
    y1, _ = _prod(m, bem.BEM_LAPLACE, 0.0, x, p=8, leaf_size=16, eta=2.0, p_min=8)
    assert np.array_equal(y0, y1)


def test_laplace_between_uniform_orders(oracle_lib):
    m = I.icosphere(4)
    P = Plan(m, p=10, leaf_size=16, eta=2.0)
    try:
        A, _, _ = oracle_lib.operators(m.nodes, m.elems, P.chi_idx, P.n_chi)
    finally:
        P.close()
    x = I.random_vector(m.n_nodes, 4)
    ref = A @ x
    e = {}
    for name, prm in (("hi", dict(p=10)), ("lo", dict(p=6)), ("var", dict(p=10, p_min=6))):
        y, _ = _prod(m, bem.BEM_LAPLACE, 0.0, x, leaf_size=16, eta=2.0, **prm)
        e[name] = rel_l2(y, ref)
    print("laplace product errors", e)
    assert e["var"] <= 1.5 * e["lo"] and e["var"] >= 0.5 * e["hi"]
    assert e["var"] <= 1e-4


def test_helmholtz_k8(oracle_lib):
    """The error falls monotonically from uniform order 10 through orders
    10..16 and 13..16 to uniform order 16: the level-dependent product sits
    between its smallest and its largest uniform order, and raising the
    smallest-box order p_min tightens it."""
    k = 8.0
    m = I.icosphere(4)
    P = Plan(m, bem.BEM_HELMHOLTZ, k, p=10, leaf_size=16, eta=2.0)
    try:
        A, _, _ = oracle_lib.operators(m.nodes, m.elems, P.chi_idx, P.n_chi, oracle_lib.HELMHOLTZ, k)
    finally:
        P.close()
    x = I.random_vector(m.n_nodes, 5, complex_=True)
    ref = A @ x
    e = {}
    for name, prm in (("p16", dict(p=16)), ("p10", dict(p=10)), ("var10", dict(p=16, p_min=10)),
                      ("var13", dict(p=16, p_min=13))):
        y, _ = _prod(m, bem.BEM_HELMHOLTZ, k, x, leaf_size=16, eta=2.0, **prm)
        e[name] = rel_l2(y, ref)
    ym, _ = _prod(m, bem.BEM_HELMHOLTZ, k, x, leaf_size=16, eta=2.0, p=16, p_min=10, precision=bem.BEM_MIXED)
    e["var10_mixed"] = rel_l2(ym, ref)
    print("helmholtz k=8 product errors", e)
    assert e["p16"] <= e["var13"] * 1.05 and e["var13"] <= e["var10"] * 1.05 and e["var10"] <= e["p10"] * 0.5
    assert abs(e["var10_mixed"] - e["var10"]) <= 2e-6


def test_solve_mie_level_order(oracle_lib):
    k = 8.0
    m = I.geodesic(12, I.TRI6)
    P = Plan(m, bem.BEM_HELMHOLTZ, k, p=16, p_min=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED)
    try:
        chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, I.plane_wave_rigid(m, k))
        phi, code, info = P.solve(chi, tol=1e-10, max_iter=600)
        mie = oracle_lib.mie_rigid_sphere_scattered(k, m.nodes[:, 2])
        err = rel_l2(phi, mie)
        print("k=8 level-order mixed solve vs Mie", err, info.iters)
        assert code == bem.BEM_OK and err <= 2e-2
    finally:
        P.close()
