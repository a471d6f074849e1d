"""GPU parity of the Helmholtz path (Eq. 1b, G = exp(jkR) / (4 pi R)) against
the complex float64 oracle, through the C ABI.

* stored correction (complex) equal to the oracle's;
* the float64 product within 1e-6 relative L2 of the dense oracle, and equal
  to the oracle's four-step product on the same tree up to rounding;
* the solve of the rigid-sphere plane-wave problem within 1e-5 of the oracle's
  LU solve, and within the discretisation error of the Mie series;
* the mixed form within its stated errors (2e-6 product, 1e-5 solve).
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, coo_sum, rel_l2

pytestmark = pytest.mark.gpu

K = 2.0
PRM = dict(p=10, leaf_size=16, eta=2.0)


@pytest.fixture(scope="module")
def sphere():
    m = I.icosphere(2, I.TRI6)
    P = Plan(m, bem.BEM_HELMHOLTZ, K, **PRM)
    yield P
    P.close()


def test_helmholtz_correction(oracle_lib, sphere):
    P = sphere
    ref = oracle_lib.correction(P.m.nodes, P.m.elems, P.chi_idx, oracle_lib.HELMHOLTZ, K)
    got = bem.bem_plan_export_correction(P.plan, complex_=True)
    scale = max(np.max(np.abs(ref["D"])), np.max(np.abs(ref["S"])))
    for part, cc, vv in (("D", ref["col_phi"], ref["D"]), ("S", ref["col_chi"], ref["S"])):
        r = coo_sum(ref["row"], cc, vv)
        g = coo_sum(got["row" + part], got["col" + part], got["val" + part])
        assert r.keys() == g.keys()
        assert max(abs(g[k] - r[k]) for k in r) < 1e-11 * scale


def test_helmholtz_matvec(oracle_lib, sphere):
    P = sphere
    A, B, d0 = oracle_lib.operators(P.m.nodes, P.m.elems, P.chi_idx, P.n_chi, oracle_lib.HELMHOLTZ, K)
    x = I.random_vector(P.n_phi, 1, complex_=True)
    xs = I.random_vector(P.n_chi, 2, complex_=True)
    ya, yb = P.matvec(bem.BEM_OP_A, x), P.matvec(bem.BEM_OP_B, xs)
    assert rel_l2(ya, A @ x) <= 1e-6 and rel_l2(yb, B @ xs) <= 1e-6
    # same tree and truncation as the oracle's fast product
    T = oracle_lib.Tree(P.m.nodes, P.m.elems, B=PRM["leaf_size"], eta=PRM["eta"])
    corr = oracle_lib.correction(P.m.nodes, P.m.elems, P.chi_idx, oracle_lib.HELMHOLTZ, K)
    dg = bem.bem_plan_diagonal(P.plan, P.n_phi) - 1.0
    ref = oracle_lib.fmm_apply(T, P.chi_idx, oracle_lib.OP_A, x, dg, corr, PRM["p"], oracle_lib.HELMHOLTZ, K)
    assert rel_l2(ya, ref) < 1e-9


def test_helmholtz_solve_vs_lu_and_mie(oracle_lib, sphere):
    P = sphere
    A, B, _ = oracle_lib.operators(P.m.nodes, P.m.elems, P.chi_idx, P.n_chi, oracle_lib.HELMHOLTZ, K)
    chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, I.plane_wave_rigid(P.m, K))
    ref = oracle_lib.solve_dense(A, B @ chi)
    phi, code, info = P.solve(chi, tol=1e-10)
    assert code == bem.BEM_OK and info.rel_residual <= 1e-10
    assert rel_l2(phi, ref) <= 1e-5
    mie = oracle_lib.mie_rigid_sphere_scattered(K, P.m.nodes[:, 2])
    assert rel_l2(phi, mie) < 1e-2


def test_helmholtz_mixed(oracle_lib):
    m = I.icosphere(2, I.TRI6)
    P = Plan(m, bem.BEM_HELMHOLTZ, K, precision=bem.BEM_MIXED, **PRM)
    try:
        A, B, _ = oracle_lib.operators(m.nodes, m.elems, P.chi_idx, P.n_chi, oracle_lib.HELMHOLTZ, K)
        x = I.random_vector(P.n_phi, 3, complex_=True)
        assert rel_l2(P.matvec(bem.BEM_OP_A, x), A @ x) <= 2e-6
        chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, I.plane_wave_rigid(m, K))
        ref = oracle_lib.solve_dense(A, B @ chi)
        phi, code, info = P.solve(chi, tol=1e-10)
        assert code == bem.BEM_OK and rel_l2(phi, ref) <= 1e-5
    finally:
        P.close()
