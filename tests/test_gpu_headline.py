"""Parity at the benchmarked configuration, through the C ABI: the graded
cube of 45 x 45 quads per face (24,300 6-node triangles, split rule seed 0),
p = 10, separation factor 2, the leaf size the autotuner picks for this size
class, mixed precision (float32 near field and expansions, tcgen05 M2L,
float64 Krylov) -- the plan the benchmark times.

* A x and B x on 2000 seeded rows against the oracle's matrix-free float64
  rows, within the mixed form's stated 2e-6 relative L2;
* the mixed solve of the benchmark's point-source problem against the plain
  float64 solve on the same mesh, within 1e-5 (the float64 solve is held to
  the oracle's LU solve on the smaller meshes of the float64 parity tests);
* the tensor-core M2L is the form that ran, and its bounded waits never gave up.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I, tune

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu

MX_MATVEC_TOL = 2e-6
MX_SOLVE_TOL = 1e-5
SOURCE = (0.2, -0.1, 0.3)


@pytest.fixture(scope="module")
def cube45():
    return I.cube(45, I.TRI6, grade=1.2, seed=0)


def test_headline_mixed_rows_vs_oracle(oracle_lib, cube45):
    m = cube45
    prm = tune.choose(int(m.n_elems), bem.BEM_LAPLACE, bem.BEM_MIXED)
    assert prm["p"] == 10 and prm["eta"] == 2.0
    P = Plan(m, **prm)
    try:
        st = P.stats()
        assert st["m2l_tensor_cores"] == 1
        rows = np.sort(np.random.default_rng(0).choice(P.n_phi, 2000, replace=False))
        x = I.random_vector(P.n_phi, 5)
        xs = I.random_vector(P.n_chi, 6)
        ya = P.matvec(bem.BEM_OP_A, x)[rows]
        yb = P.matvec(bem.BEM_OP_B, xs)[rows]
        assert bem.bem_plan_device_status(P.plan) == 0
        ra = oracle_lib.apply_rows(m.nodes, m.elems, P.chi_idx, oracle_lib.OP_A, x, rows)
        rb = oracle_lib.apply_rows(m.nodes, m.elems, P.chi_idx, oracle_lib.OP_B, xs, rows)
        ea, eb = rel_l2(ya, ra), rel_l2(yb, rb)
        print(f"headline mixed rows: A {ea:.3e} B {eb:.3e}, leaf {prm['leaf_size']}, "
              f"{st['n_inter']} pairs, {st['m2l_classes']} classes")
        assert ea <= MX_MATVEC_TOL and eb <= MX_MATVEC_TOL, (ea, eb)
    finally:
        P.close()


def test_headline_mixed_solve_vs_f64(cube45):
    m = cube45
    _, chi_e = I.point_source(m, SOURCE)
    prm_mx = tune.choose(int(m.n_elems), bem.BEM_LAPLACE, bem.BEM_MIXED)
    prm_64 = dict(prm_mx, precision=bem.BEM_F64)
    out = {}
    for name, prm in (("mixed", prm_mx), ("f64", prm_64)):
        P = Plan(m, **prm)
        try:
            chi = np.zeros(P.n_chi)
            chi[P.chi_idx.ravel()] = chi_e.ravel()
            phi, code, info = P.solve(chi, restart=30, tol=1e-10, max_iter=600)
            assert code == bem.BEM_OK and info.status == bem.BEM_OK, (name, info.rel_residual)
            out[name] = (phi, info)
        finally:
            P.close()
    err = rel_l2(out["mixed"][0], out["f64"][0])
    print(f"headline mixed vs f64 solve: {err:.3e} (mixed residual {out['mixed'][1].rel_residual:.2e}, "
          f"{out['mixed'][1].iters} steps; f64 {out['f64'][1].iters} steps)")
    assert out["f64"][1].rel_residual <= 1e-10
    assert err <= MX_SOLVE_TOL
