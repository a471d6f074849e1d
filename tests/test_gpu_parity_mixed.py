"""GPU parity of the mixed-precision form (float32 near field and expansions,
float64 Krylov) against the float64 oracle, through the C ABI.

Stated errors: the product within 2e-6 relative L2 of the dense oracle (the
float32 operator's rounding plus the expansion truncation), the solution
within 1e-5 of the oracle's LU solve.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu

MX_MATVEC_TOL = 2e-6
MX_SOLVE_TOL = 1e-5

CASES = {
    "sphere642": (lambda: I.icosphere(3), dict(p=8, leaf_size=32, eta=2.0), (0.1, 0.2, -0.15)),
    "cube8_tri6": (lambda: I.cube(8, I.TRI6), dict(p=10, leaf_size=32, eta=2.0), (0.2, -0.1, 0.3)),
    "sphere_tri6_l2": (lambda: I.icosphere(2, I.TRI6), dict(p=8, leaf_size=16, eta=2.0), (0.1, 0.2, -0.15)),
    "cube6_p9": (lambda: I.cube(6, I.TRI6), dict(p=9, leaf_size=24, eta=2.0), (0.2, -0.1, 0.3)),
    "cube8_p12": (lambda: I.cube(8, I.TRI6), dict(p=12, leaf_size=32, eta=2.0), (0.2, -0.1, 0.3)),
}


@pytest.mark.parametrize("p", [11, 12])
def test_two_part_class_images(p):
    """Orders 11 and 12: the class-matrix image no longer fits shared memory
    whole, so the tcgen05 M2L brings it in two parts per tile.  The product
    must still run on the tensor cores and match the float64 plan's product
    at the same order within the mixed form's 2e-6."""
    m = I.icosphere(3, I.TRI6)
    prm = dict(p=p, leaf_size=32, eta=2.0)
    Pm = Plan(m, precision=bem.BEM_MIXED, **prm)
    Pd = Plan(m, **prm)
    try:
        assert Pm.stats()["m2l_tensor_cores"] == 1
        for op, n, seed in ((bem.BEM_OP_A, Pm.n_phi, 3), (bem.BEM_OP_B, Pm.n_chi, 4)):
            x = I.random_vector(n, seed)
            e = rel_l2(Pm.matvec(op, x), Pd.matvec(op, x))
            print(f"p = {p}, op {op}: mixed vs float64 {e:.3e}")
            assert e <= MX_MATVEC_TOL, e
        assert bem.bem_plan_device_status(Pm.plan) == 0
    finally:
        Pm.close()
        Pd.close()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_matvec_and_solve(oracle_lib, name):
    mk, prm, src = CASES[name]
    m = mk()
    P = Plan(m, precision=bem.BEM_MIXED, **prm)
    try:
        A, B, _ = oracle_lib.operators(m.nodes, m.elems, P.chi_idx, P.n_chi)
        x = I.random_vector(P.n_phi, 1)
        xs = I.random_vector(P.n_chi, 2)
        ea = rel_l2(P.matvec(bem.BEM_OP_A, x), A @ x)
        eb = rel_l2(P.matvec(bem.BEM_OP_B, xs), B @ xs)
        print(f"mixed {name}: product errors A {ea:.3e} B {eb:.3e}")
        assert ea <= MX_MATVEC_TOL and eb <= MX_MATVEC_TOL, (ea, eb)
        _, chi_e = I.point_source(m, src)
        chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, chi_e)
        ref = oracle_lib.solve_dense(A, B @ chi)
        phi, code, info = P.solve(chi, tol=1e-10)
        assert code == bem.BEM_OK
        assert rel_l2(phi, ref) <= MX_SOLVE_TOL, (rel_l2(phi, ref), info.rel_residual, info.iters)
        assert bem.bem_plan_device_status(P.plan) == 0
    finally:
        P.close()


def test_stage_times_launch_count_and_peaks():
    import torch
    m = I.icosphere(3)
    P = Plan(m, p=8, leaf_size=32, eta=2.0)
    try:
        x = torch.randn(P.n_phi, device="cuda", dtype=torch.float64)
        y = torch.empty_like(x)
        c0 = bem.bem_launch_count()
        bem.bem_matvec(P.plan, bem.BEM_OP_A, x, y)
        torch.cuda.synchronize()
        st = P.stats()
        assert st["graph_kernels_A"] > 5
        assert bem.bem_launch_count() - c0 == st["graph_kernels_A"] + 1   # + the slot kernel
        ms = bem.bem_plan_stage_times(P.plan, bem.BEM_OP_A, x, y, reps=3)
        assert set(ms) == set(bem.STAGE_NAMES) and all(v >= 0 for v in ms.values())
        y2 = y.clone()
        bem.bem_matvec(P.plan, bem.BEM_OP_A, x, y)
        torch.cuda.synchronize()
        assert torch.allclose(y, y2, rtol=0, atol=0)       # deterministic
        f32 = bem.bem_measure_peak(0)
        f64 = bem.bem_measure_peak(1)
        assert 1.0 < f32 < 500.0 and 0.01 < f64 < 500.0
    finally:
        P.close()
