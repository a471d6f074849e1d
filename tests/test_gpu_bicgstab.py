"""BiCGStab (the paper's solver, Section 4) through bem_solve: the float64
solution against the oracle's LU solve (same bar as GMRES, 1e-5), against
GMRES on the same plan, a complex (Helmholtz) solve against GMRES and the
Mie series, and the mixed form against its float64 solution.  Batched and
group solves accept GMRES only."""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu

SOLVE_TOL = 1e-5


@pytest.mark.parametrize("mesh,prm,src", [
    (lambda: I.icosphere(3), dict(p=8, leaf_size=32, eta=2.0), (0.1, 0.2, -0.15)),
    (lambda: I.cube(6, I.TRI6), dict(p=10, leaf_size=24, eta=2.0), (0.2, -0.1, 0.3)),
])
def test_bicgstab_vs_lu_and_gmres(oracle_lib, mesh, prm, src):
    m = mesh()
    P = Plan(m, **prm)
    try:
        A, B, _ = oracle_lib.operators(m.nodes, m.elems, P.chi_idx, P.n_chi)
        chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, I.point_source(m, src)[1])
        ref = oracle_lib.solve_dense(A, B @ chi)
        phi, code, info = P.solve(chi, tol=1e-10, method=bem.BEM_BICGSTAB)
        print("bicgstab", info.iters, info.restarts, info.rel_residual)
        assert code == bem.BEM_OK and info.rel_residual <= 1e-10
        assert rel_l2(phi, ref) <= SOLVE_TOL
        phg, code_g, _ = P.solve(chi, tol=1e-10)
        assert code_g == bem.BEM_OK
        assert rel_l2(phi, phg) <= 1e-8
    finally:
        P.close()


def test_bicgstab_helmholtz_and_mixed(oracle_lib):
    k = 2.0
    m = I.icosphere(3, I.TRI6)
    chi_e = I.plane_wave_rigid(m, k)
    P = Plan(m, bem.BEM_HELMHOLTZ, k, p=10, leaf_size=32, eta=2.0)
    Q = Plan(m, bem.BEM_HELMHOLTZ, k, p=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED)
    try:
        chi = oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, chi_e)
        phi, code, info = P.solve(chi, tol=1e-10, method=bem.BEM_BICGSTAB)
        assert code == bem.BEM_OK, (code, info.rel_residual)
        phg, code_g, _ = P.solve(chi, tol=1e-10)
        assert rel_l2(phi, phg) <= 1e-8
        mie = oracle_lib.mie_rigid_sphere_scattered(k, m.nodes[:, 2])
        assert rel_l2(phi, mie) <= 1e-2
        phm, code_m, info_m = Q.solve(chi, tol=1e-10, method=bem.BEM_BICGSTAB)
        print("mixed bicgstab", info_m.iters, info_m.restarts, info_m.rel_residual, rel_l2(phm, phi))
        assert code_m == bem.BEM_OK and rel_l2(phm, phi) <= SOLVE_TOL
    finally:
        P.close()
        Q.close()


def test_batch_and_group_refuse_bicgstab():
    import torch
    m = I.icosphere(2)
    P = Plan(m, p=8, leaf_size=32, eta=2.0)
    try:
        sp = bem.bem_solve_params_default(method=bem.BEM_BICGSTAB)
        chi = torch.zeros(P.n_chi, device="cuda", dtype=torch.float64)
        phi = torch.zeros(P.n_phi, device="cuda", dtype=torch.float64)
        b = bem.bem_batch_create(P.ctx, 2)
        try:
            with pytest.raises(bem.BemError):
                bem.bem_batch_submit(b, P.plan, chi, phi, sp)
        finally:
            bem.bem_batch_destroy(b)
        g = bem.bem_group_create(P.ctx, [P.plan])
        try:
            with pytest.raises(bem.BemError):
                bem.bem_group_solve(g, [chi], [phi], sp)
        finally:
            bem.bem_group_destroy(g)
    finally:
        P.close()
