"""Group solves (bem_group_*): plans of uneven size, both Green's functions
and both precisions solved in lock step, every restart cycle of the whole
group one launch of a captured graph.  Each member's solution and iteration
count must be those of bem_solve on the same plan and right-hand side; a
member left out of a solve must be untouched; the graphs are reused across
calls with new right-hand sides."""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu


def _members():
    out = []
    m = I.icosphere(3)
    out.append((Plan(m, p=8, leaf_size=32, eta=2.0), m, bem.BEM_LAPLACE, 0.0))
    m = I.cube(8, I.TRI6)
    out.append((Plan(m, p=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED), m, bem.BEM_LAPLACE, 0.0))
    m = I.icosphere(2, I.TRI6)
    out.append((Plan(m, bem.BEM_HELMHOLTZ, 2.0, p=10, leaf_size=16, eta=2.0, precision=bem.BEM_MIXED), m,
                bem.BEM_HELMHOLTZ, 2.0))
    m = I.geodesic(6, I.TRI6, axes=(0.7, 1.0, 1.5))
    out.append((Plan(m, p=10, leaf_size=32, eta=2.0), m, bem.BEM_LAPLACE, 0.0))
    m = I.cube(5, I.TRI6)
    out.append((Plan(m, bem.BEM_HELMHOLTZ, 3.0, p=10, leaf_size=24, eta=2.0), m, bem.BEM_HELMHOLTZ, 3.0))
    return out


def _chi(oracle_lib, P, m, green, k, src):
    ce = I.helmholtz_point_source(m, src, k)[1] if green == bem.BEM_HELMHOLTZ else I.point_source(m, src)[1]
    return oracle_lib.chi_from_elem(P.chi_idx, P.n_chi, ce)


def test_group_equals_single_solves(oracle_lib):
    import torch
    mem = _members()
    try:
        sp = bem.bem_solve_params_default(tol=1e-10, max_iter=600)
        group = bem.bem_group_create(mem[0][0].ctx, [P.plan for P, *_ in mem])
        srcs = [(0.1, 0.2, -0.15), (-0.2, 0.05, 0.1)]
        for r, src in enumerate(srcs):
            chis, phis, alone = [], [], []
            for i, (P, m, green, k) in enumerate(mem):
                chi = _chi(oracle_lib, P, m, green, k, src)
                ph_alone, code, info_alone = P.solve(chi, tol=1e-10, max_iter=600)
                alone.append((ph_alone, info_alone))
                left_out = r == 1 and i == 2
                cd = P._dev(chi)
                pd = torch.full((P.n_phi,), 7.0, device="cuda", dtype=cd.dtype)
                chis.append(None if left_out else cd)
                phis.append(None if left_out else pd)
                if left_out:
                    phis[-1] = None
                    kept = pd
            torch.cuda.synchronize()
            code, infos, launches = bem.bem_group_solve(group, chis, phis, sp)
            torch.cuda.synchronize()
            assert code == bem.BEM_OK and launches > 0
            for i, (P, *_r) in enumerate(mem):
                if phis[i] is None:
                    continue
                got = phis[i].cpu().numpy()
                ref, info_ref = alone[i]
                assert rel_l2(got, ref) <= 1e-12, (r, i, rel_l2(got, ref))
                assert infos[i].iters == info_ref.iters and infos[i].status == bem.BEM_OK
                assert bem.bem_plan_device_status(P.plan) == 0
            if r == 1:
                assert bool((kept == 7.0).all())                # the left-out member's output untouched
        bem.bem_group_destroy(group)
    finally:
        for P, *_r in mem:
            P.close()
