"""Serving on the GPU, through the C ABI: a Poisson stream of solve requests
(spheres, ellipsoids, cubes; Laplace and Helmholtz; several right-hand sides)
runs with continuous batching in the mixed form.  Each result must be the
same as the request solved alone on its own plan, and within 1e-5 of the
plain float64 one-at-a-time path; the admission estimate must bound every
plan's measured peak footprint."""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I, tune
from paper_0908_0673_gb300.serve import CudaEngine, Server, estimate_peak_footprint, summarize, synthetic_stream

from gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _alone(req, precision):
    import torch
    ctx = bem.bem_ctx_create(0)
    mesh = bem.bem_mesh_create(ctx, req.mesh.nodes, req.mesh.elems, req.mesh.elem_type)
    n_phi, n_chi = bem.bem_mesh_sizes(mesh)
    idx = bem.bem_mesh_chi_index(mesh, req.mesh.n_elems, req.mesh.npe)
    plan = bem.bem_plan_create(mesh, req.green, req.k,
                               bem.bem_fmm_params_default(**tune.choose(req.mesh.n_elems, req.green, precision)))
    try:
        cplx = req.green == bem.BEM_HELMHOLTZ
        out = []
        for ce in req.rhs:
            chi = np.zeros(n_chi, np.complex128 if cplx else np.float64)
            chi[idx.ravel()] = np.asarray(ce).ravel()
            cd = torch.tensor(chi, device="cuda")
            pd = torch.empty(n_phi, device="cuda", dtype=cd.dtype)
            code, _ = bem.bem_solve(plan, cd, pd, 1, bem.bem_solve_params_default(tol=1e-10, max_iter=600))
            torch.cuda.synchronize()
            out.append(pd.cpu().numpy())
        return out
    finally:
        bem.bem_plan_destroy(plan)
        bem.bem_mesh_destroy(mesh)
        bem.bem_ctx_destroy(ctx)


def test_served_results_equal_alone_and_f64():
    reqs = synthetic_stream(6, rate_per_s=200.0, elems=(600, 4000), rhs=(1, 3), seed=1)
    eng = CudaEngine(precision=bem.BEM_MIXED, max_slots=4)
    try:
        res = Server(eng, setup_threads=2, keep_phi=True).run(reqs)
    finally:
        eng.close()
    assert all(r.status == "ok" for r in res), [(r.status, r.error) for r in res]
    for q, r in zip(reqs, res):
        alone = _alone(q, bem.BEM_MIXED)
        f64 = _alone(q, bem.BEM_F64)
        for a, b, c in zip(r.phi, alone, f64):
            assert rel_l2(a, b) <= 1e-12
            assert rel_l2(a, c) <= 1e-5, (q.rid, q.green, q.k, rel_l2(a, c))
        assert r.peak_footprint <= r.reserved
    s = summarize(res)
    assert s["served"] == 6 and s["solves"] == sum(len(q.rhs) for q in reqs)


@pytest.mark.parametrize("kind,green,prec", [
    ("cube20", bem.BEM_LAPLACE, bem.BEM_MIXED), ("cube20", bem.BEM_LAPLACE, bem.BEM_F64),
    ("geo30", bem.BEM_LAPLACE, bem.BEM_MIXED), ("geo30", bem.BEM_HELMHOLTZ, bem.BEM_MIXED),
    ("ell20", bem.BEM_HELMHOLTZ, bem.BEM_F64), ("geo8", bem.BEM_LAPLACE, bem.BEM_F64)])
def test_footprint_estimate_bounds_peak(kind, green, prec):
    import torch
    m = {"cube20": lambda: I.cube(20, I.TRI6), "geo30": lambda: I.geodesic(30, I.TRI6),
         "ell20": lambda: I.geodesic(20, I.TRI6, axes=(0.6, 1.0, 1.7)),
         "geo8": lambda: I.geodesic(8, I.TRI6)}[kind]()
    ctx = bem.bem_ctx_create(0)
    mesh = bem.bem_mesh_create(ctx, m.nodes, m.elems, m.elem_type)
    k = 3.0 if green == bem.BEM_HELMHOLTZ else 0.0
    plan = bem.bem_plan_create(mesh, green, k, bem.bem_fmm_params_default(p=10, leaf_size=64, eta=2.0,
                                                                          precision=prec))
    try:
        n_phi, n_chi = bem.bem_mesh_sizes(mesh)
        dt = torch.complex128 if green == bem.BEM_HELMHOLTZ else torch.float64
        chi = torch.zeros(n_chi, device="cuda", dtype=dt)
        chi[0] = 1.0
        phi = torch.empty(n_phi, device="cuda", dtype=dt)
        bem.bem_solve(plan, chi, phi, 1, bem.bem_solve_params_default(max_iter=30))
        torch.cuda.synchronize()
        peak = bem.bem_plan_peak_footprint(plan)
        est = estimate_peak_footprint(m.n_nodes, green, prec)
        print(f"footprint {kind} green={green} prec={prec}: N={m.n_nodes} peak={peak} "
              f"B/node={peak / m.n_nodes:.0f} held={bem.bem_plan_footprint(plan)} est={est}")
        assert bem.bem_plan_footprint(plan) <= peak <= est
    finally:
        bem.bem_plan_destroy(plan)
        bem.bem_mesh_destroy(mesh)
        bem.bem_ctx_destroy(ctx)
