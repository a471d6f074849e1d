"""Concurrent solves (bem_batch_*), through the C ABI.

Each result must be the same alone (bem_solve) and in the mix: four plans of
different meshes, Green's functions and precisions go through a batch with
fewer slots than solves, so later solves are admitted while earlier ones run.
The refusals (plan already in the batch, no free slot, releasing a running
slot, a wait that times out) are checked on the host path.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu


def _problems():
    out = []
    m = I.icosphere(3)
    out.append((Plan(m, p=8, leaf_size=32, eta=2.0), I.point_source(m, (0.1, 0.2, -0.15))[1]))
    m = I.cube(8, I.TRI6)
    out.append((Plan(m, p=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED), I.point_source(m, (0.2, -0.1, 0.3))[1]))
    m = I.icosphere(2, I.TRI6)
    out.append((Plan(m, bem.BEM_HELMHOLTZ, 2.0, p=10, leaf_size=16, eta=2.0), I.plane_wave_rigid(m, 2.0)))
    m = I.ellipsoid(2, (1.0, 0.7, 1.4))
    out.append((Plan(m, p=8, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED), I.point_source(m, (0.05, 0.1, -0.2))[1]))
    return out


def _chi(P, chi_e):
    dt = np.complex128 if np.iscomplexobj(chi_e) else np.float64
    chi = np.zeros(P.n_chi, dtype=dt)
    chi[P.chi_idx.ravel()] = np.asarray(chi_e).ravel()
    return chi


def test_batch_matches_single_solves():
    import torch
    probs = _problems()
    try:
        alone = []
        for P, ce in probs:
            phi, code, info = P.solve(_chi(P, ce), tol=1e-10)
            assert code == bem.BEM_OK
            alone.append(phi)
        batch = bem.bem_batch_create(probs[0][0].ctx, 2)
        sp = bem.bem_solve_params_default(tol=1e-10)
        pending = list(range(len(probs)))
        running, result = {}, {}
        bufs = {}
        while pending or running:
            while pending and len(running) < 2:
                i = pending.pop(0)
                P, ce = probs[i]
                c = P._dev(_chi(P, ce))
                ph = torch.empty(P.n_phi, device="cuda", dtype=c.dtype)
                bufs[i] = (c, ph)
                torch.cuda.synchronize()            # chi written before its slot stream reads it
                running[bem.bem_batch_submit(batch, P.plan, c, ph, sp)] = i
            bem.bem_batch_progress(batch)
            for slot, i in list(running.items()):
                done, info = bem.bem_batch_poll(batch, slot)
                if done:
                    assert info.status == bem.BEM_OK
                    torch.cuda.synchronize()
                    result[i] = bufs[i][1].cpu().numpy()
                    bem.bem_batch_release(batch, slot)
                    del running[slot]
        bem.bem_batch_destroy(batch)
        for i, (P, _) in enumerate(probs):
            assert rel_l2(result[i], alone[i]) < 1e-12, i
    finally:
        for P, _ in probs:
            P.close()


def test_batch_refusals():
    import torch
    m = I.icosphere(3)
    P = Plan(m, p=8, leaf_size=32, eta=2.0)
    Q = Plan(I.icosphere(2), p=8, leaf_size=32, eta=2.0)
    try:
        batch = bem.bem_batch_create(P.ctx, 1)
        chi = P._dev(_chi(P, I.point_source(m, (0.1, 0.2, -0.15))[1]))
        phi = torch.empty(P.n_phi, device="cuda", dtype=torch.float64)
        torch.cuda.synchronize()
        s = bem.bem_batch_submit(batch, P.plan, chi, phi)
        with pytest.raises(bem.BemError) as e:
            bem.bem_batch_submit(batch, P.plan, chi, phi)            # same plan twice
        assert e.value.code == bem.BEM_EBUSY
        chiq = torch.zeros(Q.n_chi, device="cuda", dtype=torch.float64)
        phiq = torch.empty(Q.n_phi, device="cuda", dtype=torch.float64)
        torch.cuda.synchronize()
        with pytest.raises(bem.BemError) as e:
            bem.bem_batch_submit(batch, Q.plan, chiq, phiq)          # no free slot
        assert e.value.code == bem.BEM_EBUSY
        done, _ = bem.bem_batch_poll(batch, s)
        if not done:
            with pytest.raises(bem.BemError) as e:
                bem.bem_batch_release(batch, s)                      # still running
            assert e.value.code == bem.BEM_EBUSY
        try:                                                         # a zero wait gives up at once
            bem.bem_batch_wait(batch, s, 0.0)
            assert bem.bem_batch_poll(batch, s)[0]
        except bem.BemError as err:
            assert err.code == bem.BEM_ETIMEOUT and not bem.bem_batch_poll(batch, s)[0]
        bem.bem_batch_wait(batch, s, 600.0)
        done, info = bem.bem_batch_poll(batch, s)
        assert done and info.status == bem.BEM_OK and info.rel_residual <= 1e-10
        bem.bem_batch_release(batch, s)
        s2 = bem.bem_batch_submit(batch, Q.plan, chiq, phiq)          # slot reusable; b = 0 ends at once
        bem.bem_batch_wait(batch, s2, 600.0)
        bem.bem_batch_release(batch, s2)
        bem.bem_batch_destroy(batch)
    finally:
        P.close()
        Q.close()
