"""The product that allocates nothing (bem_matvec_noalloc), through the C ABI.

It serves callers that cannot allocate device memory at the point of the call
(real-time loops that must not synchronise the device, hosts whose device
memory belongs to another allocator).  It launches the same kernels as
bem_matvec on the same inputs, so its result must equal bem_matvec's bit for
bit, on two calls in a row (the shared scratch array keeps the previous call's
contents).  Before a plan's first call the array is left holding another
plan's data (a larger mesh, other values), so a stage that read scratch it had
not written would change the result.  Plans whose scratch exceeds the fixed
array are refused.  This file is collected last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan

pytestmark = pytest.mark.gpu

NOALLOC_BYTES = 48 << 20   # size of the library's fixed scratch array


def _run(P, op, fn, x):
    import torch
    dt = torch.complex128 if P.complex else torch.float64
    xd = torch.tensor(x, device="cuda", dtype=dt)
    yd = torch.full((P.n_phi,), float("nan"), device="cuda", dtype=dt)
    fn(P.plan, op, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _vec(P, n, seed):
    x = I.random_vector(n, seed)
    if P.complex:
        x = x + 1j * I.random_vector(n, seed + 100)
    return x


def _dirty_scratch():
    """Leaves the scratch array holding a different, larger plan's data."""
    D = Plan(I.icosphere(4), p=9, leaf_size=16, eta=2.0)
    try:
        _run(D, bem.BEM_OP_A, bem.bem_matvec_noalloc, _vec(D, D.n_phi, 99))
    finally:
        D.close()


@pytest.mark.parametrize("mesh,green,k,prm", [
    (lambda: I.icosphere(3), bem.BEM_LAPLACE, 0.0, dict(p=8, leaf_size=32, eta=2.0)),
    (lambda: I.cube(8, I.TRI6), bem.BEM_LAPLACE, 0.0, dict(p=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED)),
    (lambda: I.icosphere(2, I.TRI6), bem.BEM_HELMHOLTZ, 2.0, dict(p=10, leaf_size=16, eta=2.0)),
    (lambda: I.icosphere(2, I.TRI6), bem.BEM_HELMHOLTZ, 2.0,
     dict(p=10, leaf_size=16, eta=2.0, precision=bem.BEM_MIXED)),
], ids=["laplace-f64", "laplace-mixed", "helmholtz-f64", "helmholtz-mixed"])
def test_noalloc_matches_matvec_twice(mesh, green, k, prm):
    P = Plan(mesh(), green=green, k=k, **prm)
    try:
        for op, n in ((bem.BEM_OP_A, P.n_phi), (bem.BEM_OP_B, P.n_chi)):
            x = _vec(P, n, 7 + op)
            ref = _run(P, op, bem.bem_matvec, x)
            assert np.all(np.isfinite(ref))
            _dirty_scratch()
            first = _run(P, op, bem.bem_matvec_noalloc, x)
            second = _run(P, op, bem.bem_matvec_noalloc, x)
            assert np.array_equal(first, ref)
            assert np.array_equal(second, ref)
    finally:
        P.close()


def test_noalloc_keeps_the_current_device():
    """The call switches to the plan's device only for its own enqueue."""
    import torch
    P = Plan(I.icosphere(2), p=6, leaf_size=16, eta=2.0)
    try:
        before = torch.cuda.current_device()
        _run(P, bem.BEM_OP_A, bem.bem_matvec_noalloc, _vec(P, P.n_phi, 3))
        assert torch.cuda.current_device() == before
    finally:
        P.close()


def test_noalloc_rejects_plans_beyond_the_array():
    """Level-4 6-node sphere, 4 vertices per leaf, p = 16: moments and locals
    alone need more than the 48 MiB array."""
    P = Plan(I.icosphere(4, I.TRI6), p=16, leaf_size=4, eta=2.0)
    try:
        st = P.stats()
        need = st["n_quad"] * 8 + 2 * st["n_boxes"] * st["n_p"] * 8 + P.n_phi * 8
        assert need > NOALLOC_BYTES
        import torch
        x = torch.zeros(P.n_phi, device="cuda", dtype=torch.float64)
        y = torch.zeros_like(x)
        with pytest.raises(bem.BemError) as e:
            bem.bem_matvec_noalloc(P.plan, bem.BEM_OP_A, x, y)
        assert e.value.code == bem.BEM_EINVAL and "scratch" in str(e.value)
    finally:
        P.close()
