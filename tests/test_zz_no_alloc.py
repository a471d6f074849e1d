"""The product that allocates nothing (bem_matvec_noalloc), through the C ABI.

It serves callers that cannot allocate device memory at the point of the call
(real-time loops that must not synchronise the device, hosts whose device
memory belongs to another allocator).  It must give the same result as
bem_matvec, on two calls in a row (the shared scratch array keeps the previous
call's contents), and refuse plans whose scratch exceeds the fixed array.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu

MATVEC_TOL = 1e-6          # the tolerance the float64 product tests use
NOALLOC_BYTES = 48 << 20   # size of the library's fixed scratch array


def _run(P, op, fn, x):
    import torch
    xd = torch.tensor(x, device="cuda", dtype=torch.float64)
    yd = torch.full((P.n_phi,), float("nan"), device="cuda", dtype=torch.float64)
    fn(P.plan, op, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("mesh,prm", [
    (lambda: I.icosphere(3), dict(p=8, leaf_size=32, eta=2.0)),
    (lambda: I.cube(8, I.TRI6), dict(p=10, leaf_size=32, eta=2.0, precision=bem.BEM_MIXED)),
])
def test_noalloc_matches_matvec_twice(mesh, prm):
    P = Plan(mesh(), **prm)
    try:
        for op, n in ((bem.BEM_OP_A, P.n_phi), (bem.BEM_OP_B, P.n_chi)):
            x = I.random_vector(n, 7 + op)
            ref = _run(P, op, bem.bem_matvec, x)
            first = _run(P, op, bem.bem_matvec_noalloc, x)
            second = _run(P, op, bem.bem_matvec_noalloc, x)
            assert rel_l2(first, ref) <= MATVEC_TOL
            assert rel_l2(second, ref) <= MATVEC_TOL
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
