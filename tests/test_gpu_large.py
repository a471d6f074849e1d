"""A mesh beyond the scans' two-level size, through the C ABI.

The ellipsoid (semi-axes 1, 0.7, 1.6) of 220,500 6-node triangles (the size of
a served stream's large mesh) has about 19 million special pairs: more than one scan
block of blocks (4096 x 4096 values), so the pair offsets and every other
prefix sum over the pairs take the recursive path.  The mixed product on 64
seeded rows must match the oracle's matrix-free rows within the mixed form's
2e-6 relative L2.
"""
import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I, tune

from gpu_util import Plan, rel_l2

pytestmark = pytest.mark.gpu


def test_ellipsoid_220k_mixed_rows(oracle_lib):
    m = I.geodesic(105, I.TRI6, axes=(1.0, 0.7, 1.6))
    prm = tune.choose(int(m.n_elems), bem.BEM_LAPLACE, bem.BEM_MIXED)
    P = Plan(m, **prm)
    try:
        st = P.stats()
        pairs = st["corr_nnz_D"] // m.npe
        assert pairs > 4096 * 4096, pairs
        rows = np.sort(np.random.default_rng(1).choice(P.n_phi, 64, replace=False))
        x = I.random_vector(P.n_phi, 9)
        y = P.matvec(bem.BEM_OP_A, x)[rows]
        assert bem.bem_plan_device_status(P.plan) == 0
        ref = oracle_lib.apply_rows(m.nodes, m.elems, P.chi_idx, oracle_lib.OP_A, x, rows)
        e = rel_l2(y, ref)
        print(f"ellipsoid {m.n_elems} elements: {pairs} special pairs, rows rel err {e:.3e}")
        assert e <= 2e-6
    finally:
        P.close()
