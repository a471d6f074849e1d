"""CPU checks of the C ABI library (no GPU calls): it builds for sm_103a,
loads, exports every symbol include/bem.h declares, and its host-side mesh
preparation (sharp-edge multi-indexing, Section 2.3) agrees with the oracle
bit for bit."""
import os
import re

import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = bem.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert sorted(bem.EXPORTS) == names


def test_params_defaults():
    p = bem.bem_fmm_params_default()
    assert (p.p, p.leaf_size, p.eta, p.leaf_descend, p.n_duffy, p.tau_near, p.max_subdiv, p.p_min) == \
        (8, 64, 2.0, 1, 12, 2.0, 6, 0)
    s = bem.bem_solve_params_default()
    assert (s.restart, s.tol, s.max_iter, s.method) == (30, 1e-10, 1000, bem.BEM_GMRES)
    # the struct the binding declares has the C layout: method is the last field
    import ctypes as C
    assert C.sizeof(bem.bem_solve_params) == 24 and bem.bem_solve_params.method.offset == 20
    assert C.sizeof(bem.bem_fmm_params) == 48 and bem.bem_fmm_params.p_min.offset == 44


@pytest.mark.parametrize("mesh", [lambda: I.cube(5, I.TRI3), lambda: I.cube(4, I.TRI6),
                                  lambda: I.icosphere(2, I.TRI6), lambda: I.ellipsoid(1, (1.0, 0.6, 1.7))])
def test_host_multi_index_matches_oracle(oracle_lib, mesh):
    m = mesh()
    h = bem.bem_mesh_create(None, m.nodes, m.elems, m.elem_type)
    try:
        n_phi, n_chi = bem.bem_mesh_sizes(h)
        ci = bem.bem_mesh_chi_index(h, m.n_elems, m.npe)
    finally:
        bem.bem_mesh_destroy(h)
    ref, nref = oracle_lib.chi_index(m.nodes, m.elems)
    assert n_phi == m.n_nodes and n_chi == nref
    assert np.array_equal(ci, ref)


def test_mesh_create_rejects_bad_input():
    m = I.cube(2, I.TRI3)
    bad = m.elems.copy()
    bad[3, 1] = m.n_nodes + 5
    with pytest.raises(bem.BemError) as e:
        bem.bem_mesh_create(None, m.nodes, bad, bem.BEM_TRI3)
    assert e.value.code == bem.BEM_EINVAL and "out of range" in str(e.value)
    with pytest.raises(bem.BemError):
        bem.bem_mesh_create(None, m.nodes, m.elems, 7)
    deg = m.elems.copy()
    deg[0, 2] = deg[0, 1]
    with pytest.raises(bem.BemError):
        bem.bem_mesh_create(None, m.nodes, deg, bem.BEM_TRI3)


def test_solve_stop_rule():
    """The host decision after a true residual, without a GPU: a mixed solve
    whose restart cycle fails to halve the residual stops, as converged only
    within the stall floor 1e-6 (the second-kind equation's condition number of
    order 10 keeps the solution within the 1e-5 bar there); above it the status
    is BEM_ENOCONV.  float64 solves never take the stall exit."""
    rule = bem.bem_solve_stop_rule
    F, M = bem.BEM_F64, bem.BEM_MIXED
    ok, enc = bem.BEM_OK, bem.BEM_ENOCONV
    # tolerance reached
    assert rule(F, 1e-10, 1, 5e-11, 2.0, 3, 100) == (True, ok)
    assert rule(M, 1e-10, 1, 4e-8, 2.0, 3, 100) == (True, ok)       # mixed target max(tol, 1e-7)
    assert rule(M, 1e-10, 1, 9e-8, 2.0, 3, 100) == (True, ok)
    assert rule(M, 1e-10, 1, 1.2e-7, 2.0, 3, 100) == (False, None)
    assert rule(F, 1e-10, 1, 4e-8, 2.0, 3, 100) == (False, None)
    # stall of a mixed solve: converged near the float32 floor, not above 1e-6
    assert rule(M, 1e-10, 2, 1.5e-7, 2e-7, 40, 100) == (True, ok)
    assert rule(M, 1e-10, 2, 9e-7, 1.0e-6, 40, 100) == (True, ok)
    assert rule(M, 1e-10, 2, 1e-3, 1.5e-3, 40, 100) == (True, enc)
    assert rule(M, 1e-10, 3, 2e-6, 3e-6, 40, 100) == (True, enc)
    assert rule(M, 1e-4, 2, 5e-5, 6e-5, 40, 100) == (True, ok)      # a loose tol raises the floor
    # halving, or the first residual, is no stall
    assert rule(M, 1e-10, 2, 1e-3, 2.1e-3, 40, 100) == (False, None)
    assert rule(M, 1e-10, 1, 1e-3, 2.0, 0, 100) == (False, None)
    # float64: no stall exit, only the step budget
    assert rule(F, 1e-10, 2, 1e-3, 1.5e-3, 40, 100) == (False, None)
    assert rule(F, 1e-10, 2, 1e-3, 1.5e-3, 100, 100) == (True, enc)
    assert rule(M, 1e-10, 2, 1e-3, 3e-3, 100, 100) == (True, enc)
