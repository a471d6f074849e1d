"""Pins for the oracle's Taylor machinery (Sections 3.2-3.3).

* Tausch's recursions give the same derivatives as sympy's symbolic
  differentiation of 1/(4 pi R) and exp(jkR)/(4 pi R);
* the coefficient shift (Eq. 8) is exact: moments shifted from a child centre
  equal moments computed directly about the parent centre;
* the expansion shift (Eq. 9, with binomials) is exact: the shifted local
  expansion is the same polynomial;
* P2M -> M2L -> L2P converges to the direct sum of point sources and dipoles
  at the rate set by the separation ratio.
"""
import math

import numpy as np
import pytest
import sympy as sp


def _sympy_derivs(p, r, green, k):
    x, y, z = sp.symbols("x y z", real=True)
    R = sp.sqrt(x * x + y * y + z * z)
    G = 1 / (4 * sp.pi * R) if green == 0 else sp.exp(sp.I * k * R) / (4 * sp.pi * R)
    subs = {x: r[0], y: r[1], z: r[2]}
    out = {}
    cache = {}
    for m in range(p + 1):
        for n in range(p + 1 - m):
            for kk in range(p + 1 - m - n):
                key = (m, n, kk)
                expr = G
                if m:
                    expr = sp.diff(expr, x, m)
                if n:
                    expr = sp.diff(expr, y, n)
                if kk:
                    expr = sp.diff(expr, z, kk)
                out[key] = complex(sp.N(expr.subs(subs), 30))
    return out


@pytest.mark.parametrize("green,k", [(0, 0.0), (1, 2.5)])
def test_tausch_recursion_matches_symbolic(oracle_lib, green, k):
    O = oracle_lib
    p = 5
    r = np.array([0.7, -0.4, 1.1])
    D = O.green_derivs(p, r, green, k)
    mnk = O.mindex(p)
    ref = _sympy_derivs(p, [sp.Rational(7, 10), sp.Rational(-4, 10), sp.Rational(11, 10)], green, k)
    for c, (m, n, kk) in enumerate(mnk):
        want = ref[(int(m), int(n), int(kk))]
        assert abs(D[c] - want) <= 1e-12 * max(1.0, abs(want)), (m, n, kk, D[c], want)


def test_mindex_enumeration(oracle_lib):
    O = oracle_lib
    for p in (0, 3, 8, 10):
        mnk = O.mindex(p)
        assert len(mnk) == (p + 1) * (p + 2) * (p + 3) // 6
        assert len({tuple(v) for v in mnk}) == len(mnk)
        assert np.all(mnk.sum(1)[:-1] <= mnk.sum(1)[1:])   # by degree


def _cloud(seed, n, centre, radius):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    d *= (radius * rng.random(n) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    nrm = rng.standard_normal((n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    return centre + d, nrm, rng.standard_normal(n), rng.standard_normal(n)


def test_m2m_is_exact(oracle_lib):
    O = oracle_lib
    p = 8
    c_child, c_par = np.array([0.25, -0.25, 0.25]), np.zeros(3)
    x, nrm, sig, mu = _cloud(1, 40, c_child, 0.2)
    direct = O.p2m(p, c_par, x, nrm, sig, mu)
    shifted = O.m2m(p, c_child, c_par, O.p2m(p, c_child, x, nrm, sig, mu))
    assert np.max(np.abs(shifted - direct)) < 1e-13 * np.max(np.abs(direct))


def test_l2l_is_exact(oracle_lib):
    O = oracle_lib
    p = 8
    rng = np.random.default_rng(3)
    F = rng.standard_normal(O.mindex(p).shape[0]) + 0j
    c, cp = np.zeros(3), np.array([0.25, 0.25, -0.25])
    pts = cp + 0.2 * rng.standard_normal((30, 3))
    a = O.l2p(p, c, pts, F)
    b = O.l2p(p, cp, pts, O.l2l(p, c, cp, F))
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(a))


@pytest.mark.parametrize("green,k", [(0, 0.0), (1, 1.5)])
def test_m2l_converges_to_direct_sum(oracle_lib, green, k):
    """Sources within 0.5 of c_s, targets within 0.5 of c_t, |c_t - c_s| = 3:
    ratio 1/3, so the error should shrink roughly by 3 per order."""
    O = oracle_lib
    cs, ct = np.zeros(3), np.array([3.0, 0.0, 0.0])
    x, nrm, sig, mu = _cloud(5, 30, cs, 0.5)
    tgt, _, _, _ = _cloud(6, 20, ct, 0.5)
    r = tgt[:, None, :] - x[None, :, :]
    R = np.linalg.norm(r, axis=2)
    e = np.exp(1j * k * R)
    G = e / (4 * np.pi * R)
    dG = e * (1 - 1j * k * R) * np.sum(r * nrm[None], 2) / (4 * np.pi * R ** 3)
    direct = G @ sig + dG @ mu
    errs = []
    for p in (2, 4, 6, 8, 10):
        F = O.m2l(p, ct, cs, O.p2m(p, cs, x, nrm, sig, mu), green, k)
        errs.append(np.max(np.abs(O.l2p(p, ct, tgt, F) - direct)) / np.max(np.abs(direct)))
    for a, b in zip(errs, errs[1:]):
        assert b < a / 2.5
    assert errs[-1] < 1e-5


@pytest.mark.parametrize("green,k", [(0, 0.0), (1, 2.0)])
def test_derivative_symmetry_under_signed_axis_permutations(oracle_lib, green, k):
    """The Green's functions are radial, so for r_i = s_i rhat_pi(i) the
    derivative tensors obey D_mu(r) = prod_i s_i^mu_i D_{mu o pi^-1}(rhat):
    the identity that lets interaction pairs share the translation matrix of
    a canonical offset (|components| sorted in decreasing order)."""
    import itertools
    O = oracle_lib
    p = 7
    mi = O.mindex(p)
    where = {tuple(v): i for i, v in enumerate(mi.tolist())}
    rng = np.random.default_rng(5)
    for _ in range(3):
        rhat = np.sort(np.abs(rng.uniform(1.0, 3.0, 3)))[::-1]
        Dc = O.green_derivs(p, rhat, green, k)
        for pi in itertools.permutations(range(3)):
            pinv = [pi.index(j) for j in range(3)]
            for s in itertools.product((1, -1), repeat=3):
                r = np.array([s[i] * rhat[pi[i]] for i in range(3)])
                D = O.green_derivs(p, r, green, k)
                for a, mu in enumerate(mi.tolist()):
                    g = tuple(mu[pinv[j]] for j in range(3))
                    sign = np.prod([s[i] ** mu[i] for i in range(3)])
                    assert abs(D[a] - sign * Dc[where[g]]) <= 1e-12 * (abs(D[a]) + 1e-300) + 1e-300
