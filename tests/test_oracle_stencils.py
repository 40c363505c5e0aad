"""Pins of the oracle's finite-difference operators (Sec. IV, Table III).

Each operator must satisfy the moment conditions Sec. IV derives for it
(Eqs. cond1a/b for the first derivative, sigma0 = 0 / sigma2 = 2 for the
Laplacian, sigma4 = 1 for the traceless part, sigma2 = 0 / sigma4 = 2 for the
third derivative), and, as a consequence, reproduce the derivative of a
polynomial exactly at sites whose stencil does not cross the periodic seam.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O


def _moments(dv, tau, d):
    dv = dv[:, :d].astype(float)
    s0 = tau.sum()
    s2 = np.einsum("m,ma,mb->ab", tau, dv, dv)
    s4 = np.einsum("m,ma,mb,mc,md->abcd", tau, dv, dv, dv, dv)
    return s0, s2, s4


def _iso4(d):
    I = np.eye(d)
    return np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)


@pytest.mark.parametrize("d", [2, 3])
def test_table_three_moment_conditions(d):
    I = np.eye(d)
    # first derivative: sigma2 = 1, sigma4 = 0 (odd vector moment tau_i d_i vanishes by symmetry)
    dv, tau = O.stencil(d, O.ST_D1)
    _, s2, s4 = _moments(dv, tau, d)
    np.testing.assert_allclose(s2, I, atol=1e-15)
    np.testing.assert_allclose(s4, 0 * s4, atol=1e-15)
    # Laplacian: sigma0 = 0, sigma2 = 2
    dv, tau = O.stencil(d, O.ST_LAP)
    s0, s2, _ = _moments(dv, tau, d)
    assert abs(s0) < 1e-15
    np.testing.assert_allclose(s2, 2 * I, atol=1e-15)
    # traceless second derivative: isotropic sigma4 = 1 (with traceless d_a d_b)
    dv, tau = O.stencil(d, O.ST_TRACELESS)
    dd = dv[:, :d].astype(float)
    tl = np.einsum("ma,mb->mab", dd, dd) - np.einsum("m,ab->mab", (dd ** 2).sum(1) / d, I)
    got = np.einsum("m,mab,mc,me->abce", tau, tl, dd, dd) / 2.0
    want = 0.5 * (np.einsum("ac,be->abce", I, I) + np.einsum("ae,bc->abce", I, I)) - np.einsum("ab,ce->abce", I, I) / d
    np.testing.assert_allclose(got, want, atol=1e-15)
    # third derivative: sigma2 = 0, sigma4 = 2
    dv, tau = O.stencil(d, O.ST_D3)
    _, s2, s4 = _moments(dv, tau, d)
    np.testing.assert_allclose(s2, 0 * I, atol=1e-15)
    np.testing.assert_allclose(s4, 2 * _iso4(d), atol=1e-15)


def _poly_field(d, n, deg, rng):
    """Random polynomial of total degree <= deg on an n^d grid, with its exact derivatives."""
    import sympy as sp

    xs = sp.symbols("x y z")[:d]
    terms = [m for m in itertools.product(range(deg + 1), repeat=d) if sum(m) <= deg]
    expr = sum(sp.Rational(int(rng.integers(-5, 6)), 7) * sp.prod([x ** e for x, e in zip(xs, m)]) for m in terms)
    grids = np.meshgrid(*[np.arange(n, dtype=float) - n / 2 for _ in range(d)], indexing="ij")
    f = sp.lambdify(xs, expr, "numpy")
    # C order: axis 0 is the slowest coordinate (y in 2D, z in 3D); x is the last axis
    vals = np.broadcast_to(f(*reversed(grids)), (n,) * d).astype(float)
    return xs, expr, grids, vals


@pytest.mark.parametrize("d", [2, 3])
def test_operators_exact_on_polynomials(d):
    import sympy as sp

    rng = np.random.default_rng(3)
    n = 12
    xs, expr, grids, g = _poly_field(d, n, 4 if d == 2 else 3, rng)
    lam = lambda e: sp.lambdify(xs, e, "numpy")
    interior = tuple(slice(3, n - 3) for _ in range(d))
    coords = [gr[interior] for gr in reversed(grids)]
    D1 = O.apply_stencil(d, O.ST_D1, g)
    for a in range(d):
        want = np.broadcast_to(lam(sp.diff(expr, xs[a]))(*coords), D1[a][interior].shape)
        np.testing.assert_allclose(D1[a][interior], want, atol=1e-9)
    lap = O.apply_stencil(d, O.ST_LAP, g)
    lap_e = sum(sp.diff(expr, x, 2) for x in xs)
    if expr.as_poly().total_degree() <= 3:
        np.testing.assert_allclose(lap[interior], np.broadcast_to(lam(lap_e)(*coords), lap[interior].shape), atol=1e-9)
    D3 = O.apply_stencil(d, O.ST_D3, g)
    for a in range(d):
        want = np.broadcast_to(lam(sp.diff(lap_e, xs[a]))(*coords), D3[a][interior].shape)
        np.testing.assert_allclose(D3[a][interior], want, atol=1e-9)


@pytest.mark.parametrize("d", [2, 3])
def test_first_derivative_error_is_fifth_order(d):
    """On a periodic sine the first-derivative error falls like k^5 (O(eps^4) relative)."""
    errs = []
    for n in (16, 32):
        k = 2 * np.pi / n
        shape = (n,) * d
        x = np.arange(n, dtype=float)
        g = np.broadcast_to(np.sin(k * x), shape).copy()
        D1 = O.apply_stencil(d, O.ST_D1, g)
        exact = np.broadcast_to(k * np.cos(k * x), shape)
        errs.append(np.abs(D1[0] - exact).max())
    assert 20 < errs[0] / errs[1] < 45  # 2^5 = 32
