"""Pins of the oracle's equilibrium and equation of state.

Equilibrium (Sec. III): its moments up to fourth order must be the closed
forms the paper gives (mass, momentum, Euler stress p delta + rho u u, phi^eq,
psi^eq).  EOS (App. B): derivatives against numerical differentiation, the
psi-sine closed form against direct quadrature of psi, and the worked example
of App. B against the three admissibility conditions the paper states.
"""
import math
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("lat", [O.D2Q21, O.D3Q59])
def test_equilibrium_moments(lat):
    rng = np.random.default_rng(11)
    c, _ = O.velocities(lat)
    d = 3 if lat == O.D3Q59 else 2
    c = c[:, :d].astype(float)
    I = np.eye(d)
    for _ in range(6):
        rho = rng.uniform(0.5, 1.5)
        cs2 = rng.uniform(0.45, 0.9)
        u = rng.normal(0.0, 0.05, d)
        n = O.neq(lat, rho, cs2, u)
        p = rho * cs2
        np.testing.assert_allclose(n.sum(), rho, rtol=1e-14)
        np.testing.assert_allclose(n @ c, rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", n, c, c)
        np.testing.assert_allclose(pi, p * I + rho * np.outer(u, u), atol=1e-14)
        phi = np.einsum("i,ia,ib,ig->abg", n, c, c, c)
        want = rho * cs2 * (np.einsum("ab,g->abg", I, u) + np.einsum("ag,b->abg", I, u) + np.einsum("bg,a->abg", I, u))
        np.testing.assert_allclose(phi, want, atol=1e-14)
        psi = np.einsum("i,ia,ib,ig,id->abgd", n, c, c, c, c)
        uu = np.outer(u, u)
        want4 = (rho * cs2 ** 2 * (np.einsum("ab,gd->abgd", I, I) + np.einsum("ag,bd->abgd", I, I)
                                    + np.einsum("ad,bg->abgd", I, I))
                 + rho * cs2 * (np.einsum("ab,gd->abgd", I, uu) + np.einsum("ag,bd->abgd", I, uu)
                                + np.einsum("ad,bg->abgd", I, uu))
                 + rho * cs2 * (np.einsum("gd,ab->abgd", I, uu) + np.einsum("bd,ag->abgd", I, uu)
                                + np.einsum("bg,ad->abgd", I, uu)))
        np.testing.assert_allclose(psi, want4, atol=1e-13)


def _num_deriv(f, x, h=1e-5):
    return (f(x - 2 * h) - 8 * f(x - h) + 8 * f(x + h) - f(x + 2 * h)) / (12 * h)


@pytest.mark.parametrize("kind,prm", [
    (O.EOS_VDW, O.eos_params(O.EOS_VDW, a=1.79, b=1.0 / 3.0, T=1.53)),
    (O.EOS_PSI_SINE, O.eos_params(O.EOS_PSI_SINE, rho1=0.5, rho2=1.0, A=1.2, cs2_rho1=0.6)),
])
def test_eos_items_are_derivatives_of_p(kind, prm):
    for rho in (0.55, 0.8, 1.1, 1.3, 1.45):
        p, dp, pm, rpp = O.eos_eval(kind, prm, rho)
        P = lambda r: O.eos_eval(kind, prm, r)[0]
        dP = lambda r: O.eos_eval(kind, prm, r)[1]
        assert abs(dp - _num_deriv(P, rho)) < 1e-8
        assert abs(rpp / rho - _num_deriv(dP, rho)) < 1e-7
        # the S1 identity p - rho p' = -rho^2 d(p/rho)/drho
        assert abs(pm + rho ** 2 * _num_deriv(lambda r: P(r) / r, rho)) < 1e-8


def _gold_app_b():
    vals = {}
    with open(os.path.join(GOLD, "app_b_example.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                vals[k] = float(v)
    return vals


def test_psi_sine_closed_form_matches_quadrature():
    """c_s^2(rho) = c_s^2(rho1) exp(int_{rho1}^{rho} psi): the oracle's closed form against quadrature."""
    g = _gold_app_b()
    prm = O.eos_params(O.EOS_PSI_SINE, rho1=g["rho1"], rho2=g["rho2"], A=g["A"], cs2_rho1=g["cs2_rho1"])
    rho1, rho2, A = g["rho1"], g["rho2"], g["A"]
    rho3 = 2 * rho2 - rho1

    def psi(r):
        return A * math.sin(math.pi * (r - rho1) / (rho2 - rho1)) if rho1 < r < rho3 else 0.0

    for rho in (0.3, 0.5, 0.7, 1.0, 1.2, 1.49, 1.6):
        integral = quad(psi, rho1, rho, limit=200, epsabs=1e-14, points=[rho3] if rho > rho3 else None)[0] if rho > rho1 else 0.0
        cs2 = g["cs2_rho1"] * math.exp(integral)
        p = O.eos_eval(O.EOS_PSI_SINE, prm, rho)[0]
        assert abs(p / rho - cs2) < 1e-11
    # c_s^2 takes the same value below rho1 and above rho3 (App. B)
    assert abs(O.eos_eval(O.EOS_PSI_SINE, prm, 0.4)[0] / 0.4 - O.eos_eval(O.EOS_PSI_SINE, prm, 1.7)[0] / 1.7) < 1e-14


def test_app_b_example_is_admissible():
    """App. B: A = 1.2 gives two-phase coexistence and positive bulk viscosity in d = 2,
    and c_s^2 stays inside the D2Q21 window."""
    g = _gold_app_b()
    prm = O.eos_params(O.EOS_PSI_SINE, rho1=g["rho1"], rho2=g["rho2"], A=g["A"], cs2_rho1=g["cs2_rho1"])
    d = int(g["d"])
    rr = np.linspace(0.2, 2.0, 3601)
    items = np.array([O.eos_eval(O.EOS_PSI_SINE, prm, r) for r in rr])
    p, dp = items[:, 0], items[:, 1]
    assert (dp < 0).any()                              # two-phase: dp/drho < 0 somewhere
    assert (rr * dp / p < 1.0 + 2.0 / d).all()         # bulk viscosity > 0 everywhere
    cs2 = p / rr
    assert cs2.min() > 0.3510760 and cs2.max() < 4.0 / 3.0
    # smaller amplitude: no loop; much larger amplitude: negative bulk viscosity
    small = O.eos_params(O.EOS_PSI_SINE, rho1=0.5, rho2=1.0, A=0.3, cs2_rho1=0.6)
    assert all(O.eos_eval(O.EOS_PSI_SINE, small, r)[1] > 0 for r in rr)
    big = O.eos_params(O.EOS_PSI_SINE, rho1=0.5, rho2=1.0, A=4.0, cs2_rho1=0.6)
    assert any(r * O.eos_eval(O.EOS_PSI_SINE, big, r)[1] / O.eos_eval(O.EOS_PSI_SINE, big, r)[0] >= 2.0 for r in rr)
