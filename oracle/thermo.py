"""Bulk thermodynamics of an equation of state p(rho): Maxwell construction.

TEST INFRASTRUCTURE ONLY (expected values for the coexistence tests).

App. B of the paper determines coexistence densities by a Maxwell
construction on p as a function of the specific volume v = 1/rho.  This
module does it with the equal-area rule written out: find the pressure P for
which the loop of p(v) cuts off equal areas, i.e.

    int_{v_l}^{v_g} (p(v) - P) dv = 0,

with v_l < v_m < v_g the three roots of p(v) = P.  The integral is done by
adaptive quadrature, so nothing here shares the closed-form chemical
potential that the workload generator uses.
"""
import numpy as np
from scipy.integrate import quad
from scipy.optimize import brentq


def spinodal(p, rho_lo, rho_hi, n=20001):
    """Densities where dp/drho changes sign on [rho_lo, rho_hi] (numerical derivative)."""
    r = np.linspace(rho_lo, rho_hi, n)
    pv = np.array([p(x) for x in r])
    dp = np.gradient(pv, r)
    idx = np.where(np.diff(np.sign(dp)) != 0)[0]
    if len(idx) < 2:
        raise ValueError("no unstable region: the EOS has no loop")
    return float(r[idx[0]]), float(r[idx[-1] + 1])


def maxwell(p, rho_lo, rho_hi):
    """(rho_g, rho_l, P) of the equal-area construction for p(rho) with a loop inside [rho_lo, rho_hi]."""
    rs1, rs2 = spinodal(p, rho_lo, rho_hi)
    pv = lambda v: p(1.0 / v)
    p_min, p_max = p(rs2), p(rs1)  # local minimum at the liquid spinodal, maximum at the gas spinodal

    def roots(P):
        # gas branch: rho in (rho_lo, rs1); liquid branch: rho in (rs2, rho_hi)
        rg = brentq(lambda x: p(x) - P, rho_lo, rs1, xtol=1e-15, rtol=1e-15)
        rl = brentq(lambda x: p(x) - P, rs2, rho_hi, xtol=1e-15, rtol=1e-15)
        return rg, rl

    def area(P):
        rg, rl = roots(P)
        val, _ = quad(lambda v: pv(v) - P, 1.0 / rl, 1.0 / rg, epsabs=1e-15, epsrel=1e-13, limit=200)
        return val

    lo = max(p_min, p(rho_lo)) + 1e-12 * abs(p_max)
    hi = p_max - 1e-12 * abs(p_max)
    P = brentq(area, lo, hi, xtol=1e-15, rtol=1e-14)
    rg, rl = roots(P)
    return rg, rl, P


def vdw_pressure(a, b, T):
    return lambda rho: rho * T / (1.0 - b * rho) - a * rho * rho
