"""Seeded synthetic workloads: initial fields and equation-of-state parameters.

This module holds no lattice Boltzmann arithmetic.  It builds the inputs that
both the CUDA library and the CPU oracle are fed: density and velocity fields
(flat slab, droplet, spinodal noise, serving request stream) and the van der
Waals parameters in lattice units that put the bulk sound speed inside the
positivity window of the weights.

The paper runs no experiments (its numerical tests are deferred), so these
synthetic cases stand in for workloads.

Thermodynamics used (App. B of the paper frames the EOS constraints):
  * reduced van der Waals:  p_r(rho) = 8 T_r rho / (3 - rho) - 3 rho^2
    (critical point rho_c = 1, p_c = 1, T_r = T/T_c);
  * lattice units: p(rho) = P0 p_r(rho) = rho T / (1 - b rho) - a rho^2 with
    b = 1/3, a = 3 P0, T = 8 P0 T_r / 3;
  * P0 is chosen so that min p/rho over [0.98 rho_g, 1.02 rho_l] sits 2 %
    above the lower edge of the c_s^2 window (Sec. III);
  * coexistence from equal pressure and equal chemical potential
    mu = int dp / rho;
  * interfacial stiffness kappa from the width W of a tanh profile matched to
    a quartic double well: kappa = 8 W^2 g(rho_bar) / (rho_l - rho_g)^2, g the
    free-energy density above the common tangent.
"""
from dataclasses import dataclass
import math

import numpy as np

D2Q21, D3Q59 = 0, 1

#: lower and upper edge of the c_s^2 window where all weights are positive
#: (Sec. III and App. B of the paper, printed values)
CS2_WINDOW = {D2Q21: (0.3510760, 4.0 / 3.0), D3Q59: (0.3850612, 1.1917145)}


def vdw_reduced_p(rho, Tr):
    return 8.0 * Tr * rho / (3.0 - rho) - 3.0 * rho * rho


def vdw_reduced_mu(rho, Tr):
    # mu = int p'(rho)/rho drho for p_r = 8 T_r rho/(3-rho) - 3 rho^2 (b = 1/3, a = 3, T = 8 T_r/3)
    T = 8.0 * Tr / 3.0
    g = 1.0 - rho / 3.0
    return T * (math.log(rho / g) + 1.0 / g) - 6.0 * rho


def vdw_coexistence(Tr):
    """(rho_g, rho_l) of the reduced van der Waals fluid at T_r < 1 (equal p and mu).

    Newton on the two conditions, started outside the spinodal densities."""
    if not (0.0 < Tr < 1.0):
        raise ValueError("T/Tc must lie in (0, 1)")
    x = math.sqrt(1.0 - Tr)
    rg, rl = max(1.0 - 2.0 * x, 0.05), min(1.0 + 2.0 * x, 2.9)
    T = 8.0 * Tr / 3.0

    def dp(r):
        return T / (1.0 - r / 3.0) ** 2 - 6.0 * r

    for _ in range(100):
        F1 = vdw_reduced_p(rg, Tr) - vdw_reduced_p(rl, Tr)
        F2 = vdw_reduced_mu(rg, Tr) - vdw_reduced_mu(rl, Tr)
        J = np.array([[dp(rg), -dp(rl)], [dp(rg) / rg, -dp(rl) / rl]])
        step = np.linalg.solve(J, [F1, F2])
        lam = 1.0
        while lam > 1e-4 and not (0.0 < rg - lam * step[0] < 1.0 < rl - lam * step[1] < 3.0):
            lam *= 0.5
        rg, rl = rg - lam * step[0], rl - lam * step[1]
        if abs(step[0]) + abs(step[1]) < 1e-15:
            break
    if not (0.0 < rg < 1.0 < rl < 3.0):
        raise RuntimeError("coexistence solve failed")
    return float(rg), float(rl)


def _free_energy_excess(rho, Tr, rg, rl):
    """Free-energy density of the reduced vdW fluid minus its common tangent."""
    T = 8.0 * Tr / 3.0

    def F(r):  # F = rho * f with df/drho = p/rho^2; f = T ln(rho/(1 - rho/3)) - 3 rho up to a constant
        return r * (T * math.log(r / (1.0 - r / 3.0)) - 3.0 * r)

    mu = vdw_reduced_mu(rg, Tr)
    # for this f, dF/drho = f + p/rho = mu - T (constant shift); the tangent uses the same F
    slope = (F(rl) - F(rg)) / (rl - rg)
    return F(rho) - (F(rg) + slope * (rho - rg)), mu


@dataclass
class VdwParams:
    Tr: float
    lattice: int
    P0: float
    a: float
    b: float
    T: float
    rho_g: float
    rho_l: float
    cs2_min: float
    cs2_max: float

    def p(self, rho):
        return rho * self.T / (1.0 - self.b * rho) - self.a * rho * rho


def vdw_lattice_params(Tr, lattice, margin=1.02):
    """Map the reduced vdW fluid at T_r onto lattice units for the given lattice."""
    rg, rl = vdw_coexistence(Tr)
    lo, hi = 0.98 * rg, 1.02 * rl
    rr = np.linspace(lo, hi, 4001)
    pr_over_rho = vdw_reduced_p(rr, Tr) / rr
    c2min, c2max = CS2_WINDOW[lattice]
    P0 = margin * c2min / float(pr_over_rho.min())
    prm = VdwParams(Tr=Tr, lattice=lattice, P0=P0, a=3.0 * P0, b=1.0 / 3.0, T=8.0 * P0 * Tr / 3.0,
                    rho_g=rg, rho_l=rl, cs2_min=float(P0 * pr_over_rho.min()), cs2_max=float(P0 * pr_over_rho.max()))
    if prm.cs2_max >= c2max:
        raise ValueError("T/Tc too deep: c_s^2 leaves the positive-weight window")
    return prm


def kappa_for_width(prm: VdwParams, W):
    """kappa that makes the equilibrium tanh((x)/W) interface width W (quartic-well match)."""
    rbar = 0.5 * (prm.rho_g + prm.rho_l)
    g, _ = _free_energy_excess(rbar, prm.Tr, prm.rho_g, prm.rho_l)
    g *= prm.P0  # lattice pressure units
    drho = prm.rho_l - prm.rho_g
    return 8.0 * W * W * g / (drho * drho)


# --------------------------------------------------------------------------
# Initial fields.  Shapes are C order: (ny, nx) in 2D, (nz, ny, nx) in 3D.
# --------------------------------------------------------------------------

def slab_2d(nx, ny, rho_g, rho_l, half_width=16.0, centre=None, W=2.0):
    """rho(x) = rho_bar + (drho/2) tanh((half_width - |x - centre|)/W), uniform in y."""
    centre = nx / 2.0 if centre is None else centre
    x = np.arange(nx, dtype=np.float64)
    prof = 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * np.tanh((half_width - np.abs(x - centre)) / W)
    return np.ascontiguousarray(np.broadcast_to(prof, (ny, nx)))


def droplet(dims, R, rho_g, rho_l, W=4.0, centre=None):
    """Liquid sphere (disc in 2D) of radius R: rho_bar + (drho/2) tanh((R - r)/W)."""
    dims = tuple(int(v) for v in dims)
    shape = tuple(reversed(dims))
    centre = tuple(v / 2.0 for v in dims) if centre is None else tuple(centre)
    grids = np.meshgrid(*[np.arange(n, dtype=np.float64) for n in shape], indexing="ij")
    r2 = np.zeros(shape)
    for ax, g in enumerate(grids):
        c = centre[len(dims) - 1 - ax]
        r2 += (g - c) ** 2
    r = np.sqrt(r2)
    return 0.5 * (rho_l + rho_g) + 0.5 * (rho_l - rho_g) * np.tanh((R - r) / W)


def spinodal(dims, seed=0, rho_c=1.0, amplitude=0.01):
    """rho = rho_c (1 + U(-amplitude, amplitude)), drawn in C order from default_rng(seed)."""
    shape = tuple(reversed(tuple(int(v) for v in dims)))
    rng = np.random.default_rng(seed)
    return rho_c * (1.0 + rng.uniform(-amplitude, amplitude, size=shape))


def shear_wave(dims, rho, U, mode=1):
    """Uniform density with u_x = U sin(2 pi mode y / ny): the transverse-wave start."""
    dims = tuple(int(v) for v in dims)
    shape = tuple(reversed(dims))
    d = len(dims)
    ny = dims[1]
    y = np.arange(ny, dtype=np.float64)
    ux = U * np.sin(2.0 * math.pi * mode * y / ny)
    u = np.zeros((d,) + shape)
    if d == 2:
        u[0] = ux[:, None]
    else:
        u[0] = ux[None, :, None]
    return np.full(shape, float(rho)), u


@dataclass
class Request:
    rid: int
    arrival: float
    lattice: int
    side: int
    radius: float
    Tr: float
    steps: int


#: T/Tc windows of the serving requests: inside the paper's constraints and linearly stable
SERVING_TR = {D2Q21: (0.99, 0.995), D3Q59: (0.998, 0.999)}


def serving_requests(n=256, seed=1, rate=1.0):
    """The mixed request stream of the serving workload (inter-arrival Exp(1/rate))."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        lat = D2Q21 if rng.random() < 0.5 else D3Q59
        if lat == D2Q21:
            side = int(rng.choice(np.arange(64, 513, 32)))
        else:
            side = int(rng.choice(np.arange(32, 129, 16)))
        frac = rng.uniform(0.15, 0.35)
        lo, hi = SERVING_TR[lat]
        Tr = rng.uniform(lo, hi)
        steps = int(rng.integers(500, 5001))
        out.append(Request(k, t, lat, side, frac * side, Tr, steps))
    return out


# --------------------------------------------------------------------------
# The named workloads.  T/Tc and kappa lie where the paper's constraints hold
# (positive weights, positive bulk viscosity over [0.98 rho_g, 1.02 rho_l]) and
# where, in addition, the uniform coexisting phases are linearly stable under
# the method's own update; the paper never tested stability, so this is a
# reading the design notes record.
# --------------------------------------------------------------------------

#: T/Tc of the two-dimensional and three-dimensional workloads
TR_2D = 0.99
TR_3D = 0.998
#: kappa is matched to the interface width of each workload's initial tanh profile


@dataclass
class Case:
    name: str
    lattice: int
    dims: tuple
    Tr: float
    kappa: float
    eos: VdwParams
    rho: np.ndarray
    u: object = None
    gamma: float = 0.0
    rho0: float = 1.0

    @property
    def eos_abT(self):
        return self.eos.a, self.eos.b, self.eos.T


def make_case(name, dims=None, Tr=None, gamma=0.0):
    """Build one named workload (optionally at other dims) with its initial fields."""
    if name == "slab2d":  # 64^2 flat liquid slab: rho_bar + (drho/2) tanh((16 - |x - 32|)/2)
        dims = tuple(dims or (64, 64))
        Tr = Tr or TR_2D
        prm = vdw_lattice_params(Tr, D2Q21)
        kap = kappa_for_width(prm, 2.0)
        half = 16.0 * dims[0] / 64.0
        rho = slab_2d(dims[0], dims[1], prm.rho_g, prm.rho_l, half_width=half, centre=dims[0] / 2.0, W=2.0)
        return Case(name, D2Q21, dims, Tr, kap, prm, rho, gamma=gamma)
    if name == "droplet2d":  # 512^2 disc of radius 64, tanh width 4
        dims = tuple(dims or (512, 512))
        Tr = Tr or TR_2D
        prm = vdw_lattice_params(Tr, D2Q21)
        width = 4.0 if dims[0] >= 128 else 2.0
        kap = kappa_for_width(prm, width)
        R = 64.0 * dims[0] / 512.0
        rho = droplet(dims, R, prm.rho_g, prm.rho_l, W=width)
        return Case(name, D2Q21, dims, Tr, kap, prm, rho, gamma=gamma)
    if name == "droplet3d":  # 128^3 sphere of radius 32, tanh width 4
        dims = tuple(dims or (128, 128, 128))
        Tr = Tr or TR_3D
        prm = vdw_lattice_params(Tr, D3Q59)
        width = 4.0 if dims[0] >= 64 else 2.0
        kap = kappa_for_width(prm, width)
        R = 32.0 * dims[0] / 128.0
        rho = droplet(dims, R, prm.rho_g, prm.rho_l, W=width)
        return Case(name, D3Q59, dims, Tr, kap, prm, rho, gamma=gamma)
    if name == "spinodal3d":  # 256^3, rho = 1 +- 1 % (default_rng(0)), u = 0
        dims = tuple(dims or (256, 256, 256))
        Tr = Tr or TR_3D
        prm = vdw_lattice_params(Tr, D3Q59)
        kap = kappa_for_width(prm, 4.0)
        rho = spinodal(dims, seed=0)
        return Case(name, D3Q59, dims, Tr, kap, prm, rho, gamma=gamma)
    raise KeyError(name)


def serving_case(req: Request):
    """The droplet of one serving request: its lattice and side, radius, T/Tc; tanh width 4
    (2 below side 64), kappa matched to that width."""
    d = 2 if req.lattice == D2Q21 else 3
    dims = (req.side,) * d
    prm = vdw_lattice_params(req.Tr, req.lattice)
    width = 4.0 if req.side >= 64 else 2.0
    kap = kappa_for_width(prm, width)
    rho = droplet(dims, req.radius, prm.rho_g, prm.rho_l, W=width)
    return Case("request%d" % req.rid, req.lattice, dims, req.Tr, kap, prm, rho)
