"""Pins of the oracle's collision operators and of the stability window of the workloads.

Collision (checked at every site of a small droplet with random flow, for three
values of gamma, after the oracle has run S1-S10 and the S11 tensors):
  * Delta^bulk = (gamma - 1)(n - n^eq) conserves mass and changes the momentum
    by (gamma - 1)(j0 - rho u) (Sec. II with the n^eq moments of Sec. III);
  * Delta^int transfers (1 + gamma)/2 h f of momentum and nothing else up to
    the second moment (Sec. VI);
  * Delta^corr has the moments the correction operator is built to carry
    (Sec. VIII): zero mass, (gamma - 1) j~ of momentum, Sigma as second moment
    and Xi as third moment, where Xi is the S11 tensor Xi' without its j~ part
    (Xi' = Xi + (1 - gamma) c_s^2(rho0) (delta j~)_sym);
  * in total the collision conserves mass and transfers h f of momentum
    (Sec. V), which needs the u-solve's u = (j0 + f/2 + j~)/rho.
The Hermite prefactors of Delta^corr (w/(2 c_s^4), w/(6 c_s^6) with the
c_s^2 traces) and of Delta^int are what these moments fix: a wrong power of
c_s^2(rho0) or a dropped trace term changes one of them.

Stability: the workloads run at T/Tc = 0.99 (2D) and 0.998 (3D), not at the
deeper 0.96 and 0.985, because the method's whole update is linearly unstable
in the gas phase at the deeper quenches.  Uniform gas with 1e-7 noise must grow by
orders of magnitude within a few steps at the deeper T/Tc and decay at the
workloads' T/Tc.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1402_2920_gb300 import workloads as W


def _droplet_sim(lat, dims, Tr, gamma, seed):
    prm = W.vdw_lattice_params(Tr, lat)
    kap = W.kappa_for_width(prm, 2.0)
    ep = O.eos_params(O.EOS_VDW, a=prm.a, b=prm.b, T=prm.T)
    s = O.Sim(lat, dims, O.EOS_VDW, ep, gamma, kap, 1.0, tol=1e-15, maxit=3000)
    rho = W.droplet(dims, min(dims) / 4.0, prm.rho_g, prm.rho_l, W=2.0)
    rng = np.random.default_rng(seed)
    u = 0.02 * rng.standard_normal((len(dims),) + rho.shape)
    s.init(rho, u)
    assert s.step(2) == 0  # let the populations carry non-equilibrium parts
    assert s.prepare() == 0
    return s


CASES = [(O.D2Q21, (12, 12), 0.99), (O.D3Q59, (9, 9, 9), 0.998)]


@pytest.mark.parametrize("lat,dims,Tr", CASES)
@pytest.mark.parametrize("gamma", [-0.3, 0.0, 0.2])
def test_collision_moment_identities(lat, dims, Tr, gamma):
    s = _droplet_sim(lat, dims, Tr, gamma, seed=11)
    d = len(dims)
    c, _ = O.velocities(lat)
    c = c[:, :d].astype(np.float64)
    cs0 = s.cs0
    rho = s.field("rho")
    j0 = s.field("j0")[:d]
    u = s.field("u")[:d]
    f = s.field("f")[:d]
    jt = s.field("jt")[:d]
    Sig = s.field("Sigma").reshape(3, 3, -1)[:d, :d]
    Xi = s.field("Xi").reshape(3, 3, 3, -1)[:d, :d, :d]
    assert np.abs(f).max() > 1e-4 and np.abs(jt).max() > 1e-6 and np.abs(Sig).max() > 1e-6
    I = np.eye(d)
    tol = 2e-13
    pops = s.pops()
    for r in range(s.N):
        parts, nstar = s.collision_parts(r)
        bulk, dint, corr = parts
        # Delta^bulk: mass conserved, momentum (gamma - 1)(j0 - rho u)
        assert abs(bulk.sum()) < tol
        np.testing.assert_allclose(bulk @ c, (gamma - 1.0) * (j0[:, r] - rho[r] * u[:, r]), atol=tol)
        # Delta^int: zero mass, (1 + gamma)/2 h f of momentum, no second moment
        assert abs(dint.sum()) < tol
        np.testing.assert_allclose(dint @ c, 0.5 * (1.0 + gamma) * f[:, r], atol=tol)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", dint, c, c), 0.0, atol=tol)
        # Delta^corr: zero mass, (gamma - 1) j~, Sigma, Xi' + (gamma - 1) cs0 (delta j~)_sym
        assert abs(corr.sum()) < tol
        np.testing.assert_allclose(corr @ c, (gamma - 1.0) * jt[:, r], atol=tol)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", corr, c, c), Sig[:, :, r], atol=tol)
        jsym = (np.einsum("ab,c->abc", I, jt[:, r]) + np.einsum("ac,b->abc", I, jt[:, r])
                + np.einsum("bc,a->abc", I, jt[:, r]))
        np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", corr, c, c, c),
                                   Xi[:, :, :, r] + (gamma - 1.0) * cs0 * jsym, atol=tol)
        # the whole collision: mass kept, h f of momentum transferred (Sec. V)
        delta = bulk + dint + corr
        assert abs(delta.sum()) < tol
        np.testing.assert_allclose(delta @ c, f[:, r], atol=tol)
        np.testing.assert_allclose(nstar, pops[:, r] + delta, atol=1e-15)  # n* = n + Delta


def _gas_growth(lat, n, Tr, width, steps):
    """max |rho - mean| after each of `steps` steps of a uniform gas with 1e-7 noise, over its start."""
    prm = W.vdw_lattice_params(Tr, lat)
    kap = W.kappa_for_width(prm, width)
    ep = O.eos_params(O.EOS_VDW, a=prm.a, b=prm.b, T=prm.T)
    dims = (n,) * (3 if lat == O.D3Q59 else 2)
    s = O.Sim(lat, dims, O.EOS_VDW, ep, 0.0, kap, 1.0, tol=1e-14, maxit=3000)
    rng = np.random.default_rng(5)
    rho = prm.rho_g * (1.0 + 1e-7 * rng.uniform(-1.0, 1.0, size=tuple(reversed(dims))))
    s.init(rho)
    a0 = np.abs(rho - rho.mean()).max()
    amp = []
    for _ in range(steps):
        assert s.step(1) == 0
        r, _, _ = s.fields()
        amp.append(np.abs(r - r.mean()).max() / a0)
    return np.array(amp)


def test_d3q59_gas_is_unstable_at_0985_and_stable_at_0998():
    deep = _gas_growth(O.D3Q59, 10, 0.985, 4.0, 6)
    ok = _gas_growth(O.D3Q59, 10, 0.998, 4.0, 6)
    assert deep[-1] > 1e3, deep          # about 9x per step
    assert np.all(np.diff(deep[2:]) > 0)
    assert ok[-1] < 0.5 and np.all(np.diff(ok) < 0), ok


def test_d2q21_gas_is_unstable_at_096_and_stable_at_099():
    deep = _gas_growth(O.D2Q21, 16, 0.96, 4.0, 8)
    ok = _gas_growth(O.D2Q21, 16, 0.99, 4.0, 8)
    assert deep[-1] > 1e3, deep
    assert ok[-1] < 0.5 and np.all(np.diff(ok) < 0), ok
