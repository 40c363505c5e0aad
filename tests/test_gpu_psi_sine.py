"""The paper's own equation of state (App. B, the psi-sine construction) on the CUDA path:
parity with the oracle for a D2Q21 droplet of the worked example (rho1 = 0.5, rho2 = 1,
A = 1.2, c_s^2(rho1) = 0.6), whose equal-area construction gives coexistence at
rho_g = 1.0367 and rho_l = 1.5113."""
import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from oracle import oracle as O
from oracle import thermo
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import perm_to_oracle, rel_linf

pytestmark = pytest.mark.gpu

PRM = dict(rho1=0.5, rho2=1.0, A=1.2, cs2_rho1=0.6)
KAPPA, RHO0 = 0.1, 1.25


def _droplet():
    ep = O.eos_params(O.EOS_PSI_SINE, **PRM)
    rg, rl, _ = thermo.maxwell(lambda r: O.eos_eval(O.EOS_PSI_SINE, ep, r)[0], 0.6, 2.2)
    dims = (48, 40)
    return dims, W.droplet(dims, 12.0, rg, rl, W=2.0), rg, rl, ep


@pytest.mark.parametrize("storage,tol_rho,tol_u", [(P.LBM_STORE_F64, 1e-12, 1e-12), (P.LBM_STORE_F32_DEV, 2e-6, 2e-4)])
def test_psi_sine_droplet_parity(storage, tol_rho, tol_u):
    dims, rho, rg, rl, ep = _droplet()
    o = O.Sim(O.D2Q21, dims, O.EOS_PSI_SINE, ep, 0.0, KAPPA, RHO0, tol=1e-14, maxit=3000)
    o.init(rho)
    assert o.step(12) == 0
    prm = P.make_params(kappa=KAPPA, rho0=RHO0, storage=storage, rho_check_min=0.98 * rg, rho_check_max=1.02 * rl)
    g = P.Sim(P.LBM_D2Q21, dims, P.make_eos(P.LBM_EOS_PSI_SINE, **PRM), prm)
    g.init(rho)
    g.step(12)
    if storage == P.LBM_STORE_F64:
        idx = perm_to_oracle(P.LBM_D2Q21)
        assert rel_linf(g.populations()[idx], o.pops()) < 1e-12
    rho_g, u_g = g.fields()
    rho_o, u_o, st = o.fields()
    assert st == 0
    assert rel_linf(rho_g, rho_o) < tol_rho
    assert np.abs(u_g - u_o).max() < tol_u * max(np.abs(u_o).max(), 1e-3)
    g.close()
