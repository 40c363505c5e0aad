"""Shared helpers of the GPU tests: build the same case on the CUDA library and the oracle."""
import numpy as np

import paper_1402_2920_gb300 as P
from oracle import oracle as O
from paper_1402_2920_gb300 import workloads as W

ORACLE_TOL = 1e-14


def lib_sim(case, storage=P.LBM_STORE_F64, usolve=P.LBM_USOLVE_NATIVE, tol=0.0, rtol=0.0, warm=1, maxit=0,
            stream=None, omega=1.0, chebyshev=0):
    """The case on the CUDA library; omega = 1 is the plain iteration of the paper, 0 the automatic one."""
    a, b, T = case.eos_abT
    eos = P.make_eos(P.LBM_EOS_VDW, a=a, b=b, T=T)
    prm = P.make_params(gamma=case.gamma, kappa=case.kappa, rho0=case.rho0, storage=storage, usolve_precision=usolve,
                        usolve_tol=tol, usolve_rtol=rtol, usolve_max_iter=maxit, usolve_warm_start=warm,
                        rho_check_min=0.98 * case.eos.rho_g, rho_check_max=1.02 * case.eos.rho_l, usolve_omega=omega,
                        usolve_chebyshev=chebyshev)
    return P.Sim(case.lattice, case.dims, eos, prm, stream)


def oracle_sim(case, tol=ORACLE_TOL, warm=True, maxit=3000):
    a, b, T = case.eos_abT
    ep = O.eos_params(O.EOS_VDW, a=a, b=b, T=T)
    return O.Sim(case.lattice, case.dims, O.EOS_VDW, ep, case.gamma, case.kappa, case.rho0, tol=tol, maxit=maxit,
                 warm=warm)


def perm_to_oracle(lattice):
    """idx with gpu_c[idx[k]] == oracle_c[k]."""
    cg = P.lbm_velocities(lattice)
    co, _ = O.velocities(lattice)
    pos = {tuple(int(x) for x in v): i for i, v in enumerate(cg)}
    idx = np.array([pos[tuple(int(x) for x in v)] for v in co])
    assert sorted(idx.tolist()) == list(range(len(cg)))
    return idx


def rel_linf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def u_err(u, u_ref, cs0):
    """|du|_inf / max(|u_ref|_inf, 1e-3 c_s(rho0)) -- the velocity error measure of the static cases."""
    return float(np.abs(u - u_ref).max() / max(np.abs(u_ref).max(), 1e-3 * np.sqrt(cs0)))
