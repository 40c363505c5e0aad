"""The benchmark's and the serving loop's exact settings against the oracle, and the FP64
conservation sums against the oracle's population sums.

The benchmark and the serving loop run the 32-bit storages with the u-solve in the storage's
own precision (FP32 sweeps), relaxation chosen per solve (omega = 0) and Chebyshev acceleration
(Sec. IX allows any solver that reaches the same fixed point).  These tests build the library's
simulation with exactly those parameters and compare it with the oracle's plain FP64 iteration,
which stops at max|j~new - j~| <= 1e-14 (S6).

Bounds: as in test_gpu_parity.py, 1e-6 relative L-infinity on rho for the FP32 storages, and the
velocity error on the scale max(|u_ref|, 1e-3 c_s(rho0)).  The spinodal's start is white noise,
whose short waves the u-solve and the streaming work hardest on, so it is the harshest start for
the accelerated sweeps.  FP16 with the sender's local reference rounds only the velocity and
non-equilibrium parts of each population to 2^-11 per step.
"""
import os

import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from oracle import oracle as O
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import lib_sim, oracle_sim, perm_to_oracle, rel_linf, u_err

pytestmark = pytest.mark.gpu


def _bench_sim(case, storage, warm=2):
    """The simulation exactly as bench.py and serving.py build it (warm = 2: the u-solve starts
    from the last two steps' j~ extrapolated)."""
    return lib_sim(case, storage=storage, usolve=P.LBM_USOLVE_NATIVE, omega=0.0, chebyshev=1, warm=warm)


@pytest.fixture(scope="module")
def spinodal48():
    """The spinodal recipe at 48^3 (white noise of +-1 % around rho_c) after 20 oracle steps."""
    case = W.make_case("spinodal3d", dims=(48, 48, 48))
    O.set_num_threads(os.cpu_count() or 1)
    o = oracle_sim(case)
    o.init(case.rho)
    assert o.step(20) == 0
    rho_o, u_o, st = o.fields()
    O.set_num_threads(1)
    assert st == 0
    return case, rho_o, u_o, o.cs0


@pytest.mark.parametrize("storage,tol_rho,tol_u,warm", [(P.LBM_STORE_F32_DEV, 1e-6, 5e-4, 2),
                                                        (P.LBM_STORE_F32_DEV, 1e-6, 5e-4, 1),
                                                        (P.LBM_STORE_F32_LOC, 1e-6, 5e-4, 2),
                                                        (P.LBM_STORE_F16_LOC, 2e-5, 5e-3, 2)])
def test_benchmark_settings_spinodal_parity(spinodal48, storage, tol_rho, tol_u, warm):
    case, rho_o, u_o, cs0 = spinodal48
    g = _bench_sim(case, storage, warm)
    g.init(case.rho)
    g.step(20)
    rho_g, u_g = g.fields()
    st = g.stats()
    assert st.status == 0
    e_rho, e_u = rel_linf(rho_g, rho_o), u_err(u_g, u_o, cs0)
    print("spinodal 48^3 storage %d warm %d: rho %.2e u %.2e sweeps/step %.2f"
          % (storage, warm, e_rho, e_u, st.usolve_sweeps_total / 20.0))
    assert e_rho < tol_rho
    assert e_u < tol_u


@pytest.mark.parametrize("storage", [P.LBM_STORE_F32_DEV, P.LBM_STORE_F16_LOC])
def test_benchmark_settings_across_z_slabs(storage):
    """Several 32-plane z-slabs, the last one ragged, with the benchmark's u-solve."""
    case = W.make_case("droplet3d", dims=(24, 18, 70))
    o = oracle_sim(case)
    o.init(case.rho)
    assert o.step(10) == 0
    rho_o, u_o, _ = o.fields()
    g = _bench_sim(case, storage)
    g.init(case.rho)
    g.step(10)
    rho_g, u_g = g.fields()
    tol_rho, tol_u = (1e-6, 5e-4) if storage == P.LBM_STORE_F32_DEV else (2e-5, 5e-3)
    assert rel_linf(rho_g, rho_o) < tol_rho
    assert u_err(u_g, u_o, o.cs0) < tol_u


@pytest.mark.parametrize("storage,tol", [(P.LBM_STORE_F64, 1e-13), (P.LBM_STORE_F32_DEV, 2e-7),
                                         (P.LBM_STORE_F16_LOC, 2e-5)])
def test_conservation_sums_match_the_oracle(storage, tol):
    """lbm_stats_get's FP64 sums of rho and sum_i n_i c_i against the oracle's sums of its own
    populations on the same state (Sec. VI: mass and total momentum are conserved, so both sides
    must keep their initial values; the flow makes the momentum non-zero)."""
    case = W.make_case("droplet3d", dims=(20, 22, 19))
    rng = np.random.default_rng(4)
    case.u = 0.01 * rng.standard_normal((3,) + case.rho.shape) + np.array([0.01, -0.005, 0.002])[:, None, None, None]
    o = oracle_sim(case)
    o.init(case.rho, case.u)
    g = lib_sim(case, storage=storage)
    g.init(case.rho, case.u)
    c, _ = O.velocities(case.lattice)
    for steps in (0, 6):
        if steps:
            assert o.step(steps) == 0
            g.step(steps)
        n = o.pops()
        mass_o = n.sum()
        mom_o = n.sum(axis=1) @ c
        st = g.stats()
        assert abs(st.mass - mass_o) < tol * mass_o
        for a in range(3):
            assert abs(st.mom[a] - mom_o[a]) < tol * mass_o
    assert abs(mom_o[0]) > 1e-3 * mass_o  # the momentum is not trivially zero
