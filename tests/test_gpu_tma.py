"""The tensor-copy (TMA) form of the u-solve sweep against the per-thread-copy form and the oracle.

The default sweep of a 3D lattice loads the planes of u and rho - rho0 of its interior tiles with
tensor copies tracked by mbarriers (tiles on the periodic seams still copy per thread);
LBM_SWEEP_COPY=cp_async at lbm_create selects per-thread copies for every tile.  Both forms load the same values into the same shared-memory ring, so the results
are bitwise equal; the lattice is large enough in x and y to have interior tiles (x tiles start
every 32 sites, y tiles every 8, and a box reaches 4 sites beyond its tile).
"""
import os

import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import lib_sim, oracle_sim, perm_to_oracle, rel_linf

pytestmark = pytest.mark.gpu


def _sim(case, storage, tma, **kw):
    old = os.environ.get("LBM_SWEEP_COPY")
    os.environ["LBM_SWEEP_COPY"] = "tma" if tma else "cp_async"
    try:
        return lib_sim(case, storage=storage, **kw)
    finally:
        if old is None:
            del os.environ["LBM_SWEEP_COPY"]
        else:
            os.environ["LBM_SWEEP_COPY"] = old


@pytest.mark.parametrize("storage,kw", [(P.LBM_STORE_F64, {}), (P.LBM_STORE_F32_DEV, dict(omega=0.0, chebyshev=1))])
def test_tma_sweep_is_bitwise_the_per_thread_sweep(storage, kw):
    case = W.make_case("droplet3d", dims=(100, 36, 40))
    a = _sim(case, storage, True, **kw)
    b = _sim(case, storage, False, **kw)
    for g in (a, b):
        g.init(case.rho)
        g.step(4)
    assert a.stats().usolve_sweeps_total == b.stats().usolve_sweeps_total
    # the tensor copies did run (interior tiles exist here), and the other form used none
    assert a.stats().usolve_tensor_copies == 1
    assert b.stats().usolve_tensor_copies == 0
    assert np.array_equal(a.populations(), b.populations())
    if storage == P.LBM_STORE_F64:
        o = oracle_sim(case)
        o.init(case.rho)
        assert o.step(4) == 0
        idx = perm_to_oracle(case.lattice)
        assert rel_linf(a.populations()[idx], o.pops()) < 1e-12
