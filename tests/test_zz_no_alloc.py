"""The allocation-free conservation sums against lbm_stats_get (collected last, so it also
runs after every other test in the session)."""
import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import lib_sim


def test_sizes_beyond_the_scratch_are_rejected():
    # checked on the host before any device work: the pointers are never touched
    max_sites = 4096 * 256 * 64
    with pytest.raises(P.LbmError) as e:
        P.lbm_moment_sums_noalloc(P.LBM_D3Q59, 16, max_sites + 1, 16)
    assert e.value.code == P.LBM_E_INVALID_ARG
    with pytest.raises(P.LbmError) as e:
        P.lbm_moment_sums_noalloc(P.LBM_D3Q59, 16, 0, 16)
    assert e.value.code == P.LBM_E_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("name,dims,storage", [("droplet3d", (24, 20, 22), P.LBM_STORE_F32_DEV),
                                               ("droplet2d", (96, 80), P.LBM_STORE_F64)])
def test_moment_sums_without_allocation_match_stats(name, dims, storage):
    import torch

    case = W.make_case(name, dims=dims)
    rng = np.random.default_rng(5)
    case.u = 0.01 * rng.standard_normal((len(dims),) + case.rho.shape)
    g = lib_sim(case, storage=storage)
    g.init(case.rho, case.u)
    n = case.rho.size
    Q = 59 if case.lattice == P.LBM_D3Q59 else 21
    pops = torch.empty((Q, n), dtype=torch.float64, device="cuda")
    sums = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):  # two consecutive calls, each against the allocating path
        g.step(4)
        st = g.stats()
        P.lbm_populations(g.handle, pops)
        P.lbm_moment_sums_noalloc(case.lattice, pops, n, sums, stream.cuda_stream)
        stream.synchronize()
        s = sums.cpu().numpy()
        assert abs(s[0] - st.mass) <= 1e-12 * st.mass
        for a in range(3):
            assert abs(s[1 + a] - st.mom[a]) <= 1e-12 * st.mass
