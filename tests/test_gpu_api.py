"""Behaviour of the C ABI on the GPU: conservation, checkpoints, batching, errors,
and properties of the full-size launch that hold at any size."""
import os

import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import lib_sim

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,tol", [(P.LBM_STORE_F64, 1e-13), (P.LBM_STORE_F32, 1e-12),
                                         (P.LBM_STORE_F32_DEV, 1e-12), (P.LBM_STORE_F16_DEV, 1e-12),
                                         (P.LBM_STORE_F32_LOC, 1e-12), (P.LBM_STORE_F16_LOC, 1e-12)])
def test_mass_and_momentum_conserved(storage, tol):
    case = W.make_case("droplet3d", dims=(24, 20, 22))
    rng = np.random.default_rng(3)
    case.u = 0.01 * rng.standard_normal((3,) + case.rho.shape)
    g = lib_sim(case, storage=storage)
    g.init(case.rho, case.u)
    s0 = g.stats()
    g.step(20)
    s1 = g.stats()
    assert s1.status == 0 and s1.steps == 20
    assert abs(s1.mass - s0.mass) < tol * s0.mass  # exact mass bookkeeping in every storage
    mom_tol = 1e-13 if storage == P.LBM_STORE_F64 else 2e-6
    for a in range(3):
        assert abs(s1.mom[a] - s0.mom[a]) < mom_tol * s0.mass
    assert s1.usolve_iters_last >= 1


@pytest.mark.parametrize("storage,warm", [(P.LBM_STORE_F32, 1), (P.LBM_STORE_F16_LOC, 1), (P.LBM_STORE_F32_DEV, 2)])
def test_checkpoint_resume_is_bitwise(tmp_path, storage, warm):
    # warm = 2 keeps two steps' j~ (the extrapolated start) and which buffer is the newer one
    case = W.make_case("droplet2d", dims=(48, 40))
    a = lib_sim(case, storage=storage, warm=warm, omega=0.0, chebyshev=1)
    a.init(case.rho)
    a.step(7)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.step(9)
    b = lib_sim(case, storage=storage, warm=warm, omega=0.0, chebyshev=1)
    b.load(path)
    b.step(9)
    assert np.array_equal(a.populations(), b.populations())
    assert b.stats().steps == 16
    # a checkpoint of the other warm-start layout is refused
    c = lib_sim(case, storage=storage, warm=3 - warm, omega=0.0, chebyshev=1)
    with pytest.raises(P.LbmError) as e:
        c.load(path)
    assert e.value.code == P.LBM_E_IO


@pytest.mark.parametrize("warm", [1, 2])
def test_step_split_is_bitwise(warm):
    case = W.make_case("droplet3d", dims=(16, 18, 20))
    a = lib_sim(case, storage=P.LBM_STORE_F32, warm=warm)
    b = lib_sim(case, storage=P.LBM_STORE_F32, warm=warm)
    a.init(case.rho)
    b.init(case.rho)
    a.step(5)
    for _ in range(5):
        b.step(1)
    assert np.array_equal(a.populations(), b.populations())
    # lbm_fields does not disturb the warm start of the run
    a.fields()
    a.step(3)
    b.step(3)
    assert np.array_equal(a.populations(), b.populations())


def test_batch_equals_alone():
    import torch

    cases = [W.make_case("droplet2d", dims=(64, 64)), W.make_case("droplet3d", dims=(20, 20, 20)),
             W.make_case("slab2d", dims=(32, 48))]
    streams = [torch.cuda.Stream() for _ in cases]
    mixed = [lib_sim(c, storage=P.LBM_STORE_F32, stream=s.cuda_stream) for c, s in zip(cases, streams)]
    alone = [lib_sim(c, storage=P.LBM_STORE_F32) for c in cases]
    for m, a, c in zip(mixed, alone, cases):
        m.init(c.rho)
        a.init(c.rho)
    P.lbm_step_batch([m.handle for m in mixed], [12, 7, 15])
    for a, n in zip(alone, [12, 7, 15]):
        a.step(n)
    for m, a in zip(mixed, alone):
        m.sync()
        assert np.array_equal(m.populations(), a.populations())


def test_invalid_arguments_are_rejected():
    case = W.make_case("droplet2d", dims=(32, 32))
    a, b, T = case.eos_abT
    eos = P.make_eos(P.LBM_EOS_VDW, a=a, b=b, T=T)
    with pytest.raises(P.LbmError) as e:
        P.Sim(P.LBM_D2Q21, (3, 32), eos, P.make_params(kappa=0.1))
    assert e.value.code == P.LBM_E_INVALID_ARG
    with pytest.raises(P.LbmError) as e:
        P.Sim(P.LBM_D2Q21, (32, 32), eos, P.make_params(gamma=1.0))
    assert e.value.code == P.LBM_E_INVALID_ARG
    with pytest.raises(P.LbmError) as e:
        P.Sim(P.LBM_D3Q59, (32, 32, 1), eos, P.make_params())
    assert e.value.code == P.LBM_E_INVALID_ARG
    for warm in (-1, 3):
        with pytest.raises(P.LbmError) as e:
            P.Sim(P.LBM_D2Q21, (32, 32), eos, P.make_params(kappa=0.1, usolve_warm_start=warm))
        assert e.value.code == P.LBM_E_INVALID_ARG
    # the create-time EOS check: a density range where p/rho leaves the window
    with pytest.raises(P.LbmError) as e:
        P.Sim(P.LBM_D2Q21, (32, 32), eos, P.make_params(rho_check_min=0.2, rho_check_max=2.5))
    assert e.value.code in (P.LBM_E_WEIGHTS, P.LBM_E_BULKVISC)


def test_window_violation_is_reported_not_trapped():
    case = W.make_case("droplet2d", dims=(32, 32))
    g = lib_sim(case, storage=P.LBM_STORE_F32)
    rho = case.rho.copy()
    rho[5, 5] = 2.6  # c_s^2 = p/rho far outside the window at one site
    g.init(rho)
    g.step(1)
    assert P.lbm_sync(g.handle) == P.LBM_E_WEIGHTS
    assert P.lbm_sync(g.handle) == P.LBM_OK  # reported once


def test_usolve_cap_is_reported():
    case = W.make_case("droplet2d", dims=(32, 32))
    g = lib_sim(case, storage=P.LBM_STORE_F64, tol=1e-30, maxit=3)
    g.init(case.rho)
    g.step(1)
    assert P.lbm_sync(g.handle) == P.LBM_E_USOLVE_DIVERGED
    st = g.stats()
    assert st.usolve_iters_last == 3


@pytest.mark.parametrize("storage", [P.LBM_STORE_F32_DEV, P.LBM_STORE_F16_DEV, P.LBM_STORE_F16_LOC])
def test_full_size_spinodal_properties(storage):
    """256^3 D3Q59 spinodal as the benchmark launches it (Chebyshev sweeps, extrapolated start,
    tensor-copy plane loads): mass and momentum conservation, a finite state, a converged u-solve,
    and bitwise covariance under a periodic shift."""
    import torch

    case = W.make_case("spinodal3d")
    kw = dict(omega=0.0, chebyshev=1, warm=2)
    g = lib_sim(case, storage=storage, **kw)
    g.init(case.rho)
    s0 = g.stats()
    g.step(3)
    s1 = g.stats()
    assert s1.status == 0
    assert s1.usolve_tensor_copies == 1
    assert abs(s1.mass - s0.mass) < 1e-12 * s0.mass
    assert max(abs(v) for v in s1.mom) < 1e-5 * s0.mass
    n = torch.empty((59, case.rho.size), dtype=torch.float64, device="cuda")
    P.lbm_populations(g.handle, n)
    assert bool(torch.isfinite(n).all())
    shift = (5, 11, 3)  # (z, y, x) roll, not a multiple of any block
    h = lib_sim(case, storage=storage, **kw)
    h.init(np.ascontiguousarray(np.roll(case.rho, shift, axis=(0, 1, 2))))
    h.step(3)
    m = torch.empty_like(n)
    P.lbm_populations(h.handle, m)
    n4 = n.view(59, 256, 256, 256)
    m4 = m.view(59, 256, 256, 256)
    assert torch.equal(torch.roll(n4, shifts=shift, dims=(1, 2, 3)), m4)


@pytest.mark.parametrize("storage,tol", [(P.LBM_STORE_F32_DEV, 1e-7), (P.LBM_STORE_F16_LOC, 1e-4)])
def test_populations_export_import_roundtrip(storage, tol):
    """lbm_set_populations stores each population relative to the reference the decode adds;
    exporting again returns the same populations up to one rounding of the storage, and the
    run continues from them."""
    case = W.make_case("droplet3d", dims=(16, 20, 24))
    a = lib_sim(case, storage=storage)
    a.init(case.rho)
    a.step(5)
    n = a.populations()
    b = lib_sim(case, storage=storage)
    b.set_populations(n)
    m = b.populations()
    assert np.abs(m - n).max() <= tol * np.abs(n).max()
    assert abs(b.stats().mass - a.stats().mass) < 1e-6 * a.stats().mass
    b.step(5)
    assert b.stats().status == 0


@pytest.mark.parametrize("zb", [5, 13, 40])
def test_slab_depth_does_not_change_results(zb):
    """The tiled kernels' z-slab depth (chosen per lattice at lbm_create; LBM_TILE_Z sets it) only
    regroups the planes among CTAs: the results are bitwise those of the default depth."""
    case = W.make_case("droplet3d", dims=(40, 24, 44))
    kw = dict(storage=P.LBM_STORE_F32_DEV, omega=0.0, chebyshev=1, warm=2)
    old = os.environ.get("LBM_TILE_Z")
    os.environ["LBM_TILE_Z"] = str(zb)
    try:
        a = lib_sim(case, **kw)
    finally:
        if old is None:
            del os.environ["LBM_TILE_Z"]
        else:
            os.environ["LBM_TILE_Z"] = old
    b = lib_sim(case, **kw)
    for g in (a, b):
        g.init(case.rho)
        g.step(6)
    assert a.stats().usolve_sweeps_total == b.stats().usolve_sweeps_total
    assert np.array_equal(a.populations(), b.populations())
