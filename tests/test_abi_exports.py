"""The C-ABI library loads and exports every entry point include/lbm.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1402_2920_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1402_2920_gb300 import build

    build.build()
    return P.load_library()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert set(declared) == set(P.ENTRY_POINTS)
    for name in declared:
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_host_only_entry_points(lib):
    assert P.lbm_velocities(P.LBM_D2Q21).shape == (21, 3)
    c = P.lbm_velocities(P.LBM_D3Q59)
    assert c.shape == (59, 3) and (c.sum(axis=0) == 0).all()
    assert P.lbm_error_string(P.LBM_E_WEIGHTS).startswith("c_s^2")
    assert P.lbm_footprint_bytes(P.LBM_D3Q59, (256, 256, 256), P.LBM_STORE_F32) > 256 ** 3 * 2 * 59 * 4
    assert P.lbm_footprint_bytes(P.LBM_D3Q59, (256, 256, 3), P.LBM_STORE_F32) == 0  # invalid dims


def test_size_limits(lib):
    """lbm_create and lbm_footprint_bytes share one validation (host only): at most 2^31 - 1 sites
    (32-bit site offsets in the streaming kernel), ny <= 524280 (the tiled kernels' grid rows),
    at least 4 sites per axis, nz = 1 exactly in 2D."""
    fp = P.lbm_footprint_bytes
    ok = fp(P.LBM_D3Q59, (1024, 1024, 2047), P.LBM_STORE_F32_DEV)  # 2^31 - 2^20 sites
    assert ok > 1024 * 1024 * 2047 * 2 * 58 * 4
    assert fp(P.LBM_D3Q59, (1024, 1024, 2048), P.LBM_STORE_F32_DEV) == 0  # 2^31 sites
    assert fp(P.LBM_D3Q59, (4, 524280, 4), P.LBM_STORE_F32_DEV) > 0
    assert fp(P.LBM_D3Q59, (4, 524281, 4), P.LBM_STORE_F32_DEV) == 0
    assert fp(P.LBM_D3Q59, (4, 4, 4), P.LBM_STORE_F16_LOC) > 0
    assert fp(P.LBM_D3Q59, (4, 4, 3), P.LBM_STORE_F16_LOC) == 0
    assert fp(P.LBM_D2Q21, (4, 4, 1), P.LBM_STORE_F32) > 0
    assert fp(P.LBM_D2Q21, (4, 4, 2), P.LBM_STORE_F32) == 0
    assert fp(P.LBM_D2Q21, (16, 16, 1), 8) == 0  # no such storage
    assert fp(2, (16, 16, 16), P.LBM_STORE_F32) == 0  # no such lattice
    # 16-bit storages need less memory per site than FP32, the local references a little more
    n = (64, 64, 64)
    assert fp(P.LBM_D3Q59, n, P.LBM_STORE_F16_DEV) < fp(P.LBM_D3Q59, n, P.LBM_STORE_F16_LOC) \
        < fp(P.LBM_D3Q59, n, P.LBM_STORE_F32_DEV) < fp(P.LBM_D3Q59, n, P.LBM_STORE_F32_LOC)


def test_no_cpu_fallback_without_gpu(lib):
    try:
        import torch

        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    eos = P.make_eos(P.LBM_EOS_VDW, a=1.7, b=1.0 / 3.0, T=1.5)
    with pytest.raises(P.LbmError) as e:
        P.Sim(P.LBM_D2Q21, (16, 16), eos, P.make_params(kappa=0.05))
    assert e.value.code == P.LBM_E_CUDA


def test_velocity_pairs_are_bases_or_power_of_two_multiples(lib):
    """The collision computes the contractions of a pair of opposite velocities once per base
    pair and scales them for the pairs whose velocity is 2 or 4 times a base velocity: every pair
    must be exactly one of the two."""
    for lat, bases in ((P.LBM_D2Q21, 4), (P.LBM_D3Q59, 13)):
        c = P.lbm_velocities(lat)
        q = len(c)

        def multiple(i, m):
            for j in range(1, q, 2):
                if (c[j] == m * c[i]).all() or (c[j] == -m * c[i]).all():
                    return j
            return 0

        derived = {multiple(j, m) for j in range(1, q, 2) for m in (2, 4)} - {0}
        base = [i for i in range(1, q, 2) if i not in derived]
        assert len(base) == bases
        count = {j: 0 for j in range(1, q, 2)}
        for i in base:
            count[i] += 1
            for m in (2, 4):
                if multiple(i, m):
                    count[multiple(i, m)] += 1
        assert all(v == 1 for v in count.values())
