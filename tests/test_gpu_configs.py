"""The named configurations at full size and step count: the error of each storage against
FP64, and the physics each one is meant to show.

The FP64 reference at these sizes is the library's own FP64 path (storage F64).  The oracle
cannot run them in minutes, so the FP64 path is itself compared with the oracle, element by
element, on each full-size state for the steps the oracle finishes in seconds (all host
threads), and on every smaller case in test_gpu_parity.py.  Results are printed and, with
LBM_CONFIG_REPORT=<file>, appended as JSON lines.
"""
import json
import math
import os

import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from oracle import oracle as O
from paper_1402_2920_gb300 import workloads as W
from tests.gpu_util import lib_sim, oracle_sim, perm_to_oracle, rel_linf, u_err

pytestmark = [pytest.mark.gpu, pytest.mark.full]


def _report(**kw):
    print(json.dumps(kw))
    path = os.environ.get("LBM_CONFIG_REPORT")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps(kw) + "\n")


def _run(case, steps, storage):
    g = lib_sim(case, storage=storage)
    g.init(case.rho, case.u)
    g.step(steps)
    rho, u = g.fields()
    st = g.stats()
    g.close()
    return rho, u, st


def _run_marks(case, marks, storage):
    """(rho, u) after each number of steps in marks (increasing)."""
    g = lib_sim(case, storage=storage)
    g.init(case.rho, case.u)
    out, done = {}, 0
    for m in marks:
        g.step(m - done)
        done = m
        out[m] = g.fields()
    g.close()
    return out


def _fp64_vs_oracle(case, steps):
    """FP64 path against the oracle on the full-size state, element by element."""
    O.set_num_threads(os.cpu_count() or 1)
    g = lib_sim(case, storage=P.LBM_STORE_F64)
    o = oracle_sim(case)
    g.init(case.rho, case.u)
    o.init(case.rho, case.u)
    g.step(steps)
    assert o.step(steps) == 0
    idx = perm_to_oracle(case.lattice)
    err = rel_linf(g.populations()[idx], o.pops())
    g.close()
    O.set_num_threads(1)
    return err


def test_config_droplet2d_512_fp32_vs_fp64_5000_steps():
    """D2Q21 512^2 static droplet R = 64, width 4: FP32 deviations against FP64 after 5000 steps,
    the Laplace pressure jump against sigma/R, and the largest spurious velocity."""
    case = W.make_case("droplet2d")
    e_orc = _fp64_vs_oracle(case, 3)
    assert e_orc < 1e-12
    r64_1k, u64_1k, _ = _run(case, 1000, P.LBM_STORE_F64)
    r32_1k, u32_1k, _ = _run(case, 1000, P.LBM_STORE_F32_DEV)
    r64, u64, s64 = _run(case, 5000, P.LBM_STORE_F64)
    r32, u32, s32 = _run(case, 5000, P.LBM_STORE_F32_DEV)
    cs0 = case.eos.T / (1 - case.eos.b) - case.eos.a  # c_s^2(rho0 = 1) of the vdW EOS
    e_rho, e_u = rel_linf(r32, r64), u_err(u32, u64, cs0)
    e_rho_1k, e_u_1k = rel_linf(r32_1k, r64_1k), u_err(u32_1k, u64_1k, cs0)
    # Laplace: Delta p = sigma / R, sigma = kappa drho^2 / (3 W) for a tanh profile of width W
    p = lambda r: r * case.eos.T / (1 - case.eos.b * r) - case.eos.a * r * r
    n = case.dims[0]
    rho_in, rho_out = float(r64[n // 2, n // 2]), float(r64[0, 0])
    drho = case.eos.rho_l - case.eos.rho_g
    sigma = case.kappa * drho ** 2 / (3 * 4.0)
    R = math.sqrt(max(((r64 - rho_out) / (rho_in - rho_out)).sum(), 0.0) / math.pi)  # equivalent radius
    dp, dp_pred = p(rho_in) - p(rho_out), sigma / R
    _report(config="droplet2d 512^2, 5000 steps", fp64_vs_oracle_3_steps=e_orc, fp32dev_rho_rel_linf=e_rho,
            fp32dev_u_err=e_u, fp32dev_rho_rel_linf_1000=e_rho_1k, fp32dev_u_err_1000=e_u_1k, laplace_dp=dp,
            laplace_sigma_over_R=dp_pred, radius=R, max_spurious_u=float(np.abs(u64).max()),
            mass_drift_fp32=abs(s32.mass - s64.mass) / s64.mass)
    # FP32: the collision's arithmetic rounding repeats on a nearly static state, so the error
    # grows about linearly: 5.5e-7 after 1000 steps, 3.4e-6 after 5000
    assert e_rho_1k < 1e-6 and e_rho < 1e-5
    # the velocity is the spurious current (~1e-4); the FP32 rounding of j0 = sum n_i c_i
    # (~3e-7 absolute) sets the floor of e_u on the scale max(|u|, 1e-3 c_s)
    assert e_u < 1e-3
    # Laplace: the diffuse interface adds O(W/R) corrections (W/R = 1/16)
    assert abs(dp / dp_pred - 1) < 0.25


def test_config_droplet3d_128_storages_vs_fp64_2000_steps():
    """D3Q59 128^3 static droplet R = 32: FP32, FP16 and BF16 deviation storage against FP64,
    after 1000 and 2000 steps."""
    case = W.make_case("droplet3d")
    e_orc = _fp64_vs_oracle(case, 1)
    assert e_orc < 1e-12
    marks = (1000, 2000)
    ref = _run_marks(case, marks, P.LBM_STORE_F64)
    cs0 = case.eos.T / (1 - case.eos.b) - case.eos.a
    out = {"config": "droplet3d 128^3, 1000 and 2000 steps", "fp64_vs_oracle_1_step": e_orc,
           "max_spurious_u": float(np.abs(ref[2000][1]).max())}
    # bounds after 2000 steps, about twice the measured error.  16-bit storages: the global
    # reference rounds the deviation from w_i(rho0) rho0, 10-20 % of n_i across the two phases, to
    # 2^-11 (half) or 2^-8 (bfloat16) each step; the sender's local reference rounds only the
    # velocity and non-equilibrium parts.  FP32: the 1e-6 target after 1000 steps holds for
    # the global-reference deviations; after 2000 steps the slow drift of the droplet's mass
    # balance under FP32 arithmetic has roughly doubled it.
    tols = {"fp32dev": (1e-6, 3e-6), "fp16dev": (None, 3e-3), "bf16dev": (None, 1.5e-2), "fp32loc": (None, 4e-6),
            "fp16loc": (None, 1e-5), "bf16loc": (None, 1e-3)}
    storages = {"fp32dev": P.LBM_STORE_F32_DEV, "fp16dev": P.LBM_STORE_F16_DEV, "bf16dev": P.LBM_STORE_BF16_DEV,
                "fp32loc": P.LBM_STORE_F32_LOC, "fp16loc": P.LBM_STORE_F16_LOC, "bf16loc": P.LBM_STORE_BF16_LOC}
    for name, st in storages.items():
        res = _run_marks(case, marks, st)
        for m in marks:
            out["%s_rho_rel_linf_%d" % (name, m)] = rel_linf(res[m][0], ref[m][0])
            out["%s_u_err_%d" % (name, m)] = u_err(res[m][1], ref[m][1], cs0)
    _report(**out)
    for name, (t1k, t2k) in tols.items():
        if t1k is not None:
            assert out[name + "_rho_rel_linf_1000"] < t1k, name
        assert out[name + "_rho_rel_linf_2000"] < t2k, name


def test_config_spinodal3d_256_fp32_vs_fp64_100_steps():
    """D3Q59 256^3 spinodal (the benchmark workload): FP32 deviations against FP64 over 100 steps."""
    case = W.make_case("spinodal3d")
    r64, u64, s64 = _run(case, 100, P.LBM_STORE_F64)
    r32, u32, s32 = _run(case, 100, P.LBM_STORE_F32_DEV)
    e_rho = rel_linf(r32, r64)
    e_u = float(np.abs(u32 - u64).max() / np.abs(u64).max())
    _report(config="spinodal3d 256^3, 100 steps", fp32dev_rho_rel_linf=e_rho, fp32dev_u_rel_linf=e_u,
            u_max=float(np.abs(u64).max()), mass_drift_fp32=abs(s32.mass - s64.mass) / s64.mass)
    assert e_rho < 1e-6
