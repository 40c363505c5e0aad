"""The serving workload over lbm_serve: a seeded stream of droplet requests of mixed lattice
and size, Poisson arrivals at a set fraction of the measured batched throughput, and the
latency of each request from arrival to result."""
import numpy as np

from . import lbm as P
from . import workloads as W


def request_dicts(reqs, storage=P.LBM_STORE_F32_DEV, time_scale=1.0, keep_rho=False):
    """lbm_serve request dicts for workloads.Request objects; arrival times are multiplied
    by time_scale (requests drawn at rate 1 then arrive at rate 1/time_scale)."""
    out = []
    for r in reqs:
        case = W.serving_case(r)
        a, b, T = case.eos_abT
        prm = P.make_params(gamma=case.gamma, kappa=case.kappa, rho0=case.rho0, storage=storage,
                            rho_check_min=0.98 * case.eos.rho_g, rho_check_max=1.02 * case.eos.rho_l,
                            usolve_omega=0.0, usolve_chebyshev=1, usolve_warm_start=2)
        d = {"lattice": case.lattice, "dims": case.dims, "eos": P.make_eos(P.LBM_EOS_VDW, a=a, b=b, T=T),
             "params": prm, "steps": r.steps, "arrival_s": r.arrival * time_scale,
             "rho_init": np.ascontiguousarray(case.rho.reshape(-1)), "sites": int(case.rho.size)}
        if keep_rho:
            d["rho_out"] = np.empty(case.rho.size)
        out.append(d)
    return out


def latency_stats(results, dicts):
    """p50 / p99 / max of arrival-to-result times (s) and the served site updates per second."""
    ok = [k for k, r in enumerate(results) if r.status == P.LBM_OK]
    lat = np.array([results[k].finish_s - dicts[k]["arrival_s"] for k in ok])
    work = sum(dicts[k]["sites"] * dicts[k]["steps"] for k in ok)
    span = max(r.finish_s for r in results) if results else 0.0
    return {"requests": len(results), "completed": len(ok),
            "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
            "max_s": float(lat.max()) if len(lat) else None,
            "mlups": work / span / 1e6 if span > 0 else None, "span_s": span}


def run(n=256, load=0.8, max_active=16, chunk_steps=50, memory_budget=0, calibrate=24, seed=1, batched=0,
        rate=None):
    """The serving workload: calibrate the batched throughput on the first `calibrate`
    requests (all present at t = 0), then replay the first n requests with Poisson arrivals
    at `load` times that throughput (in site updates per second).  batched selects lbm_serve's
    batched launches (1) or one stream per simulation (0); a given `rate` (requests per second)
    replaces the calibrated one, so that two modes can replay the same arrivals."""
    reqs = W.serving_requests(n=n, seed=seed, rate=1.0)
    m = min(calibrate, n)
    cal = request_dicts(reqs[:m], time_scale=0.0)
    res = P.lbm_serve(cal, memory_budget=memory_budget, max_active=max_active, chunk_steps=chunk_steps,
                      batched=batched)
    cal_stats = latency_stats(res, cal)
    thr = cal_stats["mlups"] * 1e6  # site updates per second, all requests resident
    mean_work = np.mean([r.side ** (2 if r.lattice == P.LBM_D2Q21 else 3) * r.steps for r in reqs])
    if rate is None:
        rate = load * thr / mean_work  # requests per second
    dicts = request_dicts(reqs, time_scale=1.0 / rate)
    res = P.lbm_serve(dicts, memory_budget=memory_budget, max_active=max_active, chunk_steps=chunk_steps,
                      batched=batched)
    st = latency_stats(res, dicts)
    st.update({"calibration_mlups": cal_stats["mlups"], "calibration_requests": m, "arrival_rate_per_s": rate,
               "offered_load": load, "max_active": max_active, "chunk_steps": chunk_steps,
               "mode": "batched launches per kernel combination" if batched else "one stream per simulation"})
    return st, res, dicts
