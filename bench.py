#!/usr/bin/env python3
"""Throughput of the two-phase lattice Boltzmann step on GB300 (MLUPS, % of HBM roofline).

Workload: D3Q59, 256^3 periodic spinodal decomposition (rho = 1 +- 1 % from
default_rng(0), u = 0), van der Waals EOS, FP32 populations.  One bench
"step" is one full time step of the method (moments, force, implicit u-solve
to convergence, derivative fields, collision, streaming) over all sites.
The populations (7.9 GB) are larger than L2, so no flush is needed between
steps.

Native arm (default): one simulation per GPU rank (independent replicas, weak
scaling), timed with CUDA events on the simulation's stream between barriers;
prints one JSON line on rank 0.  --impl reference: the FP64 CPU oracle timed
on a bounded sample of the same workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS and % of HBM roofline (FP32 vs FP16-storage); p50/p99 request latency"
UNIT = "MLUPS"
STORAGES = {"f32": 0, "f32dev": 1, "f16dev": 2, "bf16dev": 3, "f32loc": 5, "f16loc": 6, "bf16loc": 7}
STORAGE_BYTES = {"f32": 4, "f32dev": 4, "f16dev": 2, "bf16dev": 2, "f32loc": 4, "f16loc": 2, "bf16loc": 2}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                if out.returncode == 0 and out.stdout.strip():
                    self.samples.append([v.strip() for v in out.stdout.strip().split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def stop(self):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        smax = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 5 + k and s[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.samples)}


def _algorithmic_bytes(lattice, storage_bytes, read_pops, chebyshev=True):
    """Bytes each kernel must move per site if every input and output is touched once (FP32 fields).

    The rest population of the deviation storages is a float pair (8 bytes) and the density
    carries its float remainder rho_lo (4 bytes), both read once per step by the collision."""
    Q, d = (59, 3) if lattice == 1 else (21, 2)
    naux = 26 if lattice == 1 else 13
    f = 4
    pops = (Q - 1) * storage_bytes + 8
    return {
        # read the populations, write rho - rho0, rho_lo and j0
        "moments": pops + (2 + d) * f,
        # read rho - rho0, j0 and the last two steps' j~ (the extrapolated start); write f, j0' and
        # the starting u
        "force": f + 3 * d * f + 3 * d * f,
        # read u, rho - rho0, j0'; write u (Chebyshev: read and write the update vector too)
        "usolve_sweep": f + 3 * d * f + (2 * d * f if chebyshev else 0),
        # read u, rho - rho0, j0'; write A, B, C, the local Sigma and Xi'
        "derivs": f + 2 * d * f + naux * f,
        # read A, B, C, Sigma_local, Xi', rho - rho0, rho_lo, u, j0', f; write j~ and the populations
        # (gamma != 0 also reads them)
        "collide": naux * f + 2 * f + 4 * d * f + pops * (2 if read_pops else 1),
    }


def _kernel_sources_sha():
    h = hashlib.sha256()
    cdir = os.path.join(ROOT, "paper_1402_2920_gb300", "csrc")
    for name in sorted(os.listdir(cdir)):  # the files that define the kernels
        if not (name.startswith("kernels_") or name in ("lbm_kernels.cuh", "lbm_lattice.h", "lbm_common.h")):
            continue
        with open(os.path.join(cdir, name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    """Per-launch DRAM bytes of the kernel from the committed ncu summary, if it is for these sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
        e = t.get(workload, {}).get(kernel)
        if e and e.get("sources_sha") == _kernel_sources_sha():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest value of x over the ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(world, sites, steps, seconds):
    """Site updates of all replicas (each runs the same workload) per second of the slowest, in millions."""
    return world * sites * steps / seconds / 1e6


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import numpy as np

    from oracle import oracle as O
    from paper_1402_2920_gb300 import workloads as W

    cores = os.cpu_count() or 1
    O.set_num_threads(cores)

    def make(n):
        case = W.make_case("spinodal3d", dims=(n, n, n))
        a, b, T = case.eos_abT
        return case, O.Sim(case.lattice, case.dims, O.EOS_VDW, O.eos_params(O.EOS_VDW, a=a, b=b, T=T), case.gamma,
                           case.kappa, case.rho0, tol=1e-14)

    n = args.ref_side
    if n <= 0:
        # size the per-step sample so that the warm-up and timed steps take about two minutes:
        # one step of a 32^3 cube gives the oracle's rate on these cores
        case, o = make(32)
        o.init(case.rho)
        t0 = time.perf_counter()
        o.step(1)
        rate = 32 ** 3 / max(time.perf_counter() - t0, 1e-6)
        n = int((120.0 * rate / max(args.steps + args.warmup, 1)) ** (1.0 / 3.0))
        n = max(16, min(64, n))
    case, o = make(n)
    o.init(case.rho)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = n ** 3 * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "D3Q59 spinodal, bounded %d^3 sample of the 256^3 case, T/Tc=%g" % (n, case.Tr)},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d^3 periodic spinodal, %d timed steps after %d warm-up" % (n, args.steps,
                                                                                                    args.warmup)},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_baseline(seconds_hint=20.0):
    """The oracle as it stands on the host cores, on a bounded sample of the workload."""
    from oracle import oracle as O
    from paper_1402_2920_gb300 import workloads as W

    n = 64
    case = W.make_case("spinodal3d", dims=(n, n, n))
    a, b, T = case.eos_abT
    cores = os.cpu_count() or 1
    O.set_num_threads(cores)
    o = O.Sim(case.lattice, case.dims, O.EOS_VDW, O.eos_params(O.EOS_VDW, a=a, b=b, T=T), case.gamma, case.kappa,
              case.rho0, tol=1e-14)
    o.init(case.rho)
    o.step(1)
    steps, dt = 0, 0.0
    t0 = time.perf_counter()
    while dt < seconds_hint and steps < 40:
        o.step(1)
        steps += 1
        dt = time.perf_counter() - t0
    return {"value": n ** 3 * steps / dt / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d^3 periodic spinodal of the same recipe, %d steps after 1 warm-up step (FP64)" % (n, steps)}


def run_native(args):
    import numpy as np
    import torch

    import paper_1402_2920_gb300 as P
    from paper_1402_2920_gb300 import workloads as W

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.load_library()

    n = args.side
    case = W.make_case("spinodal3d", dims=(n, n, n))
    storage = STORAGES[args.storage]
    a, b, T = case.eos_abT
    stream = torch.cuda.current_stream()

    def make_sim(st, usolve=P.LBM_USOLVE_NATIVE, warm=2):
        # u-solve sweeps Chebyshev-accelerated for the spectrum bound g over the workload's density
        # range, started from the last two steps' j~ extrapolated
        prm = P.make_params(gamma=case.gamma, kappa=case.kappa, rho0=case.rho0, storage=st,
                            rho_check_min=0.98 * case.eos.rho_g, rho_check_max=1.02 * case.eos.rho_l,
                            usolve_omega=0.0, usolve_chebyshev=1, usolve_precision=usolve, usolve_warm_start=warm)
        return P.Sim(case.lattice, case.dims, P.make_eos(P.LBM_EOS_VDW, a=a, b=b, T=T), prm, stream.cuda_stream)

    def timed(sim, K, Wm):
        rho_d = torch.from_numpy(case.rho.reshape(-1)).to("cuda")
        sim.init(rho_d)
        sim.step(Wm)
        sim.sync()
        s_before = sim.stats()
        sampler = ClockSampler(local)
        sampler.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(K)
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clocks = sampler.stop()
        ms = e0.elapsed_time(e1)
        s_after = sim.stats()
        rc = P.lbm_sync(sim.handle)
        if rc != 0:
            raise RuntimeError("device reported: " + P.lbm_error_string(rc))
        ms = max_over_ranks(ms, dist)
        sweeps = s_after.usolve_sweeps_total - s_before.usolve_sweeps_total
        return ms, clocks, sweeps, s_after

    K, Wm = args.steps, args.warmup
    N = int(np.prod(case.dims))
    sim = make_sim(storage)
    ms, clocks, sweeps, st = timed(sim, K, Wm)
    tensor_copies = st.usolve_tensor_copies  # 1: the sweeps' plane loads ran as tensor copies (TMA)
    mlups = whole_job_mlups(ws, N, K, ms / 1e3)
    launches = 5 * K + 2 * sweeps  # moments, force, u-solve start, derivs, collide; sweep + control

    # dominant kernel: average launch time from CUDA events on the simulation's stream
    prof = P.lbm_profile(sim.handle, reps=5)
    per_step = {k: v * (sweeps / K if k.startswith("usolve") else 1.0) for k, v in prof.items()}
    dom = max(per_step, key=per_step.get)
    sb = STORAGE_BYTES[args.storage]
    alg = _algorithmic_bytes(case.lattice, sb, case.gamma != 0.0)
    peak, peak_kind = _peaks()
    achieved = alg[dom] * N / (prof[dom] / 1e3) / 1e9
    step_gbs = 2 * 59 * sb * N / (ms / K / 1e3) / 1e9  # whole step against 2 Q s bytes per site
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _traffic(dom, "spinodal3d_%d" % n), "kernel": dom,
                "algorithmic_bytes_per_site": alg[dom], "peak_source": peak_kind,
                "step": {"algorithmic_bytes_per_site": 2 * 59 * sb, "achieved": step_gbs,
                         "frac": step_gbs / peak}}

    # the FP16-deviation storage form of the same workload
    # the 16-bit storage forms of the same workload: deviations from w_i(rho0) rho0, and from the
    # sender's local w_i(rho) rho (error against FP64: see the configuration tests)
    # and the FP32 storage with the u-solve's sweeps in FP64 (the fixed point to FP64 tolerance)
    extra = {}
    if args.storage in ("f32", "f32dev") and not args.no_extras:
        del sim
        torch.cuda.empty_cache()
        legs = (("fp16_dev_storage", "f16dev", P.LBM_USOLVE_NATIVE), ("fp16_local_storage", "f16loc", P.LBM_USOLVE_NATIVE),
                ("bf16_dev_storage", "bf16dev", P.LBM_USOLVE_NATIVE), ("bf16_local_storage", "bf16loc", P.LBM_USOLVE_NATIVE),
                ("fp64_usolve", args.storage, P.LBM_USOLVE_F64))
        for key, st, us in legs:
            simx = make_sim(STORAGES[st], us)
            # the FP64 sweeps run at GB300's FP64 rate: that leg times at most 100 steps (the same
            # first steps as the FP32 line, whose window it is compared with)
            kx = K if us == P.LBM_USOLVE_NATIVE else min(K, 100)
            msx, _, sweepsx, _ = timed(simx, kx, Wm)
            extra[key] = {"value": whole_job_mlups(ws, N, kx, msx / 1e3), "unit": UNIT,
                          "speedup_vs_f32": (ms / K) / (msx / kx), "ms_per_step": msx / kx, "steps": kx,
                          "usolve_sweeps_per_step": sweepsx / kx,
                          "storage": st, "usolve": "FP64 sweeps, |dj~| <= 1e-14" if us == P.LBM_USOLVE_F64 else
                          "native-precision sweeps"}
            del simx
            torch.cuda.empty_cache()
        # the u-solve started from the previous step's j~ alone (Sec. IX) instead of the extrapolation
        simx = make_sim(storage, warm=1)
        msx, _, sweepsx, _ = timed(simx, K, Wm)
        extra["warm_start_previous"] = {"value": whole_job_mlups(ws, N, K, msx / 1e3), "unit": UNIT,
                                        "ms_per_step": msx / K, "usolve_sweeps_per_step": sweepsx / K}
        del simx
        torch.cuda.empty_cache()
        # the sweep's per-thread-copy form against its tensor-copy (TMA) form (the default)
        os.environ["LBM_SWEEP_COPY"] = "cp_async"
        try:
            simx = make_sim(storage)
            msx, _, _, _ = timed(simx, K, Wm)
            profx = P.lbm_profile(simx.handle, reps=5)
        finally:
            del os.environ["LBM_SWEEP_COPY"]
        extra["sweep_cp_async"] = {"usolve_sweep_ms": profx["usolve_sweep"], "usolve_sweep_ms_tma": prof["usolve_sweep"],
                                   "ms_per_step": msx / K, "value": whole_job_mlups(ws, N, K, msx / 1e3), "unit": UNIT}
        del simx
        torch.cuda.empty_cache()
        sim = make_sim(storage)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    rho_h = torch.from_numpy(case.rho.reshape(-1).copy()).pin_memory()
    out_rho = torch.empty(N, dtype=torch.float64).pin_memory()
    out_u = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.init(rho_h.numpy())
    sim.step(K)
    P.lbm_fields(sim.handle, out_rho.numpy(), out_u.numpy(), N, 3)
    t1 = time.perf_counter()
    e2e_s = t1 - t0
    e2e_s = max_over_ranks(e2e_s, dist)
    e2e = {"value": whole_job_mlups(ws, N, K, e2e_s), "unit": UNIT, "h2d_bytes_per_step": N * 8 / K,
           "d2h_bytes_per_step": 4 * N * 8 / K,
           "definition": "lbm_init from pinned host rho, %d steps, lbm_fields (S1-S8) back to pinned host" % K}

    # serving: continuous batching of the seeded droplet request stream at 0.8 of the measured
    # batched throughput; latency from arrival to the result in host memory
    serving = None
    if args.serving_requests > 0 and not args.no_extras:
        del sim
        torch.cuda.empty_cache()
        from paper_1402_2920_gb300 import serving as S

        st, _, _ = S.run(n=args.serving_requests, load=0.8, calibrate=min(24, args.serving_requests))
        serving = dict(st, unit="s", workload="%s %d requests of the seed-1 stream (droplets, D2Q21 64^2-512^2 "
                                               "and D3Q59 32^3-128^3, 500-5000 steps, FP32 deviations)"
                       % ("all" if args.serving_requests >= 256 else "first", args.serving_requests))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_extras:
        cpu = _cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": Wm,
                "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.storage in ("f32", "f32dev", "f32loc") else args.storage, "data": "synthetic",
                "config": {"workload": "D3Q59 %d^3 periodic spinodal (rho = 1 +- 1%% of noise, seed 0), vdW T/Tc=%g, "
                                       "kappa=%.5f, gamma=0" % (n, case.Tr, case.kappa),
                           "storage": {"f32": "FP32 populations", "f32dev": "FP32 deviations n_i - w_i(rho0) rho0",
                                       "f16dev": "FP16 deviations", "bf16dev": "BF16 deviations",
                                       "f32loc": "FP32 deviations from the sender's w_i(rho) rho",
                                       "f16loc": "FP16 deviations from the sender's w_i(rho) rho",
                                       "bf16loc": "BF16 deviations from the sender's w_i(rho) rho"}[args.storage],
                           "usolve": "FP32 sweeps, Chebyshev-accelerated for the spectrum [0, g], started from "
                                     "j~_n + 0.75 (j~_n - j~_n-1), stop when |dj~| of the plain iteration and the "
                                     "applied update are <= 5e-9",
                           "parallelism": "replicas x%d" % ws, "l2": "inputs (populations %.1f GB) larger than L2" % (2 * 59 * STORAGE_BYTES[args.storage] * N / 2 / 1e9),
                           "sites": N},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "usolve_sweeps_per_step": sweeps / K,
                "usolve_tensor_copies": tensor_copies,
                "kernel_ms": prof, "serving": serving}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)  # the spinodal benchmark is timed over 1000 steps
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--storage", choices=sorted(STORAGES), default="f32dev")
    # cube side of the oracle's per-step sample (0: sized so the run takes about two minutes)
    ap.add_argument("--ref-side", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true")
    # the benchmark workload is the 256^3 cube; smaller cubes of the same recipe serve profiling
    ap.add_argument("--side", type=int, default=256)
    # requests of the serving stream to replay (256 is the whole stream; 0 skips it)
    ap.add_argument("--serving-requests", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
