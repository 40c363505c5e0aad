"""The continuous-batching serving loop: results equal the same simulations run alone,
admission respects the memory budget, and requests that can never fit are refused."""
import numpy as np
import pytest

import paper_1402_2920_gb300 as P
from paper_1402_2920_gb300 import serving as S
from paper_1402_2920_gb300 import workloads as W


def _mixed_requests():
    """Six small droplets of both lattices, arriving while others run."""
    spec = [(W.D2Q21, 64, 0.00, 40), (W.D3Q59, 32, 0.00, 24), (W.D2Q21, 96, 0.02, 30),
            (W.D3Q59, 48, 0.05, 16), (W.D2Q21, 64, 0.08, 50), (W.D3Q59, 32, 0.10, 20)]
    rng = np.random.default_rng(11)
    out = []
    for k, (lat, side, t, steps) in enumerate(spec):
        lo, hi = W.SERVING_TR[lat]
        out.append(W.Request(k, t, lat, side, rng.uniform(0.15, 0.35) * side, rng.uniform(lo, hi), steps))
    return out


def test_invalid_serving_arguments_are_rejected():
    # host-side checks, before any device work
    with pytest.raises(P.LbmError) as e:
        P.lbm_serve([], max_active=0)
    assert e.value.code == P.LBM_E_INVALID_ARG
    assert P.lbm_serve([], max_active=2) == []


@pytest.mark.gpu
@pytest.mark.parametrize("batched", [1, 0])
def test_each_result_is_the_same_alone_and_in_the_mix(batched):
    """batched = 1: the resident simulations of each lattice step together in one persistent
    launch per stage; 0: one stream per simulation.  Either way bitwise the lone result."""
    reqs = _mixed_requests()
    dicts = S.request_dicts(reqs, keep_rho=True)
    res = P.lbm_serve(dicts, max_active=3, chunk_steps=8, batched=batched)
    assert all(r.status == P.LBM_OK and r.steps_done == d["steps"] for r, d in zip(res, dicts))
    # the work overlapped: some request was admitted before another one finished
    spans = sorted((r.admit_s, r.finish_s) for r in res)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))
    for d in dicts:
        g = P.Sim(d["lattice"], d["dims"], d["eos"], d["params"])
        g.init(d["rho_init"])
        g.step(d["steps"])
        rho, _ = g.fields()
        assert np.array_equal(rho.reshape(-1), d["rho_out"])  # bitwise
        g.close()


@pytest.mark.gpu
@pytest.mark.parametrize("batched", [1, 0])
def test_admission_respects_the_memory_budget(batched):
    reqs = _mixed_requests()
    dicts = S.request_dicts(reqs)
    fp = [P.lbm_footprint_bytes(d["lattice"], d["dims"], d["params"].storage) for d in dicts]
    budget = max(fp) + min(fp) // 2
    res = P.lbm_serve(dicts, memory_budget=budget, max_active=4, chunk_steps=8, batched=batched)
    assert all(r.status == P.LBM_OK for r in res)
    for a in range(len(res)):
        for b in range(a + 1, len(res)):
            if fp[a] + fp[b] > budget:  # these two never held memory at the same time
                ra, rb = res[a], res[b]
                assert ra.finish_s <= rb.admit_s or rb.finish_s <= ra.admit_s
    # a budget below one request's footprint refuses that request and serves the rest
    small = sorted(fp)[-2]
    res = P.lbm_serve(dicts, memory_budget=small, max_active=4, chunk_steps=8, batched=batched)
    for r, f in zip(res, fp):
        assert r.status == (P.LBM_OK if f <= small else P.LBM_E_OOM)


@pytest.mark.gpu
def test_batched_serving_of_many_small_simulations():
    """More requests of one lattice than fit in a batch at once, with different step counts, so
    slots idle, retire and refill between chunks; every result bitwise the lone one."""
    rng = np.random.default_rng(5)
    reqs = []
    for k in range(40):
        lat = W.D2Q21 if k % 10 else W.D3Q59
        side = 32 if lat == W.D2Q21 else 16
        lo, hi = W.SERVING_TR[lat]
        reqs.append(W.Request(k, 0.001 * k, lat, side, 0.25 * side, rng.uniform(lo, hi), int(rng.integers(1, 30))))
    dicts = S.request_dicts(reqs, keep_rho=True)
    res = P.lbm_serve(dicts, max_active=40, chunk_steps=7, batched=1)  # 36 of D2Q21: more than a batch holds
    assert all(r.status == P.LBM_OK and r.steps_done == d["steps"] for r, d in zip(res, dicts))
    for d in dicts[::3] + dicts[1:6]:
        g = P.Sim(d["lattice"], d["dims"], d["eos"], d["params"])
        g.init(d["rho_init"])
        g.step(d["steps"])
        rho, _ = g.fields()
        assert np.array_equal(rho.reshape(-1), d["rho_out"])
        g.close()
