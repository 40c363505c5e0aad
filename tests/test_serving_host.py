"""Host logic of the serving workload that runs without a GPU: the seeded request stream, the
request records handed to lbm_serve, and the latency statistics taken from its results."""
import numpy as np

import paper_1402_2920_gb300 as P
from paper_1402_2920_gb300 import serving
from paper_1402_2920_gb300 import workloads as W


def test_request_stream_is_seeded_and_in_range():
    a = W.serving_requests(n=256, seed=1, rate=2.0)
    b = W.serving_requests(n=256, seed=1, rate=2.0)
    assert a == b
    assert [r.rid for r in a] == list(range(256))
    t = np.array([r.arrival for r in a])
    assert (np.diff(t) > 0).all()
    # Poisson arrivals at rate 2: mean inter-arrival 0.5 (256 draws, 4 standard errors)
    assert abs(np.diff(np.concatenate([[0.0], t])).mean() - 0.5) < 4 * 0.5 / 16
    for r in a:
        lo, hi = W.SERVING_TR[r.lattice]
        assert lo <= r.Tr <= hi and 500 <= r.steps <= 5000
        assert 0.15 * r.side <= r.radius <= 0.35 * r.side
        if r.lattice == P.LBM_D2Q21:
            assert r.side % 32 == 0 and 64 <= r.side <= 512
        else:
            assert r.side % 16 == 0 and 32 <= r.side <= 128
    assert {r.lattice for r in a} == {P.LBM_D2Q21, P.LBM_D3Q59}


def test_request_dicts():
    reqs = W.serving_requests(n=3, seed=1, rate=1.0)
    d = serving.request_dicts(reqs, time_scale=0.25, keep_rho=True)
    for r, q in zip(reqs, d):
        n = r.side ** (2 if r.lattice == P.LBM_D2Q21 else 3)
        assert q["lattice"] == r.lattice and q["steps"] == r.steps and q["sites"] == n
        assert q["arrival_s"] == r.arrival * 0.25
        assert q["rho_init"].shape == (n,) and q["rho_out"].shape == (n,)
        assert q["rho_init"].flags["C_CONTIGUOUS"]


class _Res:
    def __init__(self, status, finish_s):
        self.status, self.finish_s = status, finish_s


def test_latency_stats():
    dicts = [{"arrival_s": float(k), "sites": 100, "steps": 10} for k in range(100)]
    # request k finishes k + 1 + k/100 seconds after t = 0, i.e. 1 + k/100 after its arrival;
    # the last one fails and counts in neither the latencies nor the served work
    res = [_Res(P.LBM_OK, k + 1.0 + k / 100.0) for k in range(99)] + [_Res(P.LBM_E_OOM, 200.0)]
    st = serving.latency_stats(res, dicts)
    lat = 1.0 + np.arange(99) / 100.0
    assert st["requests"] == 100 and st["completed"] == 99
    assert np.isclose(st["p50_s"], np.percentile(lat, 50)) and np.isclose(st["p99_s"], np.percentile(lat, 99))
    assert np.isclose(st["max_s"], lat.max())
    assert st["span_s"] == 200.0 and np.isclose(st["mlups"], 99 * 100 * 10 / 200.0 / 1e6)
    empty = serving.latency_stats([], [])
    assert empty["p50_s"] is None and empty["mlups"] is None
