"""Pins of the oracle's velocity sets and weights (Sec. III, Tables I and II).

Nothing here re-types the weight polynomials: the tests check what the paper
fixes about them -- shell structure, the sixth-rank isotropy conditions with
Gaussian moments, the printed c_s^2 window, and the 3D -> 2D projection.
"""
import itertools
import os

import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
LATS = {"D2Q21": O.D2Q21, "D3Q59": O.D3Q59}


def _read_gold(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                rows.append(ln.split())
    return rows


def _pairings(idx):
    """All ways to split the index list into unordered pairs."""
    if not idx:
        yield []
        return
    a = idx[0]
    for k in range(1, len(idx)):
        rest = idx[1:k] + idx[k + 1:]
        for p in _pairings(rest):
            yield [(a, idx[k])] + p


def _iso(d, rank):
    """Isotropic tensor sum over all pairings of products of Kronecker deltas."""
    T = np.zeros((d,) * rank)
    for ix in itertools.product(range(d), repeat=rank):
        T[ix] = sum(all(ix[a] == ix[b] for a, b in p) for p in _pairings(list(range(rank))))
    return T


def _moment(c, w, rank):
    d = c.shape[1]
    M = np.zeros((d,) * rank)
    for ix in itertools.product(range(d), repeat=rank):
        M[ix] = np.sum(w * np.prod([c[:, a] for a in ix], axis=0))
    return M


def test_shell_structure_matches_tables():
    for lat_name, b, *rep in _read_gold("table_shells.txt"):
        lat = LATS[lat_name]
        c, sh = O.velocities(lat)
        d = 3 if lat == O.D3Q59 else 2
        shell_ids = sorted(set(sh.tolist()))
        sizes = [int((sh == s).sum()) for s in shell_ids]
        reps = [tuple(sorted(np.abs(c[sh == s][0, :d]).tolist(), reverse=True)) for s in shell_ids]
        want = tuple(int(v) for v in rep[:d])
        assert want in reps, (lat_name, want)
        assert sizes[reps.index(want)] == int(b)
    for lat, q in ((O.D2Q21, 21), (O.D3Q59, 59)):
        c, _ = O.velocities(lat)
        assert c.shape[0] == q
        assert len({tuple(v) for v in c}) == q  # distinct
        # every velocity has its opposite (reflection symmetry of the lattice)
        s = {tuple(v) for v in c}
        assert all(tuple(-v) in s for v in c)


@pytest.mark.parametrize("lat", [O.D2Q21, O.D3Q59])
@pytest.mark.parametrize("cs2", [0.40, 0.55, 0.70, 1.0, 1.15])
def test_sixth_rank_isotropy(lat, cs2):
    """Sum w = 1; 2nd, 4th, 6th moments = c_s^2 delta, c_s^4 (dd+perm), c_s^6 (ddd+perm)."""
    c, _ = O.velocities(lat)
    d = 3 if lat == O.D3Q59 else 2
    c = c[:, :d].astype(float)
    w = O.weights(lat, cs2)
    assert abs(w.sum() - 1.0) < 1e-14
    for rank, power in ((2, 1), (4, 2), (6, 3)):
        M = _moment(c, w, rank)
        np.testing.assert_allclose(M, cs2 ** power * _iso(d, rank), atol=1e-13)
    for rank in (1, 3, 5):
        assert np.abs(_moment(c, w, rank)).max() < 1e-14


def test_printed_window_is_reproduced():
    """The positivity window printed in Sec. III / App. B is where min_i w_i > 0."""
    for lat_name, lo, hi in _read_gold("cs2_window.txt"):
        lat = LATS[lat_name]
        nshell = 8 if lat == O.D3Q59 else 6
        lo, hi = float(lo), float(hi)
        wmin = lambda s: min(O.weight_shell(lat, k, s) for k in range(nshell))
        mid = 0.5 * (lo + hi)
        assert wmin(mid) > 0.0
        assert wmin(lo * 0.99) < 0.0 and wmin(hi * 1.01) < 0.0
        # locate both edges to the printed 7 decimals
        edge_lo = brentq(wmin, lo * 0.9, mid, xtol=1e-13)
        edge_hi = brentq(wmin, mid, hi * 1.1, xtol=1e-13)
        assert abs(edge_lo - lo) < 5e-8, (lat_name, edge_lo)
        assert abs(edge_hi - hi) < 5e-8, (lat_name, edge_hi)


@pytest.mark.parametrize("cs2", [0.4, 0.6, 0.9, 1.1])
def test_d3q59_projects_onto_d2q21(cs2):
    """Sec. III: D2Q21 is the projection of D3Q59; summing the 3D weights over c_z gives the 2D ones."""
    c3, _ = O.velocities(O.D3Q59)
    w3 = O.weights(O.D3Q59, cs2)
    c2, _ = O.velocities(O.D2Q21)
    w2 = O.weights(O.D2Q21, cs2)
    proj = {}
    for v, w in zip(c3, w3):
        key = (int(v[0]), int(v[1]))
        proj[key] = proj.get(key, 0.0) + w
    want = {(int(v[0]), int(v[1])): w for v, w in zip(c2, w2)}
    assert set(k for k, v in proj.items() if abs(v) > 1e-15) == set(want)
    for k, v in want.items():
        assert abs(proj[k] - v) < 1e-14


def test_table_one_printed_w0_is_not_normalised():
    """Documents the reading of Table I: the printed 3D w0 breaks sum_i w_i = 1, the oracle's does not."""
    s = 0.4
    printed_w0 = 1 - 2351 / 720 * s + 1081 / 192 * s ** 2 - 363 / 192 * s ** 3
    w = O.weights(O.D3Q59, s)
    others = w[1:].sum()
    assert abs(printed_w0 + others - 1.0) > 0.1
    assert abs(w[0] + others - 1.0) < 1e-15
