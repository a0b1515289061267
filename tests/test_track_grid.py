"""The race car's track grid (host code, no GPU): the library's cell lookup and
listed-segment test, run on the host over the grid it builds, agrees with the
oracle's brute-force distance to every segment (Sec. V-C.1: unsafe off the road)
except within float32 rounding of the edge of the road."""
import numpy as np
import pytest

from oracle import safety as osafe
from workloads import data


@pytest.fixture(scope="module")
def lib(repo_root):
    from paper_1906_02318_gb300 import build, mpmi
    build.build()
    return mpmi


def _points(track, w, seed, n_box=60000, n_edge=60000):
    rng = np.random.default_rng(seed)
    lo, hi = track.min(axis=0) - 3 * w, track.max(axis=0) + 3 * w
    box = rng.uniform(lo, hi, (n_box, 2))
    # points on normals of the centre line, concentrated around the road's edges
    i = rng.integers(0, len(track), n_edge)
    a, b = track[i], np.roll(track, -1, axis=0)[i]
    f = rng.uniform(0, 1, n_edge)[:, None]
    c = a + f * (b - a)
    d = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    nrm = np.stack([-d[:, 1], d[:, 0]], axis=1)
    off = rng.choice([-1, 1], n_edge)[:, None] * (w + rng.normal(0, 0.3, n_edge))[:, None]
    return np.vstack([box, c + off * nrm]).astype(np.float32)


@pytest.mark.parametrize("seed,circular,w", [(3, False, 4.0), (3, False, 2.5), (7, False, 4.0),
                                             (5, True, 3.0)])
def test_grid_test_matches_brute_force(lib, seed, circular, w):
    track = data.track_polyline(seed, circular=circular)
    pts = _points(track, w, seed)
    got = lib.debug_track_query(track, w, pts)
    d = osafe.distance_to_polyline(track, pts.astype(np.float64))
    want = d < w
    bad = np.nonzero(got != want)[0]
    assert np.all(np.abs(d[bad] - w) < 1e-3), (len(bad), float(np.abs(d[bad] - w).max()))
    assert len(bad) <= 1e-3 * len(pts)
    assert 0.2 < want.mean() < 0.8          # the sample exercises both sides


def test_grid_query_arguments(lib):
    track = data.track_polyline(3)
    with pytest.raises(lib.MpmiError) as e:
        lib.debug_track_query(track[:2], 4.0, np.zeros((1, 2)))
    assert e.value.code == -1
    with pytest.raises(lib.MpmiError) as e:
        lib.debug_track_query(track, -1.0, np.zeros((1, 2)))
    assert e.value.code == -1
    bad = track.copy()
    bad[5, 0] = np.nan
    with pytest.raises(lib.MpmiError) as e:
        lib.debug_track_query(bad, 4.0, np.zeros((1, 2)))
    assert e.value.code == -3
