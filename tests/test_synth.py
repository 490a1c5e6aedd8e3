"""The seeded input generator (no GPU): the blocked nearest-seed search of the segment maps
equals a search over every seed, ties included."""
import numpy as np
import pytest

import synth


def _brute(seeds, width, height):
    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    dx = xs[None, :, None] - seeds[None, None, :, 0]
    dy = ys[:, None, None] - seeds[None, None, :, 1]
    return np.argmin(dx * dx + dy * dy, axis=2).astype(np.int32)


@pytest.mark.parametrize("w,h,k,seed", [(1, 1, 1, 0), (33, 17, 3, 1), (200, 120, 7, 2), (130, 97, 64, 3),
                                        (640, 64, 128, 4)])
def test_voronoi_matches_brute_force(w, h, k, seed):
    rng = np.random.default_rng(seed)
    seeds = np.stack([rng.uniform(0, w, k), rng.uniform(0, h, k)], axis=1)
    assert np.array_equal(synth.voronoi_from_seeds(seeds, w, h), _brute(seeds, w, h))


def test_voronoi_ties_go_to_the_lower_id():
    # duplicated seeds, and seeds placed symmetrically about pixel centres: exact ties
    seeds = np.array([[10.5, 10.5], [30.5, 10.5], [10.5, 10.5], [20.5, 30.5], [20.5, -9.5], [70.0, 40.0],
                      [70.0, 40.0]])
    got = synth.voronoi_from_seeds(seeds, 80, 48)
    assert np.array_equal(got, _brute(seeds, 80, 48))
    assert not (got == 2).any() and not (got == 6).any()   # each duplicate loses to its lower twin
    assert got[10, 20] == 0                                  # equidistant from seeds 0 and 1
