"""Properties of the seeded input generators that the measurement relies on
(host code only; no arithmetic of the method)."""
import numpy as np

from paper_2602_08670_gb300 import workloads as W


def test_tiled_bumps_are_cell_averages_of_one_field():
    # a 4x block mean of the 128^2 state equals the 32^2 state (both are exact
    # cell means of the same continuous field), and the 96^2 state's mass
    # equals the 32^2 state's
    fine = W.swe_random_bumps_tiled(128, 5, 3, 4)
    coarse = W.swe_random_bumps_tiled(32, 5, 3, 4)
    blk = fine.reshape(3, 3, 32, 4, 32, 4).mean(axis=(3, 5))
    assert np.abs(blk - coarse).max() <= 1e-14
    mid = W.swe_random_bumps_tiled(96, 5, 3, 4)
    assert np.allclose(mid[:, 0].mean(axis=(1, 2)), coarse[:, 0].mean(axis=(1, 2)), rtol=0, atol=1e-14)
    # fluid at rest, depth between 1 and 1 + the largest amplitude sum
    assert np.all(fine[:, 1:] == 0.0) and fine[:, 0].min() >= 1.0


def test_tiled_bumps_member_offsets_and_tiling():
    a = W.swe_random_bumps_tiled(64, 9, 5, 2)
    b = W.swe_random_bumps_tiled(64, 9, 2, 2, first=3)
    assert np.array_equal(a[3:], b)
    # one tile: the mean excess depth is the sum over bumps of A pi w^2
    # (the whole Gaussian integrates over the periodic square)
    one = W.swe_random_bumps_tiled(256, 4, 1, 1)
    spec = W.random_bump_specs(4, 1)[0]
    mass = float(np.sum(spec.amps * np.pi * spec.widths ** 2))
    assert abs(float(one[0, 0].mean() - 1.0) - mass) <= 1e-12
