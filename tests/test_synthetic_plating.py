"""The germ-grain plated-Li input generator (Sec. workflow:generation): seeded,
and on a flat anode surface its plated fraction is the coverage of a Boolean
disc model, 1 - exp(-lam pi r_s^2) (textbook stochastic geometry: the chance
that a point lies in none of the discs of a Poisson germ process)."""
import math

import numpy as np

import synthetic as syn
from synthetic.plating import DIRS, germ_grain, poisson
from synthetic.geometry import SplitMix64


def _flat_half_cell(n):
    # CN | three anode layers | two separator layers | foil | CP, n x n in y, z
    return syn.slab_1d([syn.CN, syn.G, syn.G, syn.G, syn.E, syn.E, syn.L, syn.CP], n, n)


def test_poisson_mean_and_variance():
    rng = SplitMix64(5)
    for mean in (0.7, 12.0, 180.0):
        x = np.array([poisson(rng, mean) for _ in range(4000)])
        assert abs(x.mean() - mean) <= 5 * math.sqrt(mean / 4000)
        assert abs(x.var() / mean - 1.0) <= 0.15


def test_flat_surface_coverage_is_the_boolean_model_coverage():
    h, lam, r_s = 1e-6, 0.01e12, 2.2e-6
    lab = _flat_half_cell(160)
    expect = 1.0 - math.exp(-lam * math.pi * r_s ** 2)
    fr = []
    for seed in range(4):
        mask, hits = germ_grain(lab, h, anode_end=4, lam=lam, r_s=r_s, seed=seed)
        # germs all hit the last anode layer, at the plane t = 4 h
        assert hits.shape[0] > 0 and np.allclose(hits[:, 0], 4 * h)
        # only the +t faces of the last anode layer border electrolyte
        assert not mask[:, :, :, [0, 2, 3, 4, 5]].any() and not mask[:3, :, :, 1].any()
        fr.append(mask[3, :, :, 1].mean())
    # edge effects (discs clipped within r_s of the border) lower it by ~0.3 %
    assert abs(np.mean(fr) - expect) <= 0.02, (np.mean(fr), expect)


def test_seeded_and_within_the_grains():
    lab = syn.half_cell(24, 24, 10, 4, 2, 0.35, ("uniform", 2, 4), 3)
    h, r_s = 1e-6, 2.2e-6
    m1, p1 = germ_grain(lab, h, anode_end=11, r_s=r_s, seed=9)
    m2, p2 = germ_grain(lab, h, anode_end=11, r_s=r_s, seed=9)
    m3, _ = germ_grain(lab, h, anode_end=11, r_s=r_s, seed=10)
    assert np.array_equal(m1, m2) and np.array_equal(p1, p2)
    assert not np.array_equal(m1, m3)
    t, y, z, d = np.nonzero(m1)
    assert t.size > 0
    assert np.all(lab[t, y, z] == syn.G)
    off = np.array(DIRS)[d]
    assert np.all(lab[t + off[:, 0], y + off[:, 1], z + off[:, 2]] == syn.E)
    fc = np.stack([t + 0.5 + 0.5 * off[:, 0], y + 0.5 + 0.5 * off[:, 1], z + 0.5 + 0.5 * off[:, 2]], axis=1) * h
    dist = np.sqrt(((fc[:, None, :] - p1[None, :, :]) ** 2).sum(axis=2)).min(axis=1)
    assert np.all(dist <= r_s * (1 + 1e-12))
