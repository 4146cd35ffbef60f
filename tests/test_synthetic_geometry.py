"""The synthetic microstructures that stand in for the paper's generated
electrodes (inputs only): the seeded generator's distributions, the
Boolean-sphere stopping rule, and the clean-up rules that make a cell usable
(every pore reaches the separator, every particle its collector)."""
import math

import numpy as np
import pytest

import synthetic as syn
from synthetic import geometry as geo


def test_generator_distributions():
    """Uniform doubles in [0, 1) with mean 1/2 and variance 1/12, standard
    normals with mean 0 and variance 1 (20,000 draws, 5-sigma bounds); the same
    seed repeats the sequence and another seed does not."""
    n = 20000
    r = geo.SplitMix64(12345)
    u = np.array([r.uniform() for _ in range(n)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) <= 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) <= 5 * math.sqrt(1 / 180 / n)
    g = np.array([r.normal() for _ in range(n)])
    assert abs(g.mean()) <= 5 / math.sqrt(n) and abs(g.var() - 1.0) <= 5 * math.sqrt(2 / n)
    a, b, c = geo.SplitMix64(7), geo.SplitMix64(7), geo.SplitMix64(8)
    sa = [a.next_u64() for _ in range(5)]
    assert sa == [b.next_u64() for _ in range(5)]
    assert sa != [c.next_u64() for _ in range(5)]
    assert all(0 <= v < 2 ** 64 for v in sa)


@pytest.mark.parametrize("law", [("uniform", 2, 4), ("lognormal_mean", 5.0, 0.3)])
def test_boolean_slab_stops_at_the_target(law):
    """Spheres are added until the solid fraction first reaches 1 - porosity:
    the fraction reached is at least the target and exceeds it by less than
    one sphere's volume."""
    nt, ny, nz, eps = 20, 24, 24, 0.35
    solid, nsph, frac = geo.boolean_sphere_slab(nt, ny, nz, eps, law, seed=3, stream=1)
    assert frac == np.count_nonzero(solid) / solid.size
    rmax = law[2] if law[0] == "uniform" else law[1] * math.exp(3 * law[2])
    assert 1 - eps <= frac < 1 - eps + 4 / 3 * math.pi * (rmax + 1) ** 3 / solid.size
    assert nsph > 0
    again, _, _ = geo.boolean_sphere_slab(nt, ny, nz, eps, law, seed=3, stream=1)
    assert np.array_equal(solid, again)


def _components(mask):
    from scipy import ndimage
    return ndimage.label(mask, structure=ndimage.generate_binary_structure(3, 1))


def test_full_cell_layout_and_connectivity():
    """CN at t = 0, CP at the end, an all-electrolyte separator; after the
    clean-up every electrolyte region reaches the separator, every anode
    particle cluster touches CN and every cathode cluster CP; electrode
    porosities within 0.05 of the requested ones; seeded."""
    ny = nz = 24
    na, ns, nc = 14, 6, 14
    lab = syn.full_cell(ny, nz, na, ns, nc, 0.35, 0.30, ("uniform", 2, 4), (21, 22))
    assert lab.shape == (na + ns + nc + 2, ny, nz)
    assert np.all(lab[0] == geo.CN) and np.all(lab[-1] == geo.CP)
    sep = slice(1 + na, 1 + na + ns)
    assert np.all(lab[sep] == geo.E)
    assert set(np.unique(lab[1:1 + na])) <= {geo.E, geo.G}
    assert set(np.unique(lab[1 + na + ns:-1])) <= {geo.E, geo.K}
    comp, n = _components(lab == geo.E)
    reach = set(np.unique(comp[sep])) - {0}
    assert reach == set(range(1, n + 1))
    for sol, cc in ((geo.G, geo.CN), (geo.K, geo.CP)):
        comp, n = _components((lab == sol) | (lab == cc))
        with_cc = set(np.unique(comp[lab == cc])) - {0}
        assert set(np.unique(comp[lab == sol])) - {0} <= with_cc
    assert abs(np.mean(lab[1:1 + na] == geo.E) - 0.35) <= 0.05
    assert abs(np.mean(lab[1 + na + ns:-1] == geo.E) - 0.30) <= 0.05
    again = syn.full_cell(ny, nz, na, ns, nc, 0.35, 0.30, ("uniform", 2, 4), (21, 22))
    assert np.array_equal(lab, again)
    other = syn.full_cell(ny, nz, na, ns, nc, 0.35, 0.30, ("uniform", 2, 4), (23, 22))
    assert not np.array_equal(lab, other)


def test_half_cell_layout():
    """The half cell of the paper's experiment: CN | graphite in electrolyte |
    separator | Li foil | CP, every pore reaching the separator, every graphite
    cluster touching CN, the anode porosity within 0.05 of the request."""
    ny = nz = 20
    na, ns, nf = 12, 4, 2
    lab = syn.half_cell(ny, nz, na, ns, nf, 0.35, ("uniform", 2, 4), 62)
    assert lab.shape == (na + ns + nf + 2, ny, nz)
    assert np.all(lab[0] == geo.CN) and np.all(lab[-1] == geo.CP)
    assert np.all(lab[1 + na:1 + na + ns] == geo.E)
    assert np.all(lab[1 + na + ns:1 + na + ns + nf] == geo.L)
    assert set(np.unique(lab[1:1 + na])) <= {geo.E, geo.G}
    comp, n = _components(lab == geo.E)
    assert set(np.unique(comp[1 + na:1 + na + ns])) - {0} == set(range(1, n + 1))
    comp, n = _components((lab == geo.G) | (lab == geo.CN))
    assert set(np.unique(comp[lab == geo.G])) - {0} <= set(np.unique(comp[lab == geo.CN])) - {0}
    assert abs(np.mean(lab[1:1 + na] == geo.E) - 0.35) <= 0.05
