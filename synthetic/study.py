"""Seeded parameter-study samplers (inputs only)."""
import math

import numpy as np

from .geometry import SplitMix64


def sample_rom_params(n, seed, crate=(0.5, 5.0), i0_scale=(0.5, 2.0), k_pl=(0.1, 10.0)):
    """Per-instance (C-rate, exchange-current scale, plating rate scale).

    C-rate ~ U(crate), i0 scale ~ LogU(i0_scale), k ~ LogU(k_pl).
    Returns an (n, 3) float64 array.
    """
    rng = SplitMix64(seed)
    out = np.empty((n, 3))
    la, lb = math.log(i0_scale[0]), math.log(i0_scale[1])
    ka, kb = math.log(k_pl[0]), math.log(k_pl[1])
    for i in range(n):
        out[i, 0] = crate[0] + (crate[1] - crate[0]) * rng.uniform()
        out[i, 1] = math.exp(la + (lb - la) * rng.uniform())
        out[i, 2] = math.exp(ka + (kb - ka) * rng.uniform())
    return out


def poisson_arrivals(n, rate, seed):
    """Arrival times (s) of a Poisson stream with the given rate (1/s)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = np.empty(n)
    for i in range(n):
        t += -math.log(1.0 - rng.uniform()) / rate
        out[i] = t
    return out
