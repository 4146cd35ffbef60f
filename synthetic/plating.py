"""Germ-grain initial plated lithium (inputs only).

The paper's Sec. workflow:generation seeds the plated-Li phase of its
half-cell runs with a germ-grain model: germs from a Poisson point process of
intensity lam on the separator-anode interface plane; from each germ a straight
line towards the anode current collector until it meets the anode solid, at
p*; the grain is the part of the solid surface within r_s of p*; the plated
phase is the union of the grains, one voxel thick.

Voxel reading: the line runs along the through-direction t in the germ's voxel
column; p* is the centre of the face through which it enters the first anode
solid voxel.  The labels carry no particle identities, so the grain is every
anode-solid/electrolyte face whose centre lies within r_s of p* (the paper
restricts it to the one particle that contains p*; with overlapping spheres
the union surface near p* is that particle's surface but for the necks).

The result is a mask over (voxel, direction) pairs; the caller maps it to its
own plating-face order and sets the plated amount of those faces.
"""
import math

import numpy as np

from synthetic.geometry import E, G, SplitMix64, _mix_seed

# face directions d: offsets (dt, dy, dz)
DIRS = ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def poisson(rng, mean):
    """A Poisson(mean) variate by inversion of its distribution function, over
    pieces of mean at most 50 (Poisson laws add) so that exp(-mean) stays
    representable."""
    total = 0
    left = float(mean)
    while left > 0.0:
        m = min(left, 50.0)
        left -= m
        u = rng.uniform()
        k, p = 0, math.exp(-m)
        s = p
        while u > s and p > 0.0:
            k += 1
            p *= m / k
            s += p
        total += k
    return total


def germ_grain(lab, h, anode_end, lam=0.01e12, r_s=2.2e-6, seed=0):
    """Plated-face mask (N_t, N_y, N_z, 6) of anode-solid voxels (G) whose face
    in direction DIRS[d] borders electrolyte (E) and lies in a grain.

    lab: label grid [t][y][z]; h: voxel edge [m]; anode_end: the first t-layer
    after the anode slab (the separator-anode interface plane is t = anode_end h,
    the anode collector side is t = 0); lam: germ intensity [1/m^2] (the
    paper's 0.01 per square micrometre); r_s: grain radius [m] (2.2 um).
    Returns (mask, hits): hits are the p* points (t, y, z) in metres."""
    nt, ny, nz = lab.shape
    rng = SplitMix64(_mix_seed(seed, 7))
    n_germs = poisson(rng, lam * (ny * h) * (nz * h))
    hits = []
    for _ in range(n_germs):
        y = rng.uniform() * ny * h
        z = rng.uniform() * nz * h
        iy, iz = min(int(y / h), ny - 1), min(int(z / h), nz - 1)
        for t in range(anode_end - 1, -1, -1):
            if lab[t, iy, iz] == G:
                hits.append(((t + 1) * h, y, z))
                break
    mask = np.zeros((nt, ny, nz, 6), dtype=bool)
    if not hits:
        return mask, np.zeros((0, 3))
    P = np.array(hits)
    tt, yy, zz = np.nonzero(lab == G)
    for d, (dt, dy, dz) in enumerate(DIRS):
        t2, y2, z2 = tt + dt, yy + dy, zz + dz
        ok = (t2 >= 0) & (t2 < nt) & (y2 >= 0) & (y2 < ny) & (z2 >= 0) & (z2 < nz)
        t1, y1, z1 = tt[ok], yy[ok], zz[ok]
        e = lab[t2[ok], y2[ok], z2[ok]] == E
        t1, y1, z1 = t1[e], y1[e], z1[e]
        if t1.size == 0:
            continue
        # face centres, then the faces within r_s of some p*
        ft = (t1 + 0.5 + 0.5 * dt) * h
        fy = (y1 + 0.5 + 0.5 * dy) * h
        fz = (z1 + 0.5 + 0.5 * dz) * h
        sel = np.zeros(t1.size, dtype=bool)
        for pt, py, pz in P:
            sel |= (ft - pt) ** 2 + (fy - py) ** 2 + (fz - pz) ** 2 <= r_s * r_s
        mask[t1[sel], y1[sel], z1[sel], d] = True
    return mask, P
