"""Voxel microstructure generators (inputs only).

Boolean-sphere electrodes stand in for the stochastic anode structures of the
paper's Sec. 2.1 (Laguerre tessellation + Gaussian random fields on spheres),
whose fitted parameters are not available.  Each electrode slab is filled with
spheres whose centres are uniform in the slab box and whose radii follow a
given law; spheres are added until the solid fraction first reaches
``1 - porosity``.  Voxel (t, y, z) is solid when its centre lies within a
sphere radius of a sphere centre; spheres are clipped to their slab.
"""
import json
import math
import os

import numpy as np

E, G, K, L, CN, CP = 0, 1, 2, 3, 4, 5

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), written from its
    published definition: a Weyl sequence with increment 0x9E3779B97F4A7C15
    followed by the two xor-shift-multiply finalisation rounds."""

    def __init__(self, seed):
        self.state = int(seed) & _MASK64

    def next_u64(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self):
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def normal(self):
        """Standard normal by the Box-Muller transform (one value per call)."""
        u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)


def _mix_seed(seed, stream):
    return (int(seed) * 0x100000001B3 + int(stream) * 0x9E3779B97F4A7C15) & _MASK64


def boolean_sphere_slab(nt, ny, nz, porosity, radius, seed, stream=0):
    """Boolean-sphere solid indicator for one slab of shape (nt, ny, nz).

    Sphere centres are uniform in the slab box dilated by the largest radius
    (uniform law: rmax; log-normal law: mean * exp(2 sigma_log)), radii follow
    the given law, and spheres are added until the solid fraction inside the
    slab first reaches 1 - porosity.

    radius: ("uniform", rmin, rmax) or ("lognormal_mean", mean, sigma_log),
    in voxel units.  For the log-normal law the mean of r is ``mean``, i.e.
    mu_log = ln(mean) - sigma_log**2 / 2.
    Returns (solid bool array, number of spheres, achieved solid fraction).
    """
    rng = SplitMix64(_mix_seed(seed, stream))
    solid = np.zeros((nt, ny, nz), dtype=bool)
    target = (1.0 - porosity) * solid.size
    count = 0
    nsph = 0
    tc = np.arange(nt) + 0.5
    yc = np.arange(ny) + 0.5
    zc = np.arange(nz) + 0.5
    # germs are drawn in the slab box dilated by a typical maximum radius, so
    # that the solid density does not thin out towards the slab faces (the
    # usual edge correction of a Boolean model observed in a window)
    if radius[0] == "uniform":
        rpad = radius[2]
    elif radius[0] == "lognormal_mean":
        rpad = radius[1] * math.exp(2.0 * radius[2])
    else:
        raise ValueError("unknown radius law %r" % (radius[0],))
    while count < target:
        ct = -rpad + rng.uniform() * (nt + 2 * rpad)
        cy = -rpad + rng.uniform() * (ny + 2 * rpad)
        cz = -rpad + rng.uniform() * (nz + 2 * rpad)
        if radius[0] == "uniform":
            r = radius[1] + (radius[2] - radius[1]) * rng.uniform()
        else:
            mu = math.log(radius[1]) - 0.5 * radius[2] ** 2
            r = math.exp(mu + radius[2] * rng.normal())
        t0, t1 = max(0, int(math.floor(ct - r))), min(nt, int(math.ceil(ct + r)) + 1)
        y0, y1 = max(0, int(math.floor(cy - r))), min(ny, int(math.ceil(cy + r)) + 1)
        z0, z1 = max(0, int(math.floor(cz - r))), min(nz, int(math.ceil(cz + r)) + 1)
        nsph += 1
        if t0 >= t1 or y0 >= y1 or z0 >= z1:
            continue
        d2 = ((tc[t0:t1, None, None] - ct) ** 2 + (yc[None, y0:y1, None] - cy) ** 2
              + (zc[None, None, z0:z1] - cz) ** 2)
        ball = d2 <= r * r
        sub = solid[t0:t1, y0:y1, z0:z1]
        count += int(np.count_nonzero(ball & ~sub))
        sub |= ball
    return solid, nsph, count / solid.size


def _electrode_ranges(lab):
    """t-ranges [lo, hi] of the anode solid (G) and cathode solid (K or L
    foil), and the separator layers strictly between them (None if absent)."""
    nt = lab.shape[0]

    def span(mask):
        t = np.nonzero(mask.any(axis=(1, 2)))[0]
        return (int(t[0]), int(t[-1])) if t.size else None

    ga = span(lab == G)
    kc = span((lab == K) | (lab == L))
    if ga is not None and kc is not None and kc[0] - ga[1] > 1:
        sep = (ga[1] + 1, kc[0] - 1)
    else:
        sep = (nt // 3, max(nt // 3, 2 * nt // 3 - 1))
    return span(lab == G), span(lab == K), sep


def _fill_solid(lab, mask, ga, kc):
    """Turn the voxels of ``mask`` that lie in the t-range of an electrode into
    that electrode's solid; voxels outside both ranges stay electrolyte."""
    t_idx, y_idx, z_idx = np.nonzero(mask)
    fill = np.full(t_idx.shape, E, dtype=lab.dtype)
    if ga is not None:
        fill[(t_idx >= ga[0]) & (t_idx <= ga[1])] = G
    if kc is not None:
        fill[(t_idx >= kc[0]) & (t_idx <= kc[1])] = K
    lab[t_idx, y_idx, z_idx] = fill


def _reaches(comp, n, sep):
    keep = np.zeros(n + 1, bool)
    mid = comp[sep[0]:sep[1] + 1]
    keep[np.unique(mid[mid > 0])] = True
    keep[0] = False
    return keep


def percolating(lab):
    """Keep only the connected parts of a cell, as in a wetted electrode:
    pore regions reached from the separator only through necks thinner than
    three voxels, and electrolyte pockets (6-connected) that do not reach the
    separator at all, become the solid of the electrode they lie in (closed
    pores); solid clusters that do not reach their current collector (anode
    solid with CN, cathode solid with CP) become electrolyte.  Separator
    layers are never filled.  This plays the role of the morphological
    smoothing of the paper's generator (Sec. 2.1).  Returns a new grid."""
    from scipy import ndimage
    lab = lab.copy()
    conn = ndimage.generate_binary_structure(3, 1)
    ga, kc, sep = _electrode_ranges(lab)
    # 0. pores reached only through necks thinner than three voxels: keep the
    #    pore voxels within one voxel of the morphologically opened pore network
    #    that reaches the separator; the rest become the surrounding solid
    pore = lab == E
    # the lateral walls are no-flux mirror planes: pad y and z by one mirrored
    # voxel so that a pore along a wall is not taken for a neck
    padded = np.pad(pore, ((1, 1), (1, 1), (1, 1)), mode="edge")
    padded[0] = False
    padded[-1] = False
    opened = ndimage.binary_opening(padded, structure=conn)[1:-1, 1:-1, 1:-1]
    ocomp, no = ndimage.label(opened, structure=conn)
    if no:
        keep = _reaches(ocomp, no, sep)
        near = ndimage.binary_dilation(keep[ocomp], structure=conn)
        _fill_solid(lab, pore & ~near, ga, kc)
    # 1. closed pores: E components without a voxel in the separator layers
    ecomp, ne = ndimage.label(lab == E, structure=conn)
    if ne:
        keep = _reaches(ecomp, ne, sep)
        _fill_solid(lab, (ecomp > 0) & ~keep[ecomp], ga, kc)
    # 2. floating solid: components of (solid + collector) not containing a collector voxel
    for sol, cc in ((G, CN), (K, CP)):
        comp, nc_ = ndimage.label((lab == sol) | (lab == cc), structure=conn)
        if not nc_:
            continue
        keep = np.zeros(nc_ + 1, bool)
        keep[np.unique(comp[(lab == cc) & (comp > 0)])] = True
        floating = (comp > 0) & ~keep[comp] & (lab == sol)
        lab[floating] = E
    return lab


def full_cell(ny, nz, n_anode, n_sep, n_cathode, porosity_anode, porosity_cathode,
              radius, seeds):
    """Full cell label grid with one CN layer at t=0 and one CP layer at the end.

    Layout along t: CN | anode (G spheres in E) | separator (E) | cathode (K
    spheres in E) | CP.  ``seeds`` = (anode seed, cathode seed).  Closed and
    necked pores and floating particles are removed (``percolating``); the
    sphere-filling targets are corrected twice (half the measured error each
    time) and the pass whose electrode porosities after that cleanup lie
    closest to the requested ones is returned.
    """
    nt = n_anode + n_sep + n_cathode + 2
    a0, c0 = 1, 1 + n_anode + n_sep
    ta, tc = porosity_anode, porosity_cathode
    best = None
    for _ in range(3):
        lab = np.full((nt, ny, nz), E, dtype=np.uint8)
        lab[0] = CN
        lab[-1] = CP
        sa, _, _ = boolean_sphere_slab(n_anode, ny, nz, ta, radius, seeds[0], 1)
        sc, _, _ = boolean_sphere_slab(n_cathode, ny, nz, tc, radius, seeds[1], 2)
        lab[a0:a0 + n_anode][sa] = G
        lab[c0:c0 + n_cathode][sc] = K
        lab = percolating(lab)
        ea = float(np.mean(lab[a0:a0 + n_anode] == E))
        ec = float(np.mean(lab[c0:c0 + n_cathode] == E))
        err = abs(ea - porosity_anode) + abs(ec - porosity_cathode)
        if _collectors_touch(lab) and (best is None or err < best[0]):
            best = (err, lab)
        ta = min(0.9, max(0.05, ta + 0.5 * (porosity_anode - ea)))
        tc = min(0.9, max(0.05, tc + 0.5 * (porosity_cathode - ec)))
    if best is None:
        raise ValueError("no valid cell generated: a collector touches no solid")
    return best[1]


def half_cell(ny, nz, n_anode, n_sep, n_foil, porosity_anode, radius, seed):
    """Half cell: CN | anode (G spheres in E) | separator (E) | Li foil (L) | CP."""
    nt = n_anode + n_sep + n_foil + 2
    ta = porosity_anode
    best = None
    for _ in range(3):
        lab = np.full((nt, ny, nz), E, dtype=np.uint8)
        lab[0] = CN
        lab[-1] = CP
        sa, _, _ = boolean_sphere_slab(n_anode, ny, nz, ta, radius, seed, 1)
        lab[1:1 + n_anode][sa] = G
        lab[1 + n_anode + n_sep:1 + n_anode + n_sep + n_foil] = L
        lab = percolating(lab)
        ea = float(np.mean(lab[1:1 + n_anode] == E))
        err = abs(ea - porosity_anode)
        if _collectors_touch(lab) and (best is None or err < best[0]):
            best = (err, lab)
        ta = min(0.9, max(0.05, ta + 0.5 * (porosity_anode - ea)))
    if best is None:
        raise ValueError("no valid cell generated: a collector touches no solid")
    return best[1]


def _collectors_touch(lab):
    """True when the CN layer touches anode solid and the CP layer touches
    cathode solid or a Li foil layer (the first and last t-layers)."""
    ok_n = bool(np.any(lab[1][lab[0] == CN] == G))
    ok_p = bool(np.any(np.isin(lab[-2][lab[-1] == CP], (K, L))))
    return ok_n and ok_p


def slab_1d(phases, ny=1, nz=1):
    """Label grid made of full layers: ``phases`` lists one label per t-layer."""
    lab = np.empty((len(phases), ny, nz), dtype=np.uint8)
    for t, p in enumerate(phases):
        lab[t] = p
    return lab


def load_params(path=None):
    """Load the parameter table (a JSON file of plain numbers)."""
    if path is None:
        path = os.path.join(os.path.dirname(__file__), "params.json")
    with open(path) as f:
        return json.load(f)
