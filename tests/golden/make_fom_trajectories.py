"""Write the full-order oracle trajectories that the GPU step-parity tests
compare against (tests/golden/fom_*.npz).  Calls only oracle/ and synthetic/.

* cfg1: the 16x16x48 full cell (anode 20 | separator 8 | cathode 20 voxels +
  one collector layer at each end, h = 1 um), Boolean spheres r ~ U(2, 4)
  voxels at porosity 0.35, seeds (11, 12); constant-current charge at 1C from
  the rest state, 60 implicit Euler steps of dt = 1 s (the paper's 60 s
  protocol, Sec. results).  Stored: the functionals of every step and the
  whole state after steps 1, 30 and 60.
* cell24x24x72: the same generator rules at 1.5 times the size (anode 30 |
  separator 12 | cathode 30), seeds (13, 14), plated lithium seeded on every
  third graphite-electrolyte face (4e-5 mol/m^2), 3 steps of a 2C charge.
  Large enough for a multigrid hierarchy of five levels.  Stored: the
  functionals of every step and every fifth unknown of the final state.

Usage: python tests/golden/make_fom_trajectories.py [cfg1|cell24x24x72 ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402
from oracle.fom import Cell  # noqa: E402

CASES = {
    "cfg1": dict(geom=(16, 16, 20, 8, 20, 0.35, 0.35, ("uniform", 2, 4), (11, 12)), crate=-1.0, steps=60,
                 seed_n=None, keep=(1, 30, 60), stride=1),
    "cell24x24x72": dict(geom=(24, 24, 30, 12, 30, 0.35, 0.35, ("uniform", 2, 4), (13, 14)), crate=-2.0, steps=3,
                         seed_n=4e-5, keep=(3,), stride=5),
}


def labels(name):
    return syn.full_cell(*CASES[name]["geom"])


def initial_state(oc, case):
    u = oc.initial_state()
    if case["seed_n"] is not None:
        u[2 * oc.N::3] = case["seed_n"]
    return u


def run(name):
    case = CASES[name]
    params = syn.load_params()
    oc = Cell(labels(name), 1e-6, params)
    u = initial_state(oc, case)
    I = case["crate"] * oc.i_1c
    keys = ("V_cell", "mean_c_solid", "Li_total", "Li_anode", "Li_plated")
    out = {k: [oc.functionals(u)[k]] for k in keys}
    out.update(newton_its=[0], passes=[0], flips=[0], unresolved_flips=[0])
    states = {}
    t0 = time.time()
    for k in range(1, case["steps"] + 1):
        u, info = oc.step(u, 1.0, I)
        for key in keys:
            out[key].append(info[key])
        for key in ("newton_its", "passes", "flips", "unresolved_flips"):
            out[key].append(info[key])
        if k in case["keep"]:
            states["u_%d" % k] = u[::case["stride"]].copy()
        print("%s step %d V %.12f passes %d flips %d (%.0f s)" % (name, k, info["V_cell"], info["passes"],
                                                                 info["flips"], time.time() - t0), flush=True)
    np.savez_compressed(os.path.join(HERE, "fom_%s.npz" % name), N=oc.N, F=oc.F_pl, i_1c=oc.i_1c,
                        crate=case["crate"], stride=case["stride"], keep=np.array(case["keep"]),
                        **{k: np.array(v) for k, v in out.items()}, **states)


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(CASES):
        run(nm)
