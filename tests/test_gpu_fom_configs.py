"""Step parity with the FP64 oracle on whole workload cells (GPU).

The expected values are the oracle's own trajectories, written by
tests/golden/make_fom_trajectories.py (which calls only oracle/ and
synthetic/):

* the 16x16x48 full cell of the 60 s, 1C charge protocol, all 60 steps: cell
  potential, mean graphite concentration and lithium inventory after every
  step, and every unknown after steps 1, 30 and 60;
* a 24x24x72 full cell (a five-level multigrid hierarchy) with seeded plated
  lithium, 3 steps of a 2C charge: the functionals of every step and every
  fifth unknown of the final state.

Tolerances: the FP64 path 1e-9 relative (per field in the max-norm, and on
the cell potential), the mixed-precision path 1e-6 on the cell potential and
1e-5 per field; the lithium inventory 1e-12 relative for both (conservation
holds to the Newton tolerance).  The active-set pass counts must match the
oracle's (integer decisions on the same converged states).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


def _golden(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_fom_trajectories",
                                                  os.path.join(GOLDEN, "make_fom_trajectories.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    return mk, dict(np.load(os.path.join(GOLDEN, "fom_%s.npz" % name)))


def _field_errs(a, b, N, F):
    out = {}
    for name, sl in (("c", slice(0, N)), ("phi", slice(N, 2 * N)), ("n", slice(2 * N, 2 * N + F))):
        ref = b[sl]
        scale = np.max(np.abs(ref)) if ref.size else 0.0
        if scale > 0:
            out[name] = float(np.max(np.abs(a[sl] - ref)) / scale)
    return out


def _sampled_errs(u_gpu, sample, stride, N, F):
    """Field errors of every stride-th unknown (the stored sample)."""
    idx = np.arange(0, 2 * N + F, stride)
    a = u_gpu[idx]
    out = {}
    for name, m in (("c", idx < N), ("phi", (idx >= N) & (idx < 2 * N)), ("n", idx >= 2 * N)):
        ref = sample[m]
        scale = np.max(np.abs(ref)) if ref.size else 0.0
        if scale > 0:
            out[name] = float(np.max(np.abs(a[m] - ref)) / scale)
    return out


def _run(params, name, precision):
    B = _gpu()
    mk, gd = _golden(name)
    case = mk.CASES[name]
    lab = mk.labels(name)
    opts = B.default_opts(precision=precision, newton_tol=1e-12 if precision == B.PREC_FP64 else 1e-10,
                          krylov_rtol=1e-6 if precision == B.PREC_FP64 else 1e-4)
    gc = B.Cell(lab, 1e-6, params, opts)
    N, F = int(gd["N"]), int(gd["F"])
    assert gc.N == N and gc.F == F
    assert abs(gc.i_1c - float(gd["i_1c"])) <= 1e-14 * float(gd["i_1c"])
    u = gc.state()
    if case["seed_n"] is not None:
        u[2 * N::3] = case["seed_n"]
        gc.set_state(u)
    I = float(gd["crate"]) * gc.i_1c
    infos, states = [], {}
    for k in range(1, case["steps"] + 1):
        infos.append(gc.step(1.0, I))
        if k in case["keep"]:
            states[k] = gc.state()
    gc.close()
    return gd, case, infos, states, N, F


@pytest.mark.parametrize("precision,tol_v,tol_f", [(0, 1e-9, 1e-9), (1, 1e-6, 1e-5)])
def test_cfg1_sixty_steps_match_oracle(params, precision, tol_v, tol_f):
    """16x16x48 cell, 1C charge, 60 steps of 1 s."""
    gd, case, infos, states, N, F = _run(params, "cfg1", precision)
    for k, info in enumerate(infos, start=1):
        assert abs(info["V_cell"] - gd["V_cell"][k]) <= tol_v * abs(gd["V_cell"][k]), (k, info)
        assert abs(info["mean_c_solid"] - gd["mean_c_solid"][k]) <= tol_f * abs(gd["mean_c_solid"][k]), k
        assert abs(info["Li_total"] - gd["Li_total"][k]) <= 1e-12 * gd["Li_total"][k], k
        assert info["passes"] == gd["passes"][k] and info["unresolved_flips"] == gd["unresolved_flips"][k], k
    for k, u in states.items():
        errs = _field_errs(u, gd["u_%d" % k], N, F)
        assert all(v <= tol_f for v in errs.values()), (k, errs)


@pytest.mark.parametrize("precision,tol_v,tol_f", [(0, 1e-9, 1e-9), (1, 1e-6, 1e-5)])
def test_cell24x24x72_with_plating_matches_oracle(params, precision, tol_v, tol_f):
    """24x24x72 cell (a five-level multigrid hierarchy), seeded plated lithium, 2C."""
    gd, case, infos, states, N, F = _run(params, "cell24x24x72", precision)
    for k, info in enumerate(infos, start=1):
        assert abs(info["V_cell"] - gd["V_cell"][k]) <= tol_v * abs(gd["V_cell"][k]), (k, info)
        assert abs(info["Li_total"] - gd["Li_total"][k]) <= 1e-12 * gd["Li_total"][k], k
        assert abs(info["Li_plated"] - gd["Li_plated"][k]) <= tol_f * abs(gd["Li_plated"][k]), k
        assert info["passes"] == gd["passes"][k], (k, info, gd["passes"][k])
    k = case["keep"][-1]
    errs = _sampled_errs(states[k], gd["u_%d" % k], int(gd["stride"]), N, F)
    assert all(v <= tol_f for v in errs.values()), errs
