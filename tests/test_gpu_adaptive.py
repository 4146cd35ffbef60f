"""Adaptive time stepping (mb_step_adaptive) against the oracle's controller
(oracle.fom.Cell.step_adaptive): the same local error estimate, accept/reject
decisions and proposed step sizes, over a protocol whose current reverses
(charge with seeded plated lithium, then delithiation that strips it), so that
the controller shrinks the step at the switch and grows it afterwards.

Tolerances: step sizes 1e-9 relative (they are computed from the states), cell
potential and every field 1e-9 relative (FP64 path), rejection counts equal.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell as OCell

pytestmark = pytest.mark.gpu


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("geom", ["tiny", "half"])
def test_adaptive_steps_match_oracle(params, geom):
    B = _gpu()
    if geom == "tiny":
        lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    else:
        lab = syn.half_cell(6, 5, 8, 4, 3, 0.35, ("uniform", 1.5, 3), 7)
    oc = OCell(lab, 1e-6, params)
    opts = B.default_opts(precision=0, newton_tol=1e-12, krylov_rtol=1e-6)
    gc = B.Cell(lab, 1e-6, params, opts)
    u = oc.initial_state()
    u[2 * oc.N::3] = 4e-5
    gc.set_state(u)
    tol, dt_min, dt_max = 2e-4, 1e-3, 5.0
    protocol = [-3.0] * 4 + [4.0] * 6
    u_hist, dt_hist, dt_try = None, None, 0.5
    rejects = 0
    for k, crate in enumerate(protocol):
        I = crate * oc.i_1c
        u_new, oi = oc.step_adaptive(u, u_hist, dt_hist, dt_try, I, tol, dt_min, dt_max)
        gi = gc.step_adaptive(dt_try, I, tol, dt_min, dt_max)
        assert gi["rejects"] == oi["rejects"], (k, gi, oi)
        assert abs(gi["dt_used"] - oi["dt_used"]) <= 1e-9 * oi["dt_used"], (k, gi["dt_used"], oi["dt_used"])
        assert abs(gi["dt_next"] - oi["dt_next"]) <= 1e-9 * oi["dt_next"], (k, gi["dt_next"], oi["dt_next"])
        assert abs(gi["V_cell"] - oi["V_cell"]) <= 1e-9 * abs(oi["V_cell"]), k
        ug = gc.state()
        for sl in (slice(0, oc.N), slice(oc.N, 2 * oc.N), slice(2 * oc.N, None)):
            if np.max(np.abs(u_new[sl])) > 0:
                assert _rel(ug[sl], u_new[sl]) <= 1e-9, (k, sl)
        rejects += oi["rejects"]
        u_hist, dt_hist, dt_try = u, oi["dt_used"], oi["dt_next"]
        u = u_new
    assert rejects >= 1          # the controller did reject at the current reversal
    gc.close()


def test_adaptive_history_is_reset_by_fixed_steps(params):
    """mb_step (a fixed step) and mb_state_set end the adaptive history: the
    next adaptive step is taken at the size given, without an estimate."""
    B = _gpu()
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    gc = B.Cell(lab, 1e-6, params)
    I = -2.0 * gc.i_1c
    gc.step_adaptive(0.5, I, 1e-4)
    gc.step(0.5, I)
    a = gc.step_adaptive(0.7, I, 1e-4)
    assert a["err"] == 0.0 and a["dt_used"] == 0.7 and a["rejects"] == 0
    gc.set_state(gc.state())
    b = gc.step_adaptive(0.3, I, 1e-4)
    assert b["err"] == 0.0 and b["dt_used"] == 0.3
    gc.close()
