"""The paper's half-cell model-reduction experiment (Sec. results) at small
size on the GPU (paper_1704_04139_gb300.experiment).

* Its full-order runs against the FP64 oracle: the germ-grain plated half
  cell at x_G0 = 0.75, delithiated at the largest current of the paper's
  range, 3 steps: every field and the cell potential to 1e-9 (FP64 path).
* The whole study at small size runs through (snapshots at the three training
  currents, validation and 97 % reduced models, reduced trajectories, the
  error estimate, full-order comparison, the adaptive full-order run): no
  failed instance, finite errors, the reduced model reproduces the training
  currents' trajectories more closely than the estimate's scale suggests
  nothing at all (errors below 1e-2), and the adaptive run covers 60 s.
"""
import numpy as np
import pytest

from oracle.fom import Cell as OCell

pytestmark = pytest.mark.gpu

SMALL = dict(ny=12, nz=12, n_anode=10, n_sep=4, n_foil=1, seed=62)


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


def test_experiment_full_order_matches_oracle(params):
    B = _gpu()
    from paper_1704_04139_gb300 import experiment as X
    lab, prm, mask, hits = X.half_cell_inputs(params, **SMALL)
    assert len(hits) > 0
    gc = B.Cell(lab, 1e-6, prm, B.default_opts(precision=0, newton_tol=1e-12, krylov_rtol=1e-6))
    u0, n_on = X.initial_state(gc, prm, mask)
    assert n_on > 0
    oc = OCell(lab, 1e-6, prm)
    uo = u0.copy()
    gc.set_state(u0)
    for k in range(3):
        info = gc.step(1.0, X.P_MAX)
        uo, oinfo = oc.step(uo, 1.0, X.P_MAX)
        ug = gc.state()
        for sl in (slice(0, oc.N), slice(oc.N, 2 * oc.N), slice(2 * oc.N, None)):
            ref = uo[sl]
            assert np.max(np.abs(ug[sl] - ref)) <= 1e-9 * np.max(np.abs(ref)), (k, sl)
        assert abs(info["V_cell"] - oinfo["V_cell"]) <= 1e-9 * abs(oinfo["V_cell"])
        assert info["passes"] == oinfo["passes"]
    # the plated inventory strips: it decreases under delithiation
    assert np.sum(uo[2 * oc.N:]) < np.sum(u0[2 * oc.N:])
    gc.close()


def test_experiment_runs_at_small_size(params):
    B = _gpu()
    from paper_1704_04139_gb300 import experiment as X
    res = X.run_study(B, params, steps=6, n_test=2, n_more=4, sizes=SMALL)
    assert res["failed"]["reduced"] == 0 and res["failed"]["estimate"] == 0
    assert len(res["rows"]) == 5
    for r in res["rows"]:
        assert len(r["V_fom"]) == 6 and len(r["V_rom"]) == 6
        for f in ("c", "phi"):
            assert np.isfinite(r["rel_err"][f]) and np.isfinite(r["rel_est"][f])
            if r["training"]:
                assert r["rel_err"][f] < 1e-2, (r["mu"], f, r["rel_err"][f])
    ad = res["adaptive_full_order_at_max_current"]
    assert abs(ad["trace_t_dt_V"][-1][0] - 6.0) < 1e-9 and ad["steps"] >= 2
