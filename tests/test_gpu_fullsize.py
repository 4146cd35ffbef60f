"""The bench's own workload, in the launch configuration bench.py times: the
128x128x256-voxel full cell (4.2M voxels, 0.43M plating faces), mixed
precision, Newton to 1e-10, Eisenstat-Walker forcing, the 2C charge.  The
oracle cannot solve this size, so the checks are properties that hold at any
size and that the oracle's pins fix on small cells:

* conservation of the finite-volume scheme (Sec. workflow:discretization; the
  oracle's T7 pin): the total Li (solid + electrolyte + plated) is constant and
  the anode inventory (graphite + plated) changes by -dt A_cross I / F per step
  (1e-9 of the total and 1e-5 of the per-step exchange, which is ~4e-4 of the
  anode inventory: a relative state error of 1e-10, the Newton tolerance, moves
  it by ~3e-7);
* the mixed-precision path against the FP64 path on the same steps: cell
  potential to 1e-6 relative and every field to 1e-5 (the bench's accuracy
  target), each converged to the same Newton tolerance.
"""
import types

import numpy as np
import pytest

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


def _bench_opts(B, prec):
    import bench
    args = types.SimpleNamespace(fp32_coarse=False, mg_stream=3, mg_tail=0, no_ew=False, kcycle_cgs1=False,
                                 mg_kcycle=5, mg_smooth=2, mg_coarse=[2, 2], no_pc_lag=False, pc_lag_drift=0.05, mg_pdl=0,
                                 no_newton_rate_test=False)
    return bench.fom_opts(B, prec, args)


def test_bench_cell_conservation_and_precision(params):
    B = _gpu()
    import bench
    lab = bench.workload_labels("cell128x128x256")
    h, dt, steps = 1e-6, 1.0, 3
    A_cross = lab.shape[1] * lab.shape[2] * h * h
    runs = {}
    for prec in (B.PREC_MIXED, B.PREC_FP64):
        cell = B.Cell(lab, h, params, _bench_opts(B, prec))
        I = bench.CRATE["cell128x128x256"] * cell.i_1c
        infos = [cell.step(dt, I) for _ in range(steps)]
        runs[prec] = (infos, cell.state())
        cell.close()
        tot = np.array([i["Li_total"] for i in infos])
        assert np.max(np.abs(tot - tot[0])) <= 1e-9 * tot[0], tot
        anode = np.array([i["Li_anode"] for i in infos])
        expect = -dt * A_cross * I / params["F"]
        assert np.max(np.abs(np.diff(anode) - expect)) <= 1e-5 * abs(expect), (np.diff(anode), expect)
    (im, um), (i64, u64) = runs[B.PREC_MIXED], runs[B.PREC_FP64]
    for a, b in zip(im, i64):
        assert abs(a["V_cell"] - b["V_cell"]) <= 1e-6 * abs(b["V_cell"])
    n_vox = lab.size
    for sl in (slice(0, n_vox), slice(n_vox, 2 * n_vox), slice(2 * n_vox, None)):
        ref = u64[sl]
        if np.max(np.abs(ref)) > 0:
            assert np.max(np.abs(um[sl] - ref)) <= 1e-5 * np.max(np.abs(ref))
