"""Kernel timing and launch counting around mb_step (the counters bench.py
reads): the graph-replayed preconditioner reports its smoother launches, and
enabling or disabling timing between steps leaves the step working."""
import pytest

import synthetic as syn


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


@pytest.mark.gpu
def test_profiling_counters_across_steps(params):
    B = _gpu()
    lab = syn.full_cell(5, 7, 9, 4, 8, 0.35, 0.35, ("uniform", 1.5, 3), (3, 4))
    cell = B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4))
    I = -2.0 * cell.i_1c
    cell.step(1.0, I)                      # graphs captured with timing off
    cell.prof_enable(True)
    l0 = cell.launch_count()
    info = cell.step(1.0, I)
    n_pc, ms_pc = cell.prof_read(B.Cell.PROF_PRECOND)
    n_sm, ms_sm = cell.prof_read(B.Cell.PROF_SMOOTH)
    n_op, ms_op = cell.prof_read(B.Cell.PROF_JVP)
    n_r, ms_r = cell.prof_read(B.Cell.PROF_RESIDUAL)
    assert info["krylov_its"] > 0
    assert n_pc >= info["krylov_its"] and ms_pc > 0
    # every preconditioner application runs 2 * mg_smooth - 1 fine sweeps with a product
    assert n_sm == (2 * B.default_opts().mg_smooth - 1) * n_pc and ms_sm > 0
    # and per level-1 V-cycle (one per K-cycle iteration) mg_coarse_post timed post-smoothing sweeps
    n_ls, ms_ls = cell.prof_read(B.Cell.PROF_LSMOOTH)
    if len(cell.debug_levels()) > 1:
        o = B.default_opts()
        assert n_ls == o.mg_coarse_post * o.mg_kcycle * n_pc and 0 < ms_ls < ms_pc
    else:
        assert n_ls == 0
    assert n_op >= info["krylov_its"] and n_r >= info["newton_its"]
    assert ms_sm < ms_pc
    assert cell.launch_count() > l0
    cell.prof_enable(False)
    cell.step(1.0, I)                      # and off again
    cell.close()
