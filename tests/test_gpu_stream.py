"""The ways the coarse sweeps fetch their operator rows compute the same
thing: plain loads (mg_stream 0), L2 prefetch one resident wave ahead (1)
the staged sweep with bulk asynchronous copies into shared memory (2) and
the level-1 sweep at 5 blocks per SM (3) give bit-identical preconditioner
applications and implicit steps, on a cell
whose level 1 holds more than one tile of 256 cells per SM, so that the
staged kernel runs there."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding, torch


def test_stream_modes_bit_identical(params):
    B, torch = _gpu()
    lab = syn.full_cell(64, 64, 53, 22, 53, 0.35, 0.35, ("uniform", 2, 4), (31, 32))
    cells = {s: B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4,
                                                         mg_stream=s)) for s in (0, 1, 2, 3)}
    a, b = cells[2], cells[0]
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    l1 = a.debug_levels()[0]
    assert l1[0] * l1[1] * l1[2] >= 256 * nsm
    rng = np.random.default_rng(5)
    N = a.N
    u = a.state()
    u[:N] *= 1.0 + 0.01 * rng.standard_normal(N)
    u[N:2 * N] += 0.002 * rng.standard_normal(N)
    gate = np.zeros(a.F, np.uint8)
    r = rng.standard_normal(a.n)
    z = {s: cells[s].debug_precond(u, gate, 1.0, r) for s in cells}
    assert np.all(np.isfinite(z[0]))
    assert np.array_equal(z[1], z[0]) and np.array_equal(z[2], z[0]) and np.array_equal(z[3], z[0])
    I = -2.0 * a.i_1c
    info = {s: cells[s].step(1.0, I) for s in cells}
    for s in (1, 2, 3):
        assert info[s]["krylov_its"] == info[0]["krylov_its"] and info[s]["V_cell"] == info[0]["V_cell"]
        assert np.array_equal(cells[s].state(), cells[0].state())
    for cell in cells.values():
        cell.close()


def test_coarse_tail_bit_identical(params):
    """The persistent coarse tail (levels 2, or 3, down to the coarsest solve in
    one cooperative launch, grid barriers between the phases) runs the
    per-level kernels' per-cell code in the same order: preconditioner
    applications and implicit steps are bit-identical to per-level launches."""
    B, torch = _gpu()
    lab = syn.full_cell(64, 64, 53, 22, 53, 0.35, 0.35, ("uniform", 2, 4), (31, 32))
    cells = {t: B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4,
                                                         mg_tail=t)) for t in (0, 1, 3)}
    a = cells[1]
    assert len(a.debug_levels()) >= 5
    rng = np.random.default_rng(9)
    N = a.N
    u = a.state()
    u[:N] *= 1.0 + 0.01 * rng.standard_normal(N)
    u[N:2 * N] += 0.002 * rng.standard_normal(N)
    gate = np.zeros(a.F, np.uint8)
    r = rng.standard_normal(a.n)
    z = {t: cells[t].debug_precond(u, gate, 1.0, r) for t in cells}
    assert np.all(np.isfinite(z[0]))
    assert np.array_equal(z[1], z[0]) and np.array_equal(z[3], z[0])
    I = -2.0 * a.i_1c
    for _ in range(2):
        info = {t: cells[t].step(1.0, I) for t in cells}
        for t in (1, 3):
            assert info[t]["krylov_its"] == info[0]["krylov_its"] and info[t]["V_cell"] == info[0]["V_cell"]
    assert np.array_equal(cells[1].state(), cells[0].state())
    assert np.array_equal(cells[3].state(), cells[0].state())
    for cell in cells.values():
        cell.close()


def test_lagged_preconditioner_same_solution(params):
    """With the preconditioner rebuilt only when the Krylov iterations grow
    (pc_lag = 1) the Newton iterations converge to the same states as with a
    rebuild at every iteration: only the preconditioner's age differs, the
    residual, the Krylov operator and the Newton tolerance are the same, so the
    states agree to the tolerance (1e-10 scaled update; checked at 1e-8 of each
    field and 1e-9 of the cell potential over a 2C charge with plating)."""
    B, torch = _gpu()
    lab = syn.full_cell(32, 32, 40, 16, 40, 0.35, 0.35, ("uniform", 2, 4), (11, 12))
    cells = {lag: B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4,
                                                           pc_lag=lag)) for lag in (0, 1)}
    I = -2.0 * cells[0].i_1c
    for _ in range(4):
        info = {lag: cells[lag].step(1.0, I) for lag in cells}
        assert abs(info[1]["V_cell"] - info[0]["V_cell"]) <= 1e-9 * abs(info[0]["V_cell"])
    u0, u1 = cells[0].state(), cells[1].state()
    N = cells[0].N
    for sl in (slice(0, N), slice(N, 2 * N), slice(2 * N, None)):
        if np.max(np.abs(u0[sl])) > 0:
            assert np.max(np.abs(u1[sl] - u0[sl])) <= 1e-8 * np.max(np.abs(u0[sl]))
    for cell in cells.values():
        cell.close()


def test_programmatic_dependent_launch_bit_identical(params):
    """With programmatic dependent launch (mg_pdl = 1) every kernel of an
    application waits for its predecessor before its first memory access, so
    preconditioner applications and implicit steps are bit-identical to plain
    launches (graph-captured and direct)."""
    B, torch = _gpu()
    lab = syn.full_cell(64, 64, 53, 22, 53, 0.35, 0.35, ("uniform", 2, 4), (31, 32))
    cells = {q: B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4,
                                                         mg_pdl=q)) for q in (0, 1)}
    a = cells[1]
    rng = np.random.default_rng(13)
    N = a.N
    u = a.state()
    u[:N] *= 1.0 + 0.01 * rng.standard_normal(N)
    u[N:2 * N] += 0.002 * rng.standard_normal(N)
    gate = np.zeros(a.F, np.uint8)
    r = rng.standard_normal(a.n)
    z = {q: cells[q].debug_precond(u, gate, 1.0, r) for q in cells}
    assert np.all(np.isfinite(z[0]))
    assert np.array_equal(z[1], z[0])
    I = -2.0 * a.i_1c
    for _ in range(2):
        info = {q: cells[q].step(1.0, I) for q in cells}
        assert info[1]["krylov_its"] == info[0]["krylov_its"] and info[1]["V_cell"] == info[0]["V_cell"]
    assert np.array_equal(cells[1].state(), cells[0].state())
    for cell in cells.values():
        cell.close()


def test_newton_rate_test_same_solution(params):
    """Stopping Newton once the error left after an update, estimated from the
    contraction of two full steps, is below the tolerance (newton_rate_test =
    1) skips the confirming iteration but not accuracy: over a 2C charge with
    plating the states agree with update-based stopping to 1e-9 of each field
    and 1e-10 of the cell potential (newton_tol 1e-10 in the scaled max-norm),
    with no more Newton iterations."""
    B, torch = _gpu()
    lab = syn.full_cell(32, 32, 40, 16, 40, 0.35, 0.35, ("uniform", 2, 4), (11, 12))
    cells = {q: B.Cell(lab, 1e-6, params, B.default_opts(precision=1, newton_tol=1e-10, krylov_rtol=1e-4,
                                                         newton_rate_test=q)) for q in (0, 1)}
    I = -2.0 * cells[0].i_1c
    its = {0: 0, 1: 0}
    for _ in range(4):
        info = {q: cells[q].step(1.0, I) for q in cells}
        for q in cells:
            its[q] += info[q]["newton_its"]
        assert abs(info[1]["V_cell"] - info[0]["V_cell"]) <= 1e-10 * abs(info[0]["V_cell"])
    assert its[1] <= its[0]
    u0, u1 = cells[0].state(), cells[1].state()
    N = cells[0].N
    for sl in (slice(0, N), slice(N, 2 * N), slice(2 * N, None)):
        if np.max(np.abs(u0[sl])) > 0:
            assert np.max(np.abs(u1[sl] - u0[sl])) <= 1e-9 * np.max(np.abs(u0[sl]))
    for cell in cells.values():
        cell.close()
