"""GPU reduced-model online solve (mb_rom_solve_batch) against the oracle's
reduced Newton on the same reduced model (built by the oracle from full-order
snapshots): cell potential and mean graphite concentration per step, FP64
both sides; a batch gives every instance the result it has alone."""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell as OCell
from oracle import rom as R


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


@pytest.fixture(scope="module")
def case(params):
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    oc = OCell(lab, 1e-6, params)
    i1 = oc.i_1c
    u0 = oc.initial_state()
    u0[2 * oc.N::4] = 2e-5
    snaps, _ = R.snapshots(oc, [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0)], 1.0, 5, u0=u0)
    rom = R.build(oc, snaps, (8, 6, 14, 10))
    rom.a0 = rom.U.T @ (R.weights(oc) * u0)
    return lab, oc, rom


def _gpu_rom(B, lab, params, rom):
    gc = B.Cell(lab, 1e-6, params)
    g = B.Rom(gc, rom.U, rom.Pbv, rom.P1c, rom.Ms, rom.Alin, rom.bbnd, rom.Pbv_proj, rom.P1c_proj,
              rom.s_cp, rom.s_ac, rom.a0)
    return gc, g


PRM = [(-3.5, 1.2, 0.5), (-1.0, 1.0, 1.0), (-4.5, 0.6, 4.0)]


def _coef_check(rom, a_gpu, a_ref, tol):
    """Final coefficients element by element, per block (c modes, plated-Li
    modes, phi modes) relative to the block's largest coefficient, and the
    reconstruction on the stencil closure of the points (the values the
    model's nonlinear terms see) in the unknown scales."""
    blocks = (slice(0, rom.nc), slice(rom.nc, rom.rc), slice(rom.rc, rom.rc + rom.rp))
    for name, sl in zip(("c", "n", "phi"), blocks):
        ref = a_ref[sl]
        if ref.size == 0 or np.max(np.abs(ref)) == 0:
            continue
        err = np.max(np.abs(a_gpu[sl] - ref)) / np.max(np.abs(ref))
        assert err <= tol, (name, err)
    ug = rom.Uloc @ a_gpu
    uo = rom.Uloc @ a_ref
    assert np.max(np.abs(ug - uo) / rom.us_loc) <= tol


@pytest.mark.gpu
def test_rom_solve_matches_oracle(params, case):
    B = _gpu()
    lab, oc, rom = case
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in PRM]
    out = g.solve(prm, 5, 1.0)
    assert out["ok"] and out["failed"] == 0
    for b, p in enumerate(prm):
        ref = R.solve(rom, p[0], p[1], p[2], 1.0, 5)
        assert np.max(np.abs(out["V"][b] - ref["V_cell"])) <= 1e-9 * np.max(np.abs(ref["V_cell"])), b
        assert np.max(np.abs(out["s_ac"][b] - ref["s_ac"])) <= 1e-9 * np.max(np.abs(ref["s_ac"])), b
        # reconstructed state at the stencil closure (the values the model sees)
        ug = rom.Uloc @ out["a"][b]
        uo = rom.Uloc @ ref["a"][-1]
        assert np.max(np.abs(ug - uo) / rom.us_loc) <= 1e-8, b
    g.close()
    gc.close()


@pytest.mark.gpu
def test_rom_batch_equals_alone(params, case):
    B = _gpu()
    lab, oc, rom = case
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in PRM]
    mix = g.solve(prm, 4, 1.0)
    for b, p in enumerate(prm):
        alone = g.solve([p], 4, 1.0)
        assert np.array_equal(alone["V"][0], mix["V"][b]), b
        assert np.array_equal(alone["a"][0], mix["a"][b]), b
    g.close()
    gc.close()


@pytest.mark.gpu
def test_rom_zero_current_matches_oracle(params, case):
    """Zero current (relaxation of the seeded plated Li) on the GPU and in the oracle."""
    B = _gpu()
    lab, oc, rom = case
    gc, g = _gpu_rom(B, lab, params, rom)
    out = g.solve([(0.0, 1.0, 1.0)], 3, 1.0)
    ref = R.solve(rom, 0.0, 1.0, 1.0, 1.0, 3)
    assert out["ok"]
    assert np.max(np.abs(out["V"][0] - ref["V_cell"])) <= 1e-9 * np.max(np.abs(ref["V_cell"]))
    g.close()
    gc.close()


@pytest.fixture(scope="module")
def wide_case(params):
    """A reduced model with more than 96 modes (the paper's ROMs have 252), so
    that the GPU takes its paths for large N_r (row-per-block Newton matrix,
    block LU in global memory): six trajectories of 12 steps on a 5x5x17
    cell."""
    lab = syn.full_cell(5, 5, 6, 3, 6, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    oc = OCell(lab, 1e-6, params)
    i1 = oc.i_1c
    u0 = oc.initial_state()
    u0[2 * oc.N::4] = 2e-5
    pts = [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0), (-0.5 * i1, 1.5, 0.3), (-3.5 * i1, 0.5, 8.0),
           (-1.0 * i1, 2.0, 1.5), (-4.0 * i1, 1.2, 0.1)]
    snaps, _ = R.snapshots(oc, pts, 1.0, 12, u0=u0)
    rom = R.build(oc, snaps, (70, 60, 40, 30), pod_tol=1e-12)
    rom.a0 = rom.U.T @ (R.weights(oc) * u0)
    return lab, oc, rom


@pytest.mark.gpu
def test_rom_wide_matches_oracle(params, wide_case):
    B = _gpu()
    lab, oc, rom = wide_case
    assert rom.U.shape[1] > 96
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-3.0, 1.1, 0.7), (-1.5, 0.8, 2.0)]]
    out = g.solve(prm, 3, 1.0)
    assert out["ok"] and out["failed"] == 0
    for b, p in enumerate(prm):
        ref = R.solve(rom, p[0], p[1], p[2], 1.0, 3)
        assert np.max(np.abs(out["V"][b] - ref["V_cell"])) <= 1e-9 * np.max(np.abs(ref["V_cell"])), b
        assert np.max(np.abs(out["s_ac"][b] - ref["s_ac"])) <= 1e-9 * np.max(np.abs(ref["s_ac"])), b
        _coef_check(rom, out["a"][b], ref["a"][-1], 1e-8)
    g.close()
    gc.close()


@pytest.mark.gpu
@pytest.mark.parametrize("tc,Nr,M,nb", [(1, 70, 100, 3), (0, 70, 100, 3), (2, 70, 100, 3), (2, 209, 1000, 5),
                                        (2, 256, 64, 1)])
def test_rom_newton_matrix_kernel(tc, Nr, M, nb):
    """The Newton-matrix kernels against an FP64 product: J_b = P GU_b + Ms/dt_b + Alin,
    ragged in rows (70, 209), the contraction (100, 1000) and the columns (nb x Nr);
    all keep FP32 accuracy: FP32 FMA (0), three TF32 products per pair on mma.sync
    (1) or on tcgen05 with the accumulator in tensor memory (2; also the largest
    reduced dimension it takes, 256)."""
    B = _gpu()
    rng = np.random.default_rng(7 + Nr)
    P = rng.standard_normal((Nr, M)).astype(np.float32)
    GU = rng.standard_normal((nb, M, Nr)).astype(np.float32)
    Ms = rng.standard_normal((Nr, Nr)).astype(np.float32)
    Al = rng.standard_normal((Nr, Nr)).astype(np.float32)
    dti = np.array([0.5, 2.0, 10.0, 1.0, 4.0])[:nb]
    J = B.debug_rom_jac(P, GU, Ms, Al, dti, tc=tc)
    P64, G64 = P.astype(np.float64), GU.astype(np.float64)
    for b in range(nb):
        ref = P64 @ G64[b] + Ms.astype(np.float64) * np.float32(dti[b]) + Al.astype(np.float64)
        # |P| |GU| bounds the rounding of an FP32 sum of M products
        scale = np.abs(P64) @ np.abs(G64[b]) + np.abs(Ms) * dti[b] + np.abs(Al)
        assert np.all(np.abs(J[b] - ref) <= 4 * M * 2.0 ** -24 * scale), b


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["case", "wide_case"])
def test_rom_tensor_newton_matrix_same_result(params, request, which):
    """The online solve with either tensor-core Newton matrix (mma.sync, or
    tcgen05 with the accumulator in tensor memory) converges to the same reduced
    trajectory as with the FP32-FMA one (the matrix only steers Newton)."""
    B = _gpu()
    lab, oc, rom = request.getfixturevalue(which)
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-2.0, 1.0, 1.0), (1.0, 0.9, 0.5), (-4.0, 0.7, 3.0)]]
    out = {}
    for tc in (1, 0, 2):
        g.debug_tensor(tc)
        out[tc] = g.solve(prm, 4, 1.0)
        assert out[tc]["ok"], tc
    for tc in (0, 2):
        assert np.max(np.abs(out[tc]["V"] - out[1]["V"])) <= 1e-9 * np.max(np.abs(out[1]["V"])), tc
    g.close()
    gc.close()


@pytest.mark.gpu
def test_rom_gemm_autotuning(params, request):
    """Without a fixed variant, every GEMM variant the model admits is timed
    once per model shape and the fastest kept; the solve then gives exactly
    what the same variant gives when fixed (same kernels, same arithmetic)."""
    B = _gpu()
    lab, oc, rom = request.getfixturevalue("case")
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-2.0, 1.0, 1.0), (1.0, 0.9, 0.5), (-4.0, 0.7, 3.0)]]
    auto = g.solve(prm, 3, 1.0)
    choice, ms = g.gemm_tuning()
    assert auto["ok"] and choice in (0, 1, 2)
    timed = [m for m in ms if m >= 0]
    assert len(timed) >= 2 and ms[choice] == min(timed)
    g.close()
    g2 = B.Rom(gc, rom.U, rom.Pbv, rom.P1c, rom.Ms, rom.Alin, rom.bbnd, rom.Pbv_proj, rom.P1c_proj,
               rom.s_cp, rom.s_ac, rom.a0)
    g2.debug_tensor(choice)
    fixed = g2.solve(prm, 3, 1.0)
    assert np.array_equal(fixed["V"], auto["V"])
    assert g2.gemm_tuning()[0] == choice
    g2.close()
    gc.close()


@pytest.mark.gpu
@pytest.mark.parametrize("Nr,fp64,in_place", [(70, True, False), (70, False, False), (112, True, True),
                                              (150, False, True), (209, False, False), (209, True, True),
                                              (260, False, True), (300, False, True)])
def test_rom_newton_step_lu_kernel(Nr, fp64, in_place):
    """The Newton-step LU kernel against a library solve: random matrices with rows
    scaled over twelve decades (the equilibration removes that) and a zero leading
    diagonal (the pivoting has to move it), in shared memory, or with the leading
    rows in shared memory and the rest in place (FP64 from 166 rows, FP32 from 236:
    209 and 260, 300 here)."""
    B = _gpu()
    rng = np.random.default_rng(Nr)
    nb = 5
    J = rng.standard_normal((nb, Nr, Nr))
    J[:, 0, 0] = 0.0
    J *= 10.0 ** rng.uniform(-6, 6, (nb, Nr, 1))
    r = rng.standard_normal((nb, Nr))
    d = B.debug_rom_lu(J, r, fp64=fp64, in_place=in_place)
    for b in range(nb):
        ref = -np.linalg.solve(J[b], r[b])
        scale = np.max(np.abs(ref))
        # error of a backward-stable solve: ~ cond(equilibrated J) * unit roundoff
        tol = 1e-9 if fp64 else 2e-3
        assert np.max(np.abs(d[b] - ref)) <= tol * scale, (b, np.max(np.abs(d[b] - ref)) / scale)


@pytest.mark.gpu
def test_rom_refine_matches_oracle(params, wide_case):
    """Escalated instances by GMRES on FP64 products, preconditioned by the FP32 LU
    kept from their last FP32-matrix iteration: the 112-mode model (whose FP32 matrix
    cannot converge, so instances escalate) reaches the oracle's trajectory at 1e-9
    and the FP64-LU path's."""
    B = _gpu()
    lab, oc, rom = wide_case
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-3.0, 1.1, 0.7), (-1.5, 0.8, 2.0), (-4.5, 0.6, 4.0)]]
    g.debug_refine(False)
    lu = g.solve(prm, 3, 1.0)
    g.debug_refine(True)
    out = g.solve(prm, 3, 1.0)
    assert out["ok"] and out["failed"] == 0
    for b, p in enumerate(prm):
        ref = R.solve(rom, p[0], p[1], p[2], 1.0, 3)
        assert np.max(np.abs(out["V"][b] - ref["V_cell"])) <= 1e-9 * np.max(np.abs(ref["V_cell"])), b
        assert np.max(np.abs(out["s_ac"][b] - ref["s_ac"])) <= 1e-9 * np.max(np.abs(ref["s_ac"])), b
        _coef_check(rom, out["a"][b], ref["a"][-1], 1e-8)
        _coef_check(rom, lu["a"][b], ref["a"][-1], 1e-8)
    assert np.max(np.abs(out["V"] - lu["V"])) <= 1e-9 * np.max(np.abs(lu["V"]))
    g.close()
    gc.close()


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["case", "wide_case"])
def test_rom_step_graph_bit_identical(params, request, which):
    """A reduced time step as one CUDA graph (conditional nodes run the
    active-set passes, the Newton iterations and the escalated-instance branch
    on the device) gives bit-identical trajectories, coefficients and counts to
    the host-driven step.  The 112-mode model escalates instances, so the
    escalated branch runs inside the graph."""
    B = _gpu()
    lab, oc, rom = request.getfixturevalue(which)
    gc, g = _gpu_rom(B, lab, params, rom)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-3.0, 1.1, 0.7), (-1.5, 0.8, 2.0), (-4.5, 0.6, 4.0),
                                                  (0.0, 1.0, 1.0), (2.0, 1.3, 0.3)]]
    g.debug_graph(False)
    host = g.solve(prm, 3, 1.0)
    g.debug_graph(True)
    graph = g.solve(prm, 3, 1.0)
    assert host["ok"] and graph["ok"]
    assert np.array_equal(host["V"], graph["V"]) and np.array_equal(host["s_ac"], graph["s_ac"])
    assert np.array_equal(host["a"], graph["a"])
    assert host["newton_its"] == graph["newton_its"] and host["flips"] == graph["flips"]
    g.close()
    gc.close()
