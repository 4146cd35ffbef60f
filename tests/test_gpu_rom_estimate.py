"""GPU hierarchical error estimate (mb_rom_estimate_batch, Eq. ap4:estimate)
against the oracle's error_estimate, which forms both reconstructions over
the whole grid and takes the L^2 norm of their difference (the definition).

* Arithmetic: on the GPU's own final coefficients of both models (the same
  trajectories mb_rom_solve_batch returns: an instance's arithmetic does not
  depend on the batch), the estimate matches to 1e-9 relative.
* Trajectories: at every step the estimate matches the oracle's estimate on
  the oracle's reduced trajectories within 1e-8 of each field's
  reconstruction norm (the two trajectories agree to ~1e-9).

Two pairs: a validation model whose bases extend the reduced model's (both
truncations of the same POD and EI-Greedy, as the paper's 97 % model is) and
a reduced model built from other snapshots, so that part of its basis lies
outside the validation span (the remainder term).
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell as OCell
from oracle import rom as R

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


@pytest.fixture(scope="module")
def models(params):
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    oc = OCell(lab, 1e-6, params)
    i1 = oc.i_1c
    u0 = oc.initial_state()
    u0[2 * oc.N::4] = 2e-5
    snaps, _ = R.snapshots(oc, [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0)], 1.0, 5, u0=u0)
    val = R.build(oc, snaps, (12, 9, 24, 16))
    nested = R.build(oc, snaps, (8, 6, 14, 10))
    snaps2, _ = R.snapshots(oc, [(-3 * i1, 1.3, 0.5)], 1.0, 4, u0=u0)
    other = R.build(oc, snaps2, (6, 5, 12, 8))
    for m in (val, nested, other):
        m.a0 = m.U.T @ (R.weights(oc) * u0)
    return lab, oc, val, nested, other


def _gpu_rom(B, gc, rom):
    return B.Rom(gc, rom.U, rom.Pbv, rom.P1c, rom.Ms, rom.Alin, rom.bbnd, rom.Pbv_proj, rom.P1c_proj,
                 rom.s_cp, rom.s_ac, rom.a0)


@pytest.mark.parametrize("which", ["nested", "other"])
def test_error_estimate_matches_oracle(params, models, which):
    B = _gpu()
    lab, oc, val, nested, other = models
    red = nested if which == "nested" else other
    gc = B.Cell(lab, 1e-6, params)
    g_red, g_val = _gpu_rom(B, gc, red), _gpu_rom(B, gc, val)
    prm = [(c * oc.i_1c, s, k) for (c, s, k) in [(-3.5, 1.2, 0.5), (-1.0, 1.0, 1.0), (-4.5, 0.6, 4.0)]]
    theta, steps = 0.3, 4
    out = g_red.estimate(g_val, prm, steps, 1.0, theta)
    assert out["ok"] and out["failed"] == 0
    a_red = g_red.solve(prm, steps, 1.0)
    a_val = g_val.solve(prm, steps, 1.0)
    assert np.array_equal(out["V"], a_red["V"]) and np.array_equal(out["V_val"], a_val["V"])
    w = R.weights(oc)
    N = oc.N
    fields = (slice(0, N), slice(N, 2 * N), slice(2 * N, None))
    for b, p in enumerate(prm):
        # arithmetic on the GPU's own final coefficients
        ref = R.error_estimate(red, val, a_red["a"][b], a_val["a"][b], theta)
        for f, key in enumerate(("c", "phi", "n")):
            e_ref = float(ref[key][0])
            assert abs(out["est"][b, -1, f] - e_ref) <= 1e-9 * e_ref + 1e-300, (b, key, out["est"][b, -1, f], e_ref)
        # every step against the oracle's own trajectories
        tr = R.solve(red, p[0], p[1], p[2], 1.0, steps)
        tv = R.solve(val, p[0], p[1], p[2], 1.0, steps)
        ref = R.error_estimate(red, val, np.array(tr["a"]), np.array(tv["a"]), theta)
        recon = np.array(tr["a"]) @ red.U.T
        for f, key in enumerate(("c", "phi", "n")):
            scale = np.sqrt(np.sum(w[fields[f]] * recon[:, fields[f]] ** 2, axis=1))
            assert np.all(np.abs(out["est"][b, :, f] - ref[key]) <= 1e-8 * scale + 1e-300), (b, key)
    # the validation model's field norms, and the block dimensions
    for b, p in enumerate(prm):
        recon = a_val["a"][b] @ val.U.T
        for f in range(3):
            nref = np.sqrt(np.sum(w[fields[f]] * recon[fields[f]] ** 2))
            assert abs(out["norm_val"][b, -1, f] - nref) <= 1e-12 * nref + 1e-300
    assert g_val.block_dims() == (val.nc, val.nn, val.rp)
    # the estimate scales as 1 / (1 - theta)
    out0 = g_red.estimate(g_val, prm, steps, 1.0, 0.0)
    assert np.allclose(out0["est"] / (1 - theta), out["est"], rtol=1e-14, atol=0)
    g_red.close()
    g_val.close()
    gc.close()


def test_error_estimate_rejects_bad_arguments(params, models):
    B = _gpu()
    lab, oc, val, nested, other = models
    gc = B.Cell(lab, 1e-6, params)
    g_red, g_val = _gpu_rom(B, gc, nested), _gpu_rom(B, gc, val)
    with pytest.raises(B.MBError):
        g_red.estimate(g_val, [(-oc.i_1c, 1.0, 1.0)], 2, 1.0, theta=1.0)
    with pytest.raises(B.MBError):
        g_red.estimate(g_red, [(-oc.i_1c, 1.0, 1.0)], 2, 1.0)
    g_red.close()
    g_val.close()
    gc.close()
