"""Serving loop (mb_serve_*): requests that arrive while others run join the
resident reduced batch; every reduced result is bit-identical to the same
request solved alone, and a full-order request running beside the reduced
batch equals a direct step sequence on its own cell."""
import time

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


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        if time.time() - t0 > timeout:
            raise TimeoutError("serving requests did not finish")
        time.sleep(0.002)
    return out


@pytest.mark.gpu
def test_serving_mix_equals_alone(params):
    B = _gpu()
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    oc = OCell(lab, 1e-6, params)
    i1 = oc.i_1c
    u0 = oc.initial_state()
    snaps, _ = R.snapshots(oc, [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0)], 1.0, 5)
    rom = R.build(oc, snaps, (8, 6, 14, 10))
    gc = B.Cell(lab, 1e-6, params)
    g = B.Rom(gc, rom.U, rom.Pbv, rom.P1c, rom.Ms, rom.Alin, rom.bbnd, rom.Pbv_proj, rom.P1c_proj,
              rom.s_cp, rom.s_ac, rom.a0)
    reqs = [(-3.5, 1.2, 0.5, 6), (-1.0, 1.0, 1.0, 3), (-4.5, 0.6, 4.0, 8), (-2.0, 1.5, 0.2, 2),
            (-0.5, 0.8, 2.0, 5)]
    alone = {}
    for k, (c, s, kp, n) in enumerate(reqs):
        alone[k] = g.solve([(c * i1, s, kp)], n, 1.0)
    fom_ref = B.Cell(lab, 1e-6, params)
    V_fom = [float(np.mean(fom_ref.state()[oc.N:2 * oc.N].reshape(oc.shape)[-1]))]
    for _ in range(3):
        V_fom.append(fom_ref.step(1.0, -2.0 * i1)["V_cell"])
    fom_ref.close()
    # a second full-order request with other scales: the worker reuses its cell, reset to the
    # initial state, and must give what a fresh cell gives
    fom_ref2 = B.Cell(lab, 1e-6, params)
    fom_ref2.set_scales(0.7, 3.0)
    V_fom2 = [fom_ref2.step(1.0, -4.0 * i1)["V_cell"] for _ in range(2)]
    fom_ref2.close()
    srv = B.Server(rom=g, labels=lab, params=params, rom_slots=3, fom_workers=1)
    tk = {}
    tk["fom"] = srv.submit(B.REQ_FOM, -2.0 * i1, 1.0, 1.0, 3, 1.0)
    tk["fom2"] = srv.submit(B.REQ_FOM, -4.0 * i1, 0.7, 3.0, 2, 1.0)
    for k in range(3):
        c, s, kp, n = reqs[k]
        tk[k] = srv.submit(B.REQ_ROM, c * i1, s, kp, n, 1.0)
    time.sleep(0.01)
    for k in range(3, len(reqs)):          # second wave while the first runs
        c, s, kp, n = reqs[k]
        tk[k] = srv.submit(B.REQ_ROM, c * i1, s, kp, n, 1.0)
    res = _wait(srv, list(tk.values()))
    srv.close()
    for k in range(len(reqs)):
        r = res[tk[k]]
        assert r["status"] == 0
        assert np.array_equal(r["V"], alone[k]["V"][0]), k
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
    rf = res[tk["fom"]]
    assert rf["status"] == 0
    assert np.array_equal(rf["V"][1:], np.array(V_fom[1:]))          # same kernels, same order
    assert abs(rf["V"][0] - V_fom[0]) <= 1e-14 * abs(V_fom[0])         # host means, different summation order
    rf2 = res[tk["fom2"]]
    assert rf2["status"] == 0 and rf2["t_start"] >= rf["t_done"]
    assert np.array_equal(rf2["V"][1:], np.array(V_fom2))
    g.close()
    gc.close()


@pytest.mark.gpu
def test_full_order_admission_by_device_memory(params):
    """With a device-memory budget of one cell and four workers, full-order
    requests never hold more than one cell at a time: before the first cell's
    size is known only one worker may create one, and afterwards a second cell
    does not fit the budget.  All requests still complete."""
    B = _gpu()
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    probe = B.Cell(lab, 1e-6, params)
    one_cell = int(probe.device_bytes)
    i1 = probe.i_1c
    probe.close()
    srv = B.Server(labels=lab, params=params, fom_budget_bytes=one_cell, fom_workers=4)
    tickets = [srv.submit(B.REQ_FOM, -2.0 * i1, 1.0, 1.0, 2, 1.0) for _ in range(8)]
    res = _wait(srv, tickets)
    alive, peak, cell_bytes = srv.debug_cells()
    srv.close()
    assert all(r["status"] == 0 for r in res.values())
    assert peak == 1 and cell_bytes == one_cell
    # a budget of two cells admits a second one
    srv = B.Server(labels=lab, params=params, fom_budget_bytes=2 * one_cell, fom_workers=4)
    tickets = [srv.submit(B.REQ_FOM, -2.0 * i1, 1.0, 1.0, 4, 1.0) for _ in range(8)]
    res = _wait(srv, tickets)
    _, peak2, _ = srv.debug_cells()
    srv.close()
    assert all(r["status"] == 0 for r in res.values())
    assert 1 <= peak2 <= 2
