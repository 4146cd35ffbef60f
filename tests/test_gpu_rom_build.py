"""mb_rom_build (GPU snapshots, POD, EI-Greedy, projections) checked against
the full-order oracle: a reduced model whose spaces contain the training
trajectory reproduces it; a truncated one stays close at an unseen parameter
point (not pinned by the paper: a sanity bound)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell as OCell


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


LAB = lambda: syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))


def _seeded(oc):
    u0 = oc.initial_state()
    u0[2 * oc.N::4] = 2e-5
    return u0


def _fom_V(oc, u0, I, s, k, n):
    u = u0.copy()
    V = [oc.functionals(u)["V_cell"]]
    for _ in range(n):
        u, info = oc.step(u, 1.0, I, s, k)
        V.append(info["V_cell"])
    return np.array(V)


@pytest.mark.gpu
def test_built_rom_reproduces_training_trajectory(params):
    B = _gpu()
    lab = LAB()
    oc = OCell(lab, 1e-6, params)
    u0 = _seeded(oc)
    I = -4.0 * oc.i_1c
    gc = B.Cell(lab, 1e-6, params, B.default_opts(newton_tol=1e-12, krylov_rtol=1e-8))
    gc.set_state(u0)
    rom = B.Rom.build(gc, [(I, 1.0, 1.0)], 1.0, 4, (1000, 1000, 1000, 10 ** 6, 10 ** 6), pod_tol=1e-9,
                      ei_tol=1e-14)
    out = rom.solve([(I, 1.0, 1.0)], 4, 1.0)
    assert out["ok"]
    V_ref = _fom_V(oc, u0, I, 1.0, 1.0, 4)
    # the Gram-matrix POD resolves modes down to ~1e-7 of the largest singular value
    assert np.max(np.abs(out["V"][0] - V_ref)) <= 1e-6 * np.max(np.abs(V_ref)), (out["V"][0], V_ref)
    rom.close()
    gc.close()


@pytest.mark.gpu
def test_truncated_rom_near_full_order(params):
    B = _gpu()
    lab = LAB()
    oc = OCell(lab, 1e-6, params)
    u0 = _seeded(oc)
    i1 = oc.i_1c
    gc = B.Cell(lab, 1e-6, params)
    gc.set_state(u0)
    rom = B.Rom.build(gc, [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0)], 1.0, 5, (8, 8, 6, 14, 10))
    assert rom.n_r <= 22 and rom.n_bv <= 14 and rom.n_1c <= 10
    out = rom.solve([(-3.5 * i1, 1.2, 0.5)], 5, 1.0)
    assert out["ok"]
    V_ref = _fom_V(oc, u0, -3.5 * i1, 1.2, 0.5, 5)
    assert np.max(np.abs(out["V"][0] - V_ref)) <= 1e-3 * np.max(np.abs(V_ref))
    rom.close()
    gc.close()


@pytest.mark.gpu
def test_build_pair_is_nested(params):
    """mb_rom_build_pair: the reduced model keeps ceil(0.97 x) of each of the
    validation model's POD blocks and EI bases, from the same snapshots, so its
    basis is the validation basis's leading columns of each block (the nested
    pair the error estimate assumes); the estimate then has no remainder term
    and is small where the two models agree."""
    import math
    B = _gpu()
    lab = LAB()
    oc = OCell(lab, 1e-6, params)
    gc = B.Cell(lab, 1e-6, params)
    gc.set_state(_seeded(oc))
    i1 = oc.i_1c
    snap = [(-2 * i1, 1.0, 1.0), (-5 * i1, 0.7, 3.0)]
    red, val = B.Rom.build_pair(gc, snap, 1.0, 5, (40, 40, 40, 80, 80), frac=0.97, pod_tol=1e-9)
    bv, br = val.block_dims(), red.block_dims()
    assert br == tuple(int(math.ceil(0.97 * x - 1e-9)) for x in bv)
    assert red.n_bv == int(math.ceil(0.97 * val.n_bv - 1e-9)) and red.n_1c == int(math.ceil(0.97 * val.n_1c - 1e-9))
    n = gc.n
    Ur, Uv = red.basis(n), val.basis(n)
    offs_r, offs_v = np.cumsum((0,) + br), np.cumsum((0,) + bv)
    for k in range(3):
        a = Ur[:, offs_r[k]:offs_r[k + 1]]
        b = Uv[:, offs_v[k]:offs_v[k] + br[k]]
        assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1e-300), k
    out = red.estimate(val, [(-3 * i1, 1.1, 0.7)], 3, 1.0)
    assert out["ok"] and np.all(np.isfinite(out["est"]))
    red.close()
    val.close()
    gc.close()
