"""mb_residual_dev_noalloc against mb_residual_dev (gates taken at u_old).

The no-allocation variant runs the same gate and residual kernels with the
gate scratch in static device memory, so the two agree to the last bit; two
calls in a row with different u_old (different gates) check that each call
rewrites the scratch it reads.  This file is collected last so that it also
runs after every other GPU test has used the device."""
import numpy as np
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


def _states(cell, seed):
    """u_old: rest state with plated Li on a seeded subset of faces and a
    seeded potential perturbation (so that some gates open and some stay
    closed); u: u_old plus a small seeded perturbation of every unknown."""
    rng = syn.SplitMix64(seed)
    u_old = cell.state().copy()
    N, F = cell.N, cell.F
    n = len(u_old)
    for f in range(F):
        if rng.uniform() < 0.3:
            u_old[2 * N + f] = 4e-5 * rng.uniform()
    for i in range(N, 2 * N):
        u_old[i] += 2e-3 * (rng.uniform() - 0.5)
    u = u_old.copy()
    for i in range(n):
        u[i] += 1e-4 * (rng.uniform() - 0.5) * max(abs(u_old[i]), 1e-6)
    return u, u_old


@pytest.mark.gpu
def test_noalloc_residual_matches_residual_dev(params):
    import torch
    B = _gpu()
    lab = syn.full_cell(5, 7, 9, 4, 8, 0.35, 0.35, ("uniform", 1.5, 3), (3, 4))
    cell = B.Cell(lab, 1e-6, params, B.default_opts())
    assert cell.F > 0
    dt, I_app = 0.5, -2.0 * cell.i_1c
    for call, seed in enumerate((101, 202)):
        u, u_old = _states(cell, seed)
        du = torch.tensor(u, device="cuda")
        duo = torch.tensor(u_old, device="cuda")
        r_ref = torch.full_like(du, float("nan"))
        r = torch.full_like(du, float("nan"))
        cell.residual_dev(du, duo, dt, I_app, r_ref)
        cell.residual_dev_noalloc(du, duo, dt, I_app, r)
        a, b = r.cpu().numpy(), r_ref.cpu().numpy()
        assert np.all(np.isfinite(b)), call
        # same kernels, same inputs, same summation order: bit-identical
        assert np.array_equal(a, b), (call, float(np.max(np.abs(a - b))))
    cell.close()


@pytest.mark.gpu
def test_noalloc_residual_rejects_invalid_arguments(params):
    import torch
    B = _gpu()
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    cell = B.Cell(lab, 1e-6, params, B.default_opts())
    du = torch.tensor(cell.state(), device="cuda")
    r = torch.empty_like(du)
    with pytest.raises(B.MBError):
        cell.residual_dev_noalloc(du, du, 0.0, 0.0, r)
    cell.close()


@pytest.mark.gpu
def test_noalloc_residual_rejects_another_device(params):
    """A call made while another device is current is refused: the scratch
    address and the launches would belong to a device that does not hold the
    cell's buffers.  Needs two devices."""
    import torch
    B = _gpu()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    torch.cuda.set_device(0)
    cell = B.Cell(lab, 1e-6, params, B.default_opts())
    du = torch.tensor(cell.state(), device="cuda:0")
    r = torch.empty_like(du)
    torch.cuda.set_device(1)
    try:
        with pytest.raises(B.MBError):
            cell.residual_dev_noalloc(du, du, 1.0, 0.0, r)
    finally:
        torch.cuda.set_device(0)
    cell.close()
