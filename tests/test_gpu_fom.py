"""Parity of the CUDA full-order path (through the C-ABI) with the FP64 oracle.

Tolerances.  The residual and the JVP are compared row by row against a
rounding bound: |x_gpu - x_oracle|_i <= C eps (|J| |y|)_i, where y is the
state (residual) or the direction (JVP) and |J| the element-wise absolute
oracle Jacobian, i.e. a multiple of the rounding error of the row's terms.
FP64: C = 256, eps = 2^-52.  FP32 JVP: the linearisation point itself is
rounded to FP32, which perturbs exp/sinh arguments of size F/(2RT)*|Phi| ~ 70
by ~70*2^-24, so C*eps = 2e-4.  Full steps (FP64 path) agree with the oracle to
1e-9 relative per field (max-norm) and on the cell voltage.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell as OCell

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_04139_gb300 import binding, build
    import os
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding


GEOMS = {
    "tiny": lambda: syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2)),
    "ragged": lambda: syn.full_cell(5, 7, 9, 4, 8, 0.35, 0.35, ("uniform", 1.5, 3), (3, 4)),
    "wide": lambda: syn.full_cell(37, 40, 3, 2, 3, 0.35, 0.35, ("uniform", 1, 3), (5, 6)),
    "half": lambda: syn.half_cell(6, 5, 8, 4, 3, 0.35, ("uniform", 1.5, 3), 7),
}


def _perturbed_state(oc, seed):
    rng = np.random.default_rng(seed)
    u0 = oc.initial_state()
    N = oc.N
    u = u0.copy()
    u[:N] *= 1.0 + 0.05 * rng.standard_normal(N)
    u[N:2 * N] += 0.01 * rng.standard_normal(N)
    u[2 * N:] = 6e-5 * rng.random(oc.F_pl) * (rng.random(oc.F_pl) < 0.6)
    gate = (rng.random(oc.F_pl) < 0.5).astype(np.uint8)
    return u0, u, gate


@pytest.mark.parametrize("geom", list(GEOMS))
def test_face_list_and_rest_state_match(params, geom):
    B = _gpu()
    lab = GEOMS[geom]()
    oc = OCell(lab, 1e-6, params)
    gc = B.Cell(lab, 1e-6, params)
    assert gc.F == oc.F_pl and gc.N == oc.N
    g, e, d = gc.plating_faces()
    assert np.array_equal(g, oc.pf_g) and np.array_equal(e, oc.pf_e) and np.array_equal(d, oc.pf_dir)
    u0g = gc.state()
    u0o = oc.initial_state()
    assert np.max(np.abs(u0g - u0o) / oc.unknown_scale()) < 1e-15
    assert abs(gc.i_1c - oc.i_1c) <= 1e-14 * oc.i_1c


@pytest.mark.parametrize("geom", list(GEOMS))
def test_residual_parity(params, geom):
    B = _gpu()
    lab = GEOMS[geom]()
    oc = OCell(lab, 1e-6, params)
    gc = B.Cell(lab, 1e-6, params)
    for seed, (s_i0, k_pl) in enumerate([(1.0, 1.0), (0.7, 3.0)]):
        u_old, u, gate = _perturbed_state(oc, seed)
        gc.set_scales(s_i0, k_pl)
        dt, I = 0.5, -2.5 * oc.i_1c
        r_o = oc.residual(u, u_old, dt, I, gate.astype(float), s_i0, k_pl)
        J = abs(oc.jacobian(u, u_old, dt, I, gate.astype(float), s_i0, k_pl))
        bound = 256 * EPS * (J @ np.abs(u) + np.abs(r_o)) + 1e-300
        # the C-ABI residual and the solver's two-pass Newton residual
        for r_g in (gc.residual(u, u_old, dt, I, gate), gc.debug_residual_split(u, u_old, dt, I, gate)):
            bad = np.abs(r_g - r_o) > bound
            assert not bad.any(), (np.nonzero(bad)[0][:10], (np.abs(r_g - r_o) / bound).max())


@pytest.mark.parametrize("geom", list(GEOMS))
def test_jvp_parity_fp64_and_fp32(params, geom):
    import torch
    B = _gpu()
    lab = GEOMS[geom]()
    oc = OCell(lab, 1e-6, params)
    gc = B.Cell(lab, 1e-6, params)
    rng = np.random.default_rng(11)
    u_old, u, gate = _perturbed_state(oc, 5)
    dt = 0.25
    J = oc.jacobian(u, u_old, dt, 0.0, gate.astype(float))
    Ja = abs(J)
    for trial in range(2):
        v = oc.unknown_scale() * rng.standard_normal(oc.n_unknowns)
        jv_o = J @ v
        jv_g = gc.jvp(u, v, dt, gate)
        bound = 256 * EPS * (Ja @ np.abs(v)) + 1e-300
        assert np.all(np.abs(jv_g - jv_o) <= bound), (np.abs(jv_g - jv_o) / bound).max()
        # FP32 operator through the device-pointer entry point
        dev = torch.device("cuda")
        u32 = torch.tensor(u, dtype=torch.float32, device=dev)
        v32 = torch.tensor(v, dtype=torch.float32, device=dev)
        out = torch.empty_like(u32)
        g = torch.tensor(gate, dtype=torch.uint8, device=dev)
        gc.jvp_f32_dev(u32, v32, dt, out, g)
        jv32 = out.double().cpu().numpy()
        bound32 = 2e-4 * (Ja @ np.abs(v)) + 1e-300
        assert np.all(np.abs(jv32 - jv_o) <= bound32), (np.abs(jv32 - jv_o) / bound32).max()


def _fields_rel(a, b, oc):
    N = oc.N
    out = {}
    for name, sl in (("c", slice(0, N)), ("phi", slice(N, 2 * N)), ("n", slice(2 * N, None))):
        ref = b[sl]
        if ref.size == 0:
            continue
        out[name] = float(np.max(np.abs(a[sl] - ref)) / max(np.max(np.abs(ref)), 1e-30))
    return out


@pytest.mark.parametrize("geom,precision,tol", [("tiny", 0, 1e-9), ("ragged", 0, 1e-9),
                                                ("half", 0, 1e-9), ("tiny", 1, 1e-6)])
def test_step_parity(params, geom, precision, tol):
    """Several implicit Euler steps at a charge current with seeded plated Li:
    the GPU Newton-Krylov step and the oracle's sparse direct Newton step
    reach the same discrete solution."""
    B = _gpu()
    lab = GEOMS[geom]()
    oc = OCell(lab, 1e-6, params)
    opts = B.default_opts(precision=precision, newton_tol=1e-12 if precision == 0 else 1e-10,
                          krylov_rtol=1e-6 if precision == 0 else 1e-4)
    gc = B.Cell(lab, 1e-6, params, opts)
    u = oc.initial_state()
    u[2 * oc.N::3] = 4e-5
    gc.set_state(u)
    uo = u.copy()
    for k, I in enumerate([-3.0 * oc.i_1c, -3.0 * oc.i_1c, 2.0 * oc.i_1c]):
        info = gc.step(1.0, I)
        uo, oinfo = oc.step(uo, 1.0, I)
        ug = gc.state()
        rel = _fields_rel(ug, uo, oc)
        assert all(v <= tol for v in rel.values()), (k, rel, info)
        assert abs(info["V_cell"] - oinfo["V_cell"]) <= tol * abs(oinfo["V_cell"])
        assert abs(info["Li_total"] - oinfo["Li_total"]) <= 1e-12 * oinfo["Li_total"]
        assert info["passes"] == oinfo["passes"] and info["unresolved_flips"] == oinfo["unresolved_flips"], k
