"""Pins of the full-order oracle against closed forms and invariants of the
paper's equations (Sec. 2.2-2.4).  CPU only."""
import copy
import math

import numpy as np
import pytest

import synthetic as syn
from synthetic import E, G, K, L, CN, CP
from oracle.fom import Cell, GeometryError, ocp


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------- T1 diffusion
def test_T1_solid_diffusion_discrete_cosine_mode(params):
    """Eq. (cgr) with zero-flux ends (graphite next to a collector carries
    N = 0, Table interfaceCond): the cosine mode decays by exactly
    1/(1 + 4 D dt/h^2 sin^2(pi/(2N))) per implicit Euler step."""
    n, h, dt = 10, 1e-7, 1.0
    cell = Cell(syn.slab_1d([CN] + [G] * n + [CN]), h, params)
    D, cmax = params["G"]["D"], params["G"]["cmax"]
    k = np.arange(n)
    mode = np.cos(math.pi * (k + 0.5) / n)
    u = cell.initial_state()
    cbar, a = 0.5 * cmax, 0.1 * cmax
    u[1:1 + n] = cbar + a * mode
    lam = 1.0 + 4.0 * D * dt / h ** 2 * math.sin(math.pi / (2 * n)) ** 2
    for step in range(1, 4):
        u, _ = cell.step(u, dt, 0.0)
        expect = cbar + a * mode * lam ** (-step)
        assert _rel(u[1:1 + n], expect) < 1e-13
    # no current anywhere: potentials stay at the Dirichlet value
    assert np.max(np.abs(u[cell.N:2 * cell.N])) < 1e-14


def test_T1_electrolyte_diffusion_zero_current(params):
    """Eqs. (cel, phiel) in a Li|E|Li stack at zero current: j = 0 on every
    face, so N = -D_E grad c exactly and the cosine mode decays at the
    discrete rate with D_E; the potential balances migration,
    kappa dphi = -kappa (t+ - 1)(RT/F) dc/cbar."""
    n, h, dt = 8, 1e-6, 0.01
    cell = Cell(syn.slab_1d([CN, L] + [E] * n + [L, CP]), h, params)
    D = params["E"]["D"]
    k = np.arange(n)
    mode = np.cos(math.pi * (k + 0.5) / n)
    u = cell.initial_state()
    u[cell.N:2 * cell.N] = 0.0
    u[2:2 + n] = 1000.0 + 100.0 * mode
    lam = 1.0 + 4.0 * D * dt / h ** 2 * math.sin(math.pi / (2 * n)) ** 2
    for step in range(1, 3):
        u, _ = cell.step(u, dt, 0.0)
        assert _rel(u[2:2 + n], 1000.0 + 100.0 * mode * lam ** (-step)) < 1e-12
    c = u[2:2 + n]; phi = u[cell.N + 2:cell.N + 2 + n]
    tp = params["E"]["tplus"]; RT_F = params["R"] * params["T"] / params["F"]
    dphi_expect = -(tp - 1.0) * RT_F * np.diff(c) / (0.5 * (c[1:] + c[:-1]))
    assert np.max(np.abs(np.diff(phi) - dphi_expect)) < 1e-13


# ---------------------------------------------------------------- T2 ohmic
def test_T2_ohmic_chain_closed_form(params):
    """Eq. (phigr) in conductors with harmonic face conductivity (Table
    interfaceCond 'j cont.'), Dirichlet Phi=0 half a voxel outside t=0 and a
    uniform current I out of the last face: Phi(CP) = -I h (1/(2 s_CN) +
    sum_f 1/s_f)."""
    p = copy.deepcopy(params)
    p["L"]["sigma"] = 3.0e3
    h, I = 1e-6, 7.5
    cell = Cell(syn.slab_1d([CN, L, L, L, CP], ny=2, nz=3), h, p)
    u = cell.initial_state()
    u, _ = cell.step(u, 1.0, I)
    sc, sl, sp_ = p["CN"]["sigma"], p["L"]["sigma"], p["CP"]["sigma"]
    hm = lambda a, b: 2 * a * b / (a + b)
    V = -I * h * (1 / (2 * sc) + 1 / hm(sc, sl) + 2 / sl + 1 / hm(sl, sp_))
    info = cell.functionals(u)
    assert abs(info["V_cell"] - V) / abs(V) < 1e-12


# ---------------------------------------------------------------- T3 rest
def test_T3_rest_state_is_stationary(params):
    """At zero current the equilibrium state (all overpotentials zero, uniform
    concentrations) solves Eq. (ap4:detailed): R(u0) = 0 to rounding and a
    step returns u0."""
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    cell = Cell(lab, 1e-6, params)
    u0 = cell.initial_state()
    gate = cell.gate_at(u0, u0[2 * cell.N:])
    assert not gate.any()
    R = cell.residual(u0, u0, 1.0, 0.0, gate)
    assert np.max(np.abs(R) / cell.residual_scale(1.0)) < 1e-12
    u1, info = cell.step(u0, 1.0, 0.0)
    assert np.max(np.abs(u1 - u0) / cell.unknown_scale()) < 1e-13


# ---------------------------------------------------------------- T4 Li|E|Li
def test_T4_symmetric_lithium_cell_steady_state(params):
    """Li|E|Li at current I: the steady state has a linear concentration
    profile with slope -(1 - t+) I/(F D_E) (Sec. 3.1: a linear gradient forms
    without sources), counter-electrode overpotentials (2RT/F) asinh(I/(2
    i00)) of opposite sign (Eq. ise_li), and the potential drop of Eq. (phiel).
    The constructed state has zero residual."""
    n, h, I = 6, 1e-6, 4.0
    cell = Cell(syn.slab_1d([CN, L] + [E] * n + [L, CP]), h, params)
    p = params
    F, RT = p["F"], p["R"] * p["T"]
    tp, D, kap = p["E"]["tplus"], p["E"]["D"], p["E"]["kappa"]
    sC, sL = p["CN"]["sigma"], p["L"]["sigma"]
    hm = 2 * sC * sL / (sC + sL)
    dc = -(1 - tp) * I * h / (F * D)
    c = 1000.0 + (np.arange(n) - (n - 1) / 2) * dc
    eta = 2 * RT / F * math.asinh(I / (2 * p["L"]["i00"]))
    phi = np.zeros(cell.N)
    phi[0] = -I * h / (2 * sC)
    phi[1] = phi[0] - I * h / hm
    pe = [phi[1] - eta]
    for k in range(n - 1):
        cb = 0.5 * (c[k] + c[k + 1])
        pe.append(pe[-1] - I * h / kap - (tp - 1) * RT / F * (c[k + 1] - c[k]) / cb)
    phi[2:2 + n] = pe
    phi[2 + n] = pe[-1] - eta
    phi[3 + n] = phi[2 + n] - I * h / hm
    u = np.zeros(cell.n_unknowns)
    u[2:2 + n] = c
    u[cell.N:2 * cell.N] = phi
    R = cell.residual(u, u, 1.0, I, np.zeros(0))
    # rounding floor of a potential row: eps * (largest face conductance) * |Phi|
    floor = 64 * np.finfo(float).eps * max(sC, sL) * h * np.max(np.abs(phi))
    Rc, Rp = R[:cell.N], R[cell.N:2 * cell.N]
    assert np.max(np.abs(Rc) / cell.residual_scale(1.0)[:cell.N]) < 1e-12
    assert np.max(np.abs(Rp)) < floor
    # and Newton from a perturbed guess lands on it
    u_old = u.copy()
    guess = u.copy(); guess[cell.N:2 * cell.N] += 0.01
    un, it, ok = cell.newton(guess, u_old, 1.0, I, np.zeros(0))
    assert ok and np.max(np.abs(un - u) / cell.unknown_scale()) < 1e-10


# ---------------------------------------------------------------- T5 BV
@pytest.mark.parametrize("I", [0.05, 3.0, -2.0])
def test_T5_butler_volmer_single_face(params, I):
    """Eq. (ise_gr) on one graphite-electrolyte face in a 1-D stack: at any
    converged state the face carries the whole current I, so
    eta = (2RT/F) asinh(I / (2 i00 sqrt(c_G c_E))); for small I this tends to
    the linearisation RT I/(F i00 sqrt(c_G c_E))."""
    cell = Cell(syn.slab_1d([CN, G, G, E, E, E, L, CP]), 1e-6, params)
    p = params
    u, _ = cell.step(cell.initial_state(), 1.0, I)
    c, phi = u[:cell.N], u[cell.N:2 * cell.N]
    g, e = 2, 3
    RT_F = p["R"] * p["T"] / p["F"]
    i0 = p["G"]["i00"] * math.sqrt(c[g] * c[e])
    eta = phi[g] - ocp(c[g] / p["G"]["cmax"], p["G"]["ocp"]) - phi[e]
    assert abs(eta - 2 * RT_F * math.asinh(I / (2 * i0))) < 1e-12
    if abs(I) < 0.1:
        lin = RT_F * I / i0
        x = I / (2 * i0)
        assert abs(eta - lin) / abs(lin) < x * x


# ---------------------------------------------------------------- T6 plating
@pytest.mark.parametrize("n_plated", [1e-5, 3.69e-5, 2e-4])
def test_T6_plating_equilibrium(params, n_plated):
    """Eq. (iplel) with intercalation switched off (exchange-current scale 0)
    and no applied current: the plated face carries no current, so
    f_pre(n) e^{F eta/2RT} = e^{-F eta/2RT}, i.e. eta = -(RT/F) ln f_pre(n),
    and n does not change."""
    cell = Cell(syn.slab_1d([CN, G, E, E, L, CP]), 1e-6, params)
    assert cell.F_pl == 1
    u = cell.initial_state()
    u[-1] = n_plated
    u1, info = cell.step(u, 1.0, 0.0, s_i0=0.0)
    nc = cell.nc
    fpre = n_plated ** 4 / (nc ** 4 + n_plated ** 4)
    RT_F = params["R"] * params["T"] / params["F"]
    phi = u1[cell.N:2 * cell.N]
    assert abs((phi[1] - phi[2]) - (-RT_F * math.log(fpre))) < 1e-12
    assert abs(u1[-1] - n_plated) / n_plated < 1e-13


# ---------------------------------------------------------------- T7 Li conservation
def test_T7_lithium_conservation_with_plating(params):
    """Sec. 2.4: the finite-volume scheme is conservative.  In a full cell the
    total Li (solid + electrolyte + plated) is constant, and the anode
    inventory (graphite + plated) changes by -dt A_cross I / F per step."""
    lab = syn.full_cell(4, 4, 6, 3, 6, 0.35, 0.35, ("uniform", 1, 2), (5, 6))
    cell = Cell(lab, 1e-6, params)
    u = cell.initial_state()
    u[2 * cell.N::2] = 5e-5            # seeded plated Li on every other face
    A_cross = 4 * 4 * cell.A
    f0 = cell.functionals(u)
    for I in (3 * cell.i_1c, -4 * cell.i_1c):
        u_prev = cell.functionals(u)
        u, info = cell.step(u, 1.0, I)
        assert abs(info["Li_total"] - f0["Li_total"]) / f0["Li_total"] < 1e-13
        d_anode = info["Li_anode"] - u_prev["Li_anode"]
        expect = -1.0 * A_cross * I / params["F"]
        assert abs(d_anode - expect) / abs(expect) < 1e-9
    assert info["Li_plated"] > 0


# ---------------------------------------------------------------- T8 Jacobian
def test_T8_jacobian_complex_step_vs_directional_and_fd(params):
    """The coloured complex-step Jacobian equals directional complex-step
    derivatives to rounding and central differences to truncation error, on a
    grid with all phases and active plating."""
    lab = syn.full_cell(4, 4, 5, 3, 4, 0.35, 0.35, ("uniform", 1, 2), (3, 4))
    cell = Cell(lab, 1e-6, params)
    rng = np.random.default_rng(8)
    u0 = cell.initial_state()
    us = cell.unknown_scale()
    u = u0 + 1e-3 * us * rng.standard_normal(cell.n_unknowns) * (u0 != 0)
    u[2 * cell.N:] = 4e-5 * rng.random(cell.F_pl)
    gate = np.ones(cell.F_pl)
    args = (u0, 1.0, -2.0 * cell.i_1c, gate)
    J = cell.jacobian(u, *args)
    rs = cell.residual_scale(1.0)
    for trial in range(3):
        v = us * rng.standard_normal(cell.n_unknowns)
        hcs = 1e-20
        jv_cs = cell.residual(u + 1j * hcs * v, *args).imag / hcs
        assert np.max(np.abs(J @ v - jv_cs) / rs) <= 1e-12 * np.max(np.abs(jv_cs) / rs)
        eps = 1e-6
        jv_fd = (cell.residual(u + eps * v, *args) - cell.residual(u - eps * v, *args)) / (2 * eps)
        assert np.max(np.abs(J @ v - jv_fd) / rs) <= 1e-6 * np.max(np.abs(jv_cs) / rs)


# ---------------------------------------------------------------- T9 affine
def test_T9_residual_affine_in_current(params):
    """Eq. (ap4:operator_subdecomposition): the current enters affinely,
    R(u; mu) - R(u; 0) = mu b_bnd with b_bnd = A on the potential rows of the
    collector voxels at the outer CP face."""
    lab = syn.full_cell(3, 4, 4, 2, 4, 0.35, 0.35, ("uniform", 1, 2), (7, 8))
    cell = Cell(lab, 1e-6, params)
    rng = np.random.default_rng(9)
    u = cell.initial_state() * (1 + 1e-3 * rng.standard_normal(cell.n_unknowns))
    gate = np.zeros(cell.F_pl)
    mu = 12.5
    R0 = cell.residual(u, u, 1.0, 0.0, gate)
    d = cell.residual(u, u, 1.0, mu, gate) - R0
    b = np.zeros(cell.n_unknowns)
    b[cell.N + cell.bc_neu] = cell.A
    # exact up to the rounding of adding mu*b to each row's other terms
    eps = np.finfo(float).eps
    assert np.all(np.abs(d - mu * b) <= 2 * eps * (np.abs(R0) + np.abs(mu * b)))


# ---------------------------------------------------------------- T10 symmetry
def test_T10_mirror_symmetry(params):
    """A label grid mirror-symmetric in y gives mirror-symmetric fields."""
    lab = syn.full_cell(3, 3, 5, 2, 5, 0.35, 0.35, ("uniform", 1, 2), (9, 10))
    lab = np.concatenate([lab, lab[:, ::-1, :]], axis=1)
    cell = Cell(lab, 1e-6, params)
    u, _ = cell.step(cell.initial_state(), 1.0, -3 * cell.i_1c)
    N = cell.N
    for fld in (u[:N], u[N:2 * N]):
        f = fld.reshape(cell.shape)
        assert np.max(np.abs(f - f[:, ::-1, :])) <= 1e-11 * max(1.0, np.max(np.abs(f)))


# ---------------------------------------------------------------- geometry
def test_forbidden_contacts_rejected(params):
    """Graphite touching cathode material is a short circuit (not a pair of
    Table interfaceCond) and is rejected."""
    with pytest.raises(GeometryError):
        Cell(syn.slab_1d([CN, G, K, CP]), 1e-6, params)


def test_plating_face_order(params):
    """Plating faces are every G-E face, ordered by the graphite voxel's linear
    index, then by direction (-t, +t, -y, +y, -z, +z)."""
    lab = np.full((3, 3, 3), E, np.uint8)
    lab[1, 1, 1] = G
    lab[0, 1, 1] = G
    cell = Cell(lab, 1e-6, params)
    g = cell.pf_g; d = cell.pf_dir
    assert list(zip(g.tolist(), d.tolist())) == (
        [(4, 2), (4, 3), (4, 4), (4, 5)] + [(13, 1), (13, 2), (13, 3), (13, 4), (13, 5)])
