"""Pins of the reduced-order model oracle (CPU): each checks it against
something other than itself (the full-order oracle's residual and
trajectories, the interpolation property, the rest state)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.fom import Cell
from oracle import rom as R


@pytest.fixture(scope="module")
def tiny(params):
    lab = syn.full_cell(4, 4, 5, 3, 5, 0.35, 0.35, ("uniform", 1, 2), (1, 2))
    return Cell(lab, 1e-6, params)


def _state(cell, seed):
    rng = np.random.default_rng(seed)
    u = cell.initial_state()
    N = cell.N
    u[:N] *= 1.0 + 0.02 * rng.standard_normal(N)
    u[N:2 * N] += 0.004 * rng.standard_normal(N)
    u[2 * N:] = 3e-5 * (rng.random(cell.F_pl) < 0.5)
    gate = (rng.random(cell.F_pl) < 0.6).astype(float)
    return u, gate


def test_split_reproduces_full_order_residual(tiny):
    """storage + A_lin + mu A_bnd + A_1c + s A_bv + A_ce + k A_pl = R (Eqs.
    ap4:operator_decomposition and ap4:operator_subdecomposition)."""
    cell = tiny
    for seed in range(3):
        u, gate = _state(cell, seed)
        u_old, _ = _state(cell, seed + 10)
        dt, mu, s, k = 0.7, -2.0 * cell.i_1c, 1.3, 0.4
        r_full = cell.residual(u, u_old, dt, mu, gate, s, k)
        r_split = R.full_residual_from_split(cell, u, u_old, dt, mu, gate, s, k)
        scale = np.abs(cell.jacobian(u, u_old, dt, mu, gate, s, k)) @ np.abs(u) + np.abs(r_full)
        assert np.all(np.abs(r_split - r_full) <= 64 * np.finfo(float).eps * scale + 1e-300)


def test_boundary_term_is_the_current_derivative(tiny):
    """A_bnd equals dR/dmu of the full-order residual (finite difference in mu
    of an affine function is exact up to rounding)."""
    cell = tiny
    u, gate = _state(cell, 4)
    r1 = cell.residual(u, u, 1.0, 5.0, gate)
    r0 = cell.residual(u, u, 1.0, 0.0, gate)
    bnd = R.suboperators(cell, u, gate)["bnd"]
    tol = 16 * np.finfo(float).eps * (np.abs(r1) + np.abs(r0)) / 5.0
    assert np.all(np.abs((r1 - r0) / 5.0 - bnd) <= tol + 1e-15 * np.max(np.abs(bnd)))
    assert np.count_nonzero(bnd) == len(cell.bc_neu) > 0


@pytest.fixture(scope="module")
def trained(tiny):
    cell = tiny
    mu = -4.0 * cell.i_1c
    u0 = cell.initial_state()
    u0[2 * cell.N::4] = 2e-5          # seeded plated Li on every fourth face
    snaps, trajs = R.snapshots(cell, [(mu, 1.0, 1.0)], 1.0, 4, u0=u0)
    rom = R.build(cell, snaps, (10 ** 6, 10 ** 6, 10 ** 6, 10 ** 6), pod_tol=1e-15, ei_tol=1e-14)
    return cell, mu, snaps, trajs[0], rom


def test_ei_interpolation_identity(trained):
    """I_M[O](x) agrees with O(x) at the interpolation points (Sec.
    workflow:MOR) for states outside the training set."""
    cell, mu, snaps, traj, rom = trained
    for seed in range(2):
        u, gate = _state(cell, 20 + seed)
        so = R.suboperators(cell, u, gate)
        for key, (Q, P) in (("bv", (rom.Qbv, rom.Pbv)), ("pl", (rom.Qbv, rom.Pbv)),
                            ("c1", (rom.Q1c, rom.P1c))):
            if len(P) == 0:
                continue
            vals = so[key][P]
            interp = R.ei_interpolate(Q, P, vals)
            assert np.allclose(interp[P], vals, rtol=1e-9, atol=1e-12 * np.max(np.abs(so[key])))


def test_full_basis_rom_reproduces_the_training_trajectory(trained):
    """With bases spanning every snapshot and EI spaces spanning every training
    evaluation, the full-order states solve the fully reduced model (Eq.
    ap4:fully_reduced): the reduced trajectory is the full-order one, up to
    the two Newton solves' tolerance carried through the time steps (the
    deviation enters at ~3e-10 per step in the graphite concentration of this
    23-snapshot model and accumulates over the 4 steps; the bound is 1e-8)."""
    cell, mu, snaps, traj, rom = trained
    # start the reduced model from the seeded state the full-order run started from
    rom.a0 = rom.U.T @ (R.weights(cell) * traj[0])
    out = R.solve(rom, mu, 1.0, 1.0, 1.0, len(traj) - 1)
    for n in range(len(traj)):
        fom = cell.functionals(traj[n])
        assert abs(out["V_cell"][n] - fom["V_cell"]) <= 1e-9 * abs(fom["V_cell"]), n
        assert abs(out["s_ac"][n] - fom["mean_c_solid"]) <= 1e-8 * abs(fom["mean_c_solid"]), n
        u_rom = rom.U @ out["a"][n]
        for sl, tol in ((slice(0, cell.N), 1e-8), (slice(cell.N, 2 * cell.N), 1e-9),
                        (slice(2 * cell.N, None), 1e-8)):
            ref = traj[n][sl]
            assert np.max(np.abs(u_rom[sl] - ref)) <= tol * np.max(np.abs(traj[:, sl])), n


def test_rest_state_is_stationary(tiny):
    """At zero current from the rest state the reduced model stays at rest."""
    cell = tiny
    snaps, trajs = R.snapshots(cell, [(-3.0 * cell.i_1c, 1.0, 1.0)], 1.0, 2)
    rom = R.build(cell, snaps, (10 ** 6, 10 ** 6, 10 ** 6, 10 ** 6), pod_tol=1e-15, ei_tol=1e-14)
    out = R.solve(rom, 0.0, 1.0, 1.0, 1.0, 3)
    assert np.max(np.abs(out["V_cell"] - out["V_cell"][0])) <= 1e-12 * abs(out["V_cell"][0])
    assert np.max(np.abs(out["a"] - out["a"][0])) <= 1e-10 * np.max(np.abs(out["a"][0]))


def test_pod_bases_are_w_orthonormal(trained):
    cell, mu, snaps, traj, rom = trained
    w = R.weights(cell)
    G = rom.U.T @ (w[:, None] * rom.U)
    assert np.allclose(G, np.eye(G.shape[0]), atol=1e-10)


def test_error_estimate_norm_of_a_constant_field(tiny):
    """The estimate's norm is the L^2 norm of the voxel grid: two models whose
    reconstructions differ by a constant delta in one field give delta times the
    square root of that field's measure (N V for c and phi, F A for the plated Li)
    in that field and zero in the others, scaled by 1/(1 - theta) (Eq. ap4:estimate)."""
    cell = tiny
    N, F = cell.N, cell.F_pl
    n = cell.n_unknowns

    class M:
        pass

    zero = M()
    zero.cell, zero.U = cell, np.zeros((n, 1))
    for name, sl, measure in (("c", slice(0, N), N * cell.V), ("phi", slice(N, 2 * N), N * cell.V),
                              ("n", slice(2 * N, n), F * cell.A)):
        ind = M()
        ind.cell = cell
        ind.U = np.zeros((n, 1))
        ind.U[sl, 0] = 1.0
        delta = np.array([[0.0], [2.5], [-7.0]])
        for theta in (0.0, 0.5, 0.9):
            est = R.error_estimate(zero, ind, np.zeros((3, 1)), delta, theta)
            expect = np.abs(delta[:, 0]) * np.sqrt(measure) / (1.0 - theta)
            assert np.allclose(est[name], expect, rtol=1e-14, atol=0.0), (name, theta)
            for other in {"c", "phi", "n"} - {name}:
                assert np.all(est[other] == 0.0)
    with pytest.raises(ValueError):
        R.error_estimate(zero, zero, np.zeros((1, 1)), np.zeros((1, 1)), 1.0)


def test_error_estimate_is_the_error_for_an_exact_validation_model(trained):
    """With theta = 0 and a validation model that reproduces the full-order
    trajectory (bases and EI spaces spanning it), the estimate is the reduced
    model's true error up to the validation model's own error: by the triangle
    inequality | ||c~ - c^|| - ||c~ - c|| | <= ||c^ - c|| (Eq. ap4:estimate with
    its saturation assumption met); identical models estimate zero."""
    cell, mu, snaps, traj, full = trained
    w = R.weights(cell)
    N = cell.N
    full.a0 = full.U.T @ (w * traj[0])
    of = R.solve(full, mu, 1.0, 1.0, 1.0, len(traj) - 1)
    small = R.build(cell, snaps, (4, 3, 8, 8), pod_tol=1e-15, ei_tol=1e-14)
    small.a0 = small.U.T @ (w * traj[0])
    os_ = R.solve(small, mu, 1.0, 1.0, 1.0, len(traj) - 1)
    est = R.error_estimate(small, full, os_["a"], of["a"])

    def dist(u, v, sl):
        d = (u - v)[sl]
        return float(np.sqrt(np.dot(w[sl] * d, d)))

    for n in range(len(traj)):
        u_s, u_v = small.U @ os_["a"][n], full.U @ of["a"][n]
        for key, sl in (("c", slice(0, N)), ("phi", slice(N, 2 * N))):
            true = dist(u_s, traj[n], sl)
            val = dist(u_v, traj[n], sl)
            assert abs(est[key][n] - true) <= val + 1e-14 * dist(traj[n], 0 * traj[n], sl), (key, n)
    # a real truncation error, far above the validation model's
    assert np.all(est["c"][1:] > 1e3 * max(dist(full.U @ of["a"][n], traj[n], slice(0, N))
                                           for n in range(len(traj))))
    same = R.error_estimate(small, small, os_["a"], os_["a"])
    assert all(np.all(v == 0.0) for v in same.values())


def test_dt_halving_retakes_failed_steps(trained, monkeypatch):
    """A failed step is retaken from the state before it as 2^h steps of
    dt / 2^h, h = 1 .. max_halvings.  The failure is planted on the host: the
    step raises for dt > 0.3, so the solve must settle at h = 2 and equal four
    direct steps of 0.25 (a wrong restart state, dt or substep count breaks the
    equality), and with max_halvings = 1 it must fail."""
    cell, mu, snaps, traj, rom = trained
    real = R._step
    calls = []

    def flaky(rom_, a_old, mu_, s_i0, k_pl, dt, tol, maxit):
        calls.append(dt)
        if dt > 0.3:
            raise R._NoConvergence("planted")
        return real(rom_, a_old, mu_, s_i0, k_pl, dt, tol, maxit)

    direct = R.solve(rom, mu, 1.0, 1.0, 0.25, 4)
    monkeypatch.setattr(R, "_step", flaky)
    out = R.solve(rom, mu, 1.0, 1.0, 1.0, 1, max_halvings=3)
    assert calls == [1.0, 0.5, 0.25, 0.25, 0.25, 0.25]
    assert np.array_equal(out["a"][-1], direct["a"][-1])
    assert out["newton_its"] == direct["newton_its"]
    with pytest.raises(RuntimeError):
        R.solve(rom, mu, 1.0, 1.0, 1.0, 1, max_halvings=1)


def _jacobian_fd_error(rom, cell, traj, mu):
    """Largest relative difference between the reduced Jacobian's products and
    central differences of the reduced residual (step 1e-5 in each mode's own
    scale), over two (s_i0, k_pl) pairs and three directions."""
    w = R.weights(cell)
    a_old = rom.U.T @ (w * traj[1])
    a = rom.U.T @ (w * traj[2])
    u_old = rom.U @ a_old
    gate = cell.gate_at(u_old, u_old[2 * cell.N:])
    assert np.count_nonzero(gate) > 0            # the plating terms take part
    rng = np.random.default_rng(7)
    h, dt = 1e-5, 0.1
    worst = 0.0
    for s_i0, k_pl in ((1.0, 1.0), (1.7, 0.3)):
        J = R.reduced_jacobian(rom, a, dt, s_i0, k_pl, gate)
        for _ in range(3):
            v = rng.standard_normal(len(a)) * np.maximum(np.abs(a), 1e-6 * np.max(np.abs(a)))
            rp = R.reduced_residual(rom, a + h * v, a_old, dt, mu, s_i0, k_pl, gate)
            rm = R.reduced_residual(rom, a - h * v, a_old, dt, mu, s_i0, k_pl, gate)
            jv = J @ v
            worst = max(worst, float(np.max(np.abs((rp - rm) / (2 * h) - jv)) / np.max(np.abs(jv))))
    return worst


def _mutated(fn, old, new):
    """fn recompiled from its source with one planted change (in its module's namespace)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(fn))
    assert old in src
    ns = dict(fn.__globals__)
    exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    return ns[fn.__name__]


def test_reduced_jacobian_is_the_residual_derivative(trained, monkeypatch):
    """The reduced Newton matrix (Ms/dt + Alin + P_bv (s_i0 J_bv + J_ce + k_pl J_pl)
    U + P_1c J_1c U, Eq. ap4:fully_reduced differentiated) against central
    differences of the reduced residual: the differences converge as h^2 and
    agree to ~1e-11 at h = 1e-5, 1e-9 is the bound.  Each plausible slip planted
    in the oracle's Jacobian (the plating rate constant or the exchange-current
    scale dropped, the storage term multiplied by dt, the interpolation rows of
    the migration term left out) fails it."""
    cell, mu, snaps, traj, rom = trained
    assert _jacobian_fd_error(rom, cell, traj, mu) <= 1e-9
    real = R.reduced_jacobian
    for old, new in (('k_pl * J["pl"]', 'J["pl"]'), ('s_i0 * J["bv"]', 'J["bv"]'),
                     ("rom.Ms / dt", "rom.Ms * dt"), ("+ rom.P1c_proj @ J1c", "")):
        monkeypatch.setattr(R, "reduced_jacobian", _mutated(real, old, new))
        assert _jacobian_fd_error(rom, cell, traj, mu) > 1e-6, (old, new)
    monkeypatch.setattr(R, "reduced_jacobian", real)
