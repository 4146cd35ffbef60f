"""Pins of the oracle parts that the invariant tests cannot see (CPU only).

* The cathode's Butler-Volmer face (Eq. ise_gr with the cathode's
  parameters): conservation, rest state and the complex-step Jacobian hold for
  any kinetics, so the magnitude of the cathode term is pinned by a planar
  K|E face that must carry the whole cell current.
* EI-Greedy point and basis selection (Sec. workflow:MOR, the EI-Greedy
  paragraph): a hand-worked training matrix whose selection sequence,
  including two ties, is written out below.
* POD truncation (Sec. workflow:MOR, snapshot POD in the L^2 inner product): a
  snapshot matrix built from a known W-orthonormal basis and known singular
  values, so that the k kept modes must span the k dominant directions.

Each pin is followed by a test that plants a plausible mistake in the oracle
(on the CPU) and checks that the pin then fails.
"""
import copy
import math

import numpy as np
import pytest

import synthetic as syn
from synthetic import E, K, L, CN, CP
from oracle import rom as R
from oracle.fom import Cell, ocp


# ------------------------------------------------------ cathode Butler-Volmer
def _cathode_cell(params):
    # CN | L | E E E | K K | CP: the Li-foil face and the cathode face each
    # carry the whole current in a 1-D stack
    return Cell(syn.slab_1d([CN, L, E, E, E, K, K, CP]), 1e-6, params)


def _cathode_overpotential_error(params, I, step_cell=None):
    """|eta_K - (2RT/F) asinh(i / (2 i00_K sqrt(c_K c_E)))| at the converged
    state of one step at current I, with i = -I the current density from the
    cathode into the electrolyte (I > 0 delithiates the anode, so the cathode
    takes lithium up)."""
    cell = step_cell if step_cell is not None else _cathode_cell(params)
    u, _ = cell.step(cell.initial_state(), 1.0, I)
    c, phi = u[:cell.N], u[cell.N:2 * cell.N]
    k, e = 5, 4                     # first cathode voxel and its electrolyte neighbour
    p = params
    RT_F = p["R"] * p["T"] / p["F"]
    i0 = p["K"]["i00"] * math.sqrt(c[k] * c[e])
    eta = phi[k] - ocp(c[k] / p["K"]["cmax"], p["K"]["ocp"]) - phi[e]
    return abs(eta - 2 * RT_F * math.asinh(-I / (2 * i0))), eta, i0


@pytest.mark.parametrize("I", [0.05, 3.0, -2.0])
def test_cathode_butler_volmer_single_face(params, I):
    """Eq. (ise_gr) for the cathode: the single K|E face carries -I, so its
    overpotential is the asinh of the current over 2 i00_K sqrt(c_K c_E); for
    small currents it tends to the linearisation -RT I / (F i00_K sqrt(c_K c_E))."""
    err, eta, i0 = _cathode_overpotential_error(params, I)
    assert err < 1e-12
    if abs(I) < 0.1:
        RT_F = params["R"] * params["T"] / params["F"]
        lin = -RT_F * I / i0
        x = I / (2 * i0)
        assert abs(eta - lin) / abs(lin) < x * x


def test_cathode_pin_detects_planted_mistakes(params):
    """The pin fails when the oracle's cathode term uses the graphite's
    exchange current density, or loses its sqrt(c_K c_E) factor."""
    I = 3.0

    class GraphiteI00(Cell):
        def residual(self, u, u_old, dt, I_app, gate, s_i0=1.0, k_pl=1.0):
            saved = self.p
            self.p = copy.deepcopy(saved)
            self.p["K"]["i00"] = saved["G"]["i00"]
            try:
                return Cell.residual(self, u, u_old, dt, I_app, gate, s_i0, k_pl)
            finally:
                self.p = saved

    class NoConcentrationFactor(Cell):
        # i = 2 i00_K sinh(F eta / 2RT): the same residual with i00_K divided
        # by the sqrt(c_K c_E) of the rest state (constant here)
        def residual(self, u, u_old, dt, I_app, gate, s_i0=1.0, k_pl=1.0):
            saved = self.p
            self.p = copy.deepcopy(saved)
            ck = np.atleast_2d(u)[:, 5].real
            ce = np.atleast_2d(u)[:, 4].real
            self.p["K"]["i00"] = saved["K"]["i00"] / float(np.sqrt(ck[0] * ce[0]))
            try:
                return Cell.residual(self, u, u_old, dt, I_app, gate, s_i0, k_pl)
            finally:
                self.p = saved

    lab = syn.slab_1d([CN, L, E, E, E, K, K, CP])
    for Mut in (GraphiteI00, NoConcentrationFactor):
        err, _, _ = _cathode_overpotential_error(params, I, Mut(lab, 1e-6, params))
        assert err > 1e-6, Mut.__name__


# ------------------------------------------------------------------ EI-Greedy
# Training columns t0, t1, t2 (rows 0..3).  Worked by hand:
#   step 1: max-norm errors (3, 3, 3), a three-way tie -> column 0; |t0| =
#           (1, 1, 3, 0) -> row 2; q1 = t0 / (-3) = (-1/3, -1/3, 1, 0).
#           With R[2, :] = (-3, -3, 0) the residuals R -= q1 R[2, :] are
#           t1 = (0, 2, 0, 0), t2 = (3, 3, 0, 2).
#   step 2: errors (0, 2, 3) -> column 2; |t2| = (3, 3, 0, 2) has a tie
#           between rows 0 and 1 -> row 0; q2 = t2 / 3 = (1, 1, 0, 2/3).
#           R[0, :] = (0, 0, 3) leaves t1 = (0, 2, 0, 0).
#   step 3: column 1, row 1; q3 = (0, 1, 0, 0).
# A rule on the largest 1-norm picks column 2 first, the highest index of a
# tie picks row 1 in step 2, and the largest signed error picks row 0 in step 1.
EI_T = np.array([[1.0, 1.0, 3.0],
                 [1.0, 3.0, 3.0],
                 [-3.0, -3.0, 0.0],
                 [0.0, 0.0, 2.0]])
EI_POINTS = [2, 0, 1]
EI_BASIS = np.array([[-1 / 3, -1 / 3, 1.0, 0.0],
                     [1.0, 1.0, 0.0, 2 / 3],
                     [0.0, 1.0, 0.0, 0.0]]).T


def _ei_check(greedy):
    Q, P = greedy(EI_T, 10)
    assert list(P) == EI_POINTS
    assert Q.shape == EI_BASIS.shape
    assert np.allclose(Q, EI_BASIS, rtol=0, atol=1e-15)
    # the interpolant of every training column is exact (the three columns
    # span the same space as the basis)
    for j in range(EI_T.shape[1]):
        assert np.allclose(R.ei_interpolate(Q, P, EI_T[P, j]), EI_T[:, j], atol=1e-14)


def test_ei_greedy_worked_example():
    """EI-Greedy takes the training column with the largest max-norm
    interpolation error, the row where that error is largest (ties: lowest
    index) and the error scaled to one there as the next basis vector."""
    _ei_check(R.ei_greedy)
    Q, P = R.ei_greedy(EI_T, 2)          # the bound on the number of points
    assert list(P) == EI_POINTS[:2]


def _mutant_greedy(pick_col, pick_row):
    def greedy(T, M, rel_tol=1e-12):
        Rm = np.array(T, dtype=np.float64, copy=True)
        Q, P = [], []
        for _ in range(M):
            if Rm.shape[1] == 0:
                break
            err = np.max(np.abs(Rm), axis=0)
            if err.max() <= rel_tol * np.max(np.abs(T)):
                break
            k = pick_col(Rm, err)
            r = Rm[:, k]
            p = pick_row(r)
            q = r / r[p]
            Q.append(q)
            P.append(p)
            Rm = Rm - np.outer(q, Rm[p, :])
        return np.array(Q).T, np.array(P, dtype=np.int64)
    return greedy


def test_ei_pin_detects_planted_mistakes():
    """Wrong column rule (largest 1-norm), wrong tie rule (highest index) and
    a wrong row (the maximum of the signed error instead of its magnitude)
    each change the selection."""
    first_max = lambda v: int(np.argmax(v))
    mutants = [
        _mutant_greedy(lambda Rm, err: int(np.argmax(np.sum(np.abs(Rm), axis=0))),
                       lambda r: int(np.argmax(np.abs(r)))),
        _mutant_greedy(lambda Rm, err: first_max(err),
                       lambda r: int(len(r) - 1 - np.argmax(np.abs(r)[::-1]))),
        _mutant_greedy(lambda Rm, err: first_max(err), lambda r: int(np.argmax(r))),
    ]
    for greedy in mutants:
        with pytest.raises(AssertionError):
            _ei_check(greedy)


# ------------------------------------------------------------------------ POD
def _pod_problem(seed=3, L=40, m=6, K=9):
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, L)                       # inner-product weights
    Qo, _ = np.linalg.qr(rng.standard_normal((L, m)))  # orthonormal in the plain inner product
    Vo, _ = np.linalg.qr(rng.standard_normal((K, m)))
    sv = np.array([10.0, 3.0, 1.0, 0.3, 1e-3, 1e-6])
    S = (Qo / np.sqrt(w)[:, None]) @ np.diag(sv) @ Vo.T  # = W^-1/2 Q Sigma V^T
    return S, w, Qo, sv


def _pod_check(pod):
    S, w, Qo, sv = _pod_problem()
    for k in (1, 2, 4):
        U, s = pod(S, w, k)
        assert U.shape[1] == k
        assert np.allclose(s[:len(sv)], sv, rtol=1e-10)
        # W-orthonormal
        assert np.allclose(U.T @ (w[:, None] * U), np.eye(k), atol=1e-12)
        # span(U) = span(W^-1/2 Q[:, :k]): the projection of the dominant
        # directions onto span(U) in the W inner product is the identity
        D = Qo[:, :k] / np.sqrt(w)[:, None]
        proj = U @ (U.T @ (w[:, None] * D))
        assert np.allclose(proj, D, atol=1e-10)
    # the relative cut-off keeps exactly the modes above it
    U, _ = pod(S, w, 10, rel_tol=1e-5)
    assert U.shape[1] == 5


def test_pod_keeps_the_dominant_modes():
    """The truncated POD basis spans the k dominant singular directions of the
    weighted snapshot matrix, with the singular values it was built from."""
    _pod_check(R.pod)


def test_pod_pin_detects_planted_mistakes():
    """Keeping the trailing modes, or weighting by W instead of W^(1/2), fails
    the pin."""
    def trailing(S, w, r, rel_tol=1e-10):
        sw = np.sqrt(w)[:, None]
        Uw, s, _ = np.linalg.svd(sw * S, full_matrices=False)
        k = int(min(r, np.count_nonzero(s > rel_tol * s[0])))
        return Uw[:, s.size - k:] / sw, s

    def full_weight(S, w, r, rel_tol=1e-10):
        sw = w[:, None]
        Uw, s, _ = np.linalg.svd(sw * S, full_matrices=False)
        k = int(min(r, np.count_nonzero(s > rel_tol * s[0])))
        return Uw[:, :k] / np.sqrt(sw), s

    for pod in (trailing, full_weight):
        with pytest.raises(AssertionError):
            _pod_check(pod)


# ------------------------------------------------------------- adaptive time step
def _mode_cell(params, n=10, h=1e-7):
    # the graphite slab of T1: zero-flux ends, cosine eigenmode of the discrete
    # diffusion operator with rate lam = (4 D / h^2) sin^2(pi / (2 n))
    cell = Cell(syn.slab_1d([CN] + [syn.G] * n + [CN]), h, params)
    D = params["G"]["D"]
    lam = 4.0 * D / h ** 2 * math.sin(math.pi / (2 * n)) ** 2
    mode = np.cos(math.pi * (np.arange(n) + 0.5) / n)
    return cell, lam, mode


def _mode_state(cell, params, mode, amp):
    n = len(mode)
    u = cell.initial_state()
    cmax = params["G"]["cmax"]
    u[1:1 + n] = 0.5 * cmax + amp * cmax * mode
    return u


@pytest.mark.parametrize("dt,dt_hist", [(0.05, 0.05), (0.05, 0.1), (0.1, 0.03)])
def test_local_error_estimate_is_the_implicit_euler_error(params, dt, dt_hist):
    """On a diffusion eigenmode the solution of the semi-discrete system is
    known in time (amplitude a e^{-lam t}) and the implicit Euler step has the
    amplitude a / (1 + lam dt): the local error estimate from the two previous
    exact states approaches the step's true error |a/(1+lam dt) - a e^{-lam
    dt}| (in the unknown scale c_max) as lam dt -> 0."""
    cell, lam, mode = _mode_cell(params)
    a = 0.1
    u_hist = _mode_state(cell, params, mode, a * math.exp(lam * dt_hist))
    u_start = _mode_state(cell, params, mode, a)
    u_new, _ = cell.step(u_start, dt, 0.0)
    true = abs(a / (1 + lam * dt) - a * math.exp(-lam * dt)) * np.max(np.abs(mode))
    est = cell.local_error(u_new, u_start, u_hist, dt, dt_hist)
    assert abs(est / true - 1.0) < 5 * lam * (dt + dt_hist), (est, true)


def test_local_error_pin_detects_planted_mistakes(params, monkeypatch):
    """The pin fails when the estimate's factor is dt / (dt + dt_hist) (a
    plausible slip: off by 3/2 for equal steps) or when the extrapolation
    uses the wrong sign."""
    def wrong_factor(self, u_new, u_start, u_hist, dt, dt_hist):
        u_pred = u_start + (dt / dt_hist) * (u_start - u_hist)
        return float(np.max(np.abs(u_new - u_pred) / self.unknown_scale())) * dt / (dt + dt_hist)

    def wrong_sign(self, u_new, u_start, u_hist, dt, dt_hist):
        u_pred = u_start - (dt / dt_hist) * (u_start - u_hist)
        return float(np.max(np.abs(u_new - u_pred) / self.unknown_scale())) * dt / (2.0 * dt + dt_hist)

    for mut in (wrong_factor, wrong_sign):
        monkeypatch.setattr(Cell, "local_error", mut)
        with pytest.raises(AssertionError):
            test_local_error_estimate_is_the_implicit_euler_error(params, 0.05, 0.05)
        monkeypatch.undo()


def test_adaptive_step_controller(params):
    """The controller: without history the step is taken as given; a step
    whose estimate exceeds tol is rejected and retried smaller; an accepted
    step proposes dt * clamp(0.9 sqrt(tol/e), 0.2, 2); a stationary state
    (zero estimate) doubles the step, up to dt_max."""
    cell, lam, mode = _mode_cell(params)
    u0 = _mode_state(cell, params, mode, 0.1)
    u1, i1 = cell.step_adaptive(u0, None, None, 1.0, 0.0, tol=1e-6)
    assert i1["dt_used"] == 1.0 and i1["rejects"] == 0
    # a tolerance the 1 s step cannot meet: rejections down to an accepted size
    u2, i2 = cell.step_adaptive(u1, u0, 1.0, 1.0, 0.0, tol=1e-7)
    assert i2["rejects"] >= 1 and i2["dt_used"] < 1.0 and i2["err"] <= 1e-7
    fac = min(2.0, max(0.2, 0.9 * math.sqrt(1e-7 / i2["err"])))
    assert abs(i2["dt_next"] - i2["dt_used"] * fac) <= 1e-15 * i2["dt_used"]
    # rest state: nothing changes, the estimate is zero, the step doubles
    r0 = cell.initial_state()
    r1, _ = cell.step_adaptive(r0, None, None, 2.0, 0.0, tol=1e-6)
    r2, i3 = cell.step_adaptive(r1, r0, 2.0, 2.0, 0.0, tol=1e-6, dt_max=3.0)
    assert i3["err"] == 0.0 and i3["dt_next"] == 3.0


def test_open_circuit_potentials_are_monotone(params):
    """The project's placeholder open-circuit potentials (the paper prints
    none) are strictly decreasing in the lithiation x on (0, 1), graphite within
    0.1-0.8 V and the cathode within 3.5-4.4 V, so that the full cell's
    open-circuit voltage is monotone in its state of charge."""
    from oracle.fom import ocp
    x = np.linspace(0.001, 0.999, 2000)
    for key, lo, hi in (("G", 0.1, 0.8), ("K", 3.5, 4.4)):
        a = params[key]["ocp"]
        u = np.array([ocp(v, a) for v in x])
        assert np.all(np.diff(u) < 0), key
        assert lo <= u.min() and u.max() <= hi, key
