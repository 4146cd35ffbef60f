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
