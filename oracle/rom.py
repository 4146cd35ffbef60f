"""Reduced-order model oracle (test infrastructure only; see package header).

What it computes
----------------
The POD / empirical-interpolation reduced model of Sec. workflow:MOR for the
full-order system of oracle.fom (Eq. ap4:detailed), in the paper's order:

1. Snapshots (Sec. workflow:MOR): full-order trajectories at a few parameter
   points, including every intermediate Newton stage.
2. POD of the concentration part and of the potential part separately (Sec.
   workflow:MOR), with the plated-Li inventory n (a state of this
   discretisation the paper's volume-phase picture does not have) in a block
   of its own, in the L^2 inner product of the voxel grid (weight V per voxel
   value, A per face value): the method of snapshots by an SVD (a library
   routine) of the weighted snapshot matrix.  (In one block with c, whose
   weighted entries are ~1e6 times larger, n is represented only to c's
   rounding.)
3. Operator split (Eqs. ap4:operator_decomposition,
   ap4:operator_subdecomposition):
       R(u) = storage(u, u_old)/dt + A_lin(u) + mu A_bnd + A_1c(u)
              + s_i0 A_bv(u) + A_ce(u) + k_pl A_pl(u; g)
   A_lin: diffusion, conduction, the potential part of the electrolyte flux,
   the collector ghost term and the identity rows of voxels without c;
   A_bnd: the applied-current boundary term (mu = I_app); A_1c: the
   migration term with 1/cbar (the dmu/dc summand of Eq. phiel); A_bv,
   A_ce, A_pl: the interface currents of Eqs. ise_gr (graphite and cathode,
   scaled by the exchange-current scale s_i0), ise_li (Li foil) and iplel
   (plating, scaled by the rate scale k_pl, with the gate g), each entering
   the voxel rows and, for plating, the face rows.  A_const is zero in this
   discretisation.
4. EI-Greedy (Barrault et al. 2004; Drohmann et al. 2012): on the training set
   {A_bv, A_ce, A_pl at every snapshot} (one common basis, so that the scales
   s_i0 and k_pl stay exact: I[s O1 + k O2] = s I[O1] + k I[O2]) and
   separately on {A_1c at every snapshot}.  Each step takes the training
   vector with the largest max-norm interpolation error, the point where that
   error is largest (ties: lowest index) and the error vector scaled to one at
   that point as the new basis vector.
5. Galerkin projection of the fully reduced model, Eq. ap4:fully_reduced,
   with test space = trial space: the residual rows are weighted by D = (1 for
   the volume-integrated c and phi rows, A for the per-area face rows).
6. Online solve: per time step a reduced Newton iteration with the Jacobian
   assembled from the projected linear parts and the derivatives of the
   interpolated operators at the EI points; LU solve (library).  The plating
   gate uses the reconstructed state with the full-order rule and its
   active-set passes.  Outputs: s_cp (mean potential of the last layer) and
   s_ac (mean graphite concentration), as vectors on the reduced coefficients.

The oracle reconstructs the full state to evaluate the interpolated operators
(the definition); the GPU evaluates them on the stencil closure of the points.

Reduced Newton (the build's reading; the paper gives no solver details for
the reduced system): from the previous time step's coefficients, with the
full-order rule on the reconstructed update restricted to the stencil
closure of the EI points (the only values the interpolated nonlinearities
see): step length min(1, 0.25 / ||U_loc delta||_s) in the max-norm scaled by
the voxel unknowns' scales (c_ref, 1 V) and, for plated inventories, by
max(n_c, |n|) of the current reconstruction; stop after the first update with
lam ||U_loc delta||_s <= tol in the same scaled norm, or at a full step below
1e-10 that no longer halves the previous update (the rounding floor of the
reconstruction; at the experiment's full size the update of the float-float
GPU reconstruction levels off at 1e-12 - 5e-12).  The reduced linear
systems are solved by LU after row and column equilibration.

7. The hierarchical a-posteriori error estimate (Eq. ap4:estimate): the
   distance of the reduced model's reconstruction from a larger validation
   model's, per field and time step, scaled by 1/(1 - theta).

Parity status: pinned by tests/test_oracle_rom.py (the split reproduces the
full-order residual; the EI identity at the points; a ROM whose bases and EI
spaces contain the training trajectory reproduces that trajectory; rest-state
invariance at zero current; the reduced residual is affine in mu; the error
estimate is the L^2 norm of a constant field in closed form, scales as
1/(1 - theta), vanishes for identical models and equals the true error when
the validation model reproduces the full-order trajectory) and by
tests/test_oracle_pins.py (EI-Greedy's selection sequence on a hand-worked
training matrix with ties; POD truncation keeps the dominant directions of a
snapshot matrix built from known singular values).  The
accuracy of a truncated ROM against the full-order model is not pinned by the
paper for these inputs (parity unpinned for that comparison).
"""
import numpy as np
import scipy.linalg as sla

from synthetic.geometry import G
from oracle.fom import ocp as _ocp

TOL_NEWTON = 1e-12
TOL_FLOOR = 1e-10      # the full-order production tolerance: the rounding-floor stop
MAX_PASSES = 3
DELTA_MAX = 0.25


# ------------------------------------------------------------------ split
def suboperators(cell, u, gate, linear_only=False):
    """Sub-operator outputs for one state (n,) or a batch (B, n) (complex
    capable), each of the residual's shape: dict lin, c1, bv, ce, pl and the
    constant vector bnd (to be multiplied by mu).  linear_only: A_lin and
    A_bnd only (the others stay zero)."""
    single = u.ndim == 1
    U = np.atleast_2d(u)
    p = cell.p
    N, h, A = cell.N, cell.h, cell.A
    F = p["F"]
    c, phi, n = U[:, :N], U[:, N:2 * N], U[:, 2 * N:]
    B = U.shape[0]
    z = lambda: np.zeros((B, cell.n_unknowns), dtype=U.dtype)
    out = {k: z() for k in ("lin", "c1", "bv", "ce", "pl")}

    def add(key, Rc=None, Rp=None, Rn=None):
        o = out[key]
        if Rc is not None: o[:, :N] += Rc
        if Rp is not None: o[:, N:2 * N] += Rp
        if Rn is not None: o[:, 2 * N:] += Rn

    def clamp(x, lo):
        return np.where(x.real < lo, lo, x)

    cr = p["clamp_rel"]
    kap, tp = p["E"]["kappa"], p["E"]["tplus"]
    # identity rows of voxels without c
    Rc = np.zeros_like(c)
    Rc[:, ~cell.diffusive] = c[:, ~cell.diffusive]
    add("lin", Rc=Rc)
    # E-E faces: the linear (diffusion, potential) and the 1/cbar parts
    a, b = cell.ee
    if len(a):
        dc = c[:, b] - c[:, a]; dp = phi[:, b] - phi[:, a]
        j_lin = -kap * dp / h
        add("lin", Rc=(cell.M_ee @ (A * (-p["E"]["D"] * dc / h + (tp / F) * j_lin)).T).T,
            Rp=(cell.M_ee @ (A * j_lin).T).T)
    if len(a) and not linear_only:
        ca = clamp(c[:, a], cr * p["E"]["c0"]); cb = clamp(c[:, b], cr * p["E"]["c0"])
        cbar = 0.5 * (ca + cb)
        j_m = -kap * (tp - 1.0) * (cell.RT / F) * p["E"]["tdf"] * dc / (cbar * h)
        add("c1", Rc=(cell.M_ee @ (A * (tp / F) * j_m).T).T, Rp=(cell.M_ee @ (A * j_m).T).T)
    a, b, Ds, ss = cell.sd
    if len(a):
        add("lin", Rc=(cell.M_sd @ (A * (-Ds * (c[:, b] - c[:, a]) / h)).T).T,
            Rp=(cell.M_sd @ (A * (-ss * (phi[:, b] - phi[:, a]) / h)).T).T)
    a, b, sh = cell.cd
    if len(a):
        add("lin", Rp=(cell.M_cd @ (A * (-sh * (phi[:, b] - phi[:, a]) / h)).T).T)
    if len(cell.bc_dir):
        Rp = np.zeros_like(phi)
        Rp[:, cell.bc_dir] = 2.0 * A * p["CN"]["sigma"] * phi[:, cell.bc_dir] / h
        add("lin", Rp=Rp)
    f2 = cell.f2
    g, e = cell.pf_g, cell.pf_e
    if len(g) and not linear_only:
        cg = clamp(c[:, g], cr * p["G"]["cmax"]); ce = clamp(c[:, e], cr * p["E"]["c0"])
        eta = phi[:, g] - _ocp(cg / p["G"]["cmax"], p["G"]["ocp"]) - phi[:, e]
        ibv = 2.0 * p["G"]["i00"] * np.sqrt(cg * ce) * np.sinh(f2 * eta)
        add("bv", Rc=(cell.S_pg @ (A * ibv / F).T).T - (cell.S_pe @ (A * ibv / F).T).T,
            Rp=(cell.S_pg @ (A * ibv).T).T - (cell.S_pe @ (A * ibv).T).T)
        etap = phi[:, g] - phi[:, e]
        npos = np.where(n.real > 0, n, 0.0)
        fpre = npos ** 4 / (cell.nc ** 4 + npos ** 4)
        ipl = gate * p["Pl"]["i00"] * np.sqrt(ce) * (fpre * np.exp(f2 * etap) - np.exp(-f2 * etap))
        add("pl", Rc=-(cell.S_pe @ (A * ipl / F).T).T,
            Rp=(cell.S_pg @ (A * ipl).T).T - (cell.S_pe @ (A * ipl).T).T, Rn=ipl / F)
    s, e = cell.kitf
    if len(s) and not linear_only:
        cs = clamp(c[:, s], cr * p["K"]["cmax"]); ce = clamp(c[:, e], cr * p["E"]["c0"])
        eta = phi[:, s] - _ocp(cs / p["K"]["cmax"], p["K"]["ocp"]) - phi[:, e]
        ibv = 2.0 * p["K"]["i00"] * np.sqrt(cs * ce) * np.sinh(f2 * eta)
        add("bv", Rc=(cell.S_ks @ (A * ibv / F).T).T - (cell.S_ke @ (A * ibv / F).T).T,
            Rp=(cell.S_ks @ (A * ibv).T).T - (cell.S_ke @ (A * ibv).T).T)
    s, e = cell.litf
    if len(s) and not linear_only:
        ice = 2.0 * p["L"]["i00"] * np.sinh(f2 * (phi[:, s] - phi[:, e]))
        add("ce", Rc=-(cell.S_le @ (A * ice / F).T).T,
            Rp=(cell.S_ls @ (A * ice).T).T - (cell.S_le @ (A * ice).T).T)
    bnd = np.zeros(cell.n_unknowns)
    bnd[N + cell.bc_neu] = A
    if single:
        out = {k: v[0] for k, v in out.items()}
    out["bnd"] = bnd
    return out


def storage_diag(cell):
    """M_s with storage(u) = M_s (u - u_old) / dt: V on the c rows of E, G, K,
    1 on the face rows, 0 elsewhere."""
    N = cell.N
    m = np.zeros(cell.n_unknowns)
    m[:N][cell.diffusive] = cell.V
    m[2 * N:] = 1.0
    return m


def full_residual_from_split(cell, u, u_old, dt, mu, gate, s_i0, k_pl):
    so = suboperators(cell, u, gate)
    return (storage_diag(cell) * (u - u_old) / dt + so["lin"] + mu * so["bnd"] + so["c1"]
            + s_i0 * so["bv"] + so["ce"] + k_pl * so["pl"])


def sub_jacobians(cell, u, gate):
    """Jacobians (CSR) of the nonlinear sub-operators by complex-step
    differentiation with the full-order colouring (its pattern contains theirs)."""
    import scipy.sparse as sp
    rows, cols, color = cell._pattern()
    n = cell.n_unknowns
    hstep = 1e-20 * cell.unknown_scale()
    ncol = int(color.max()) + 1
    P = np.zeros((ncol, n), dtype=complex)
    P[color, np.arange(n)] = 1j * hstep
    so = suboperators(cell, u[None, :] + P, gate)
    J = {}
    for k in ("c1", "bv", "ce", "pl"):
        vals = so[k].imag[color[cols], rows] / hstep[cols]
        J[k] = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return J


# -------------------------------------------------------------- snapshots
def snapshots(cell, params, dt, n_steps, u0=None):
    """Full-order trajectories at the parameter points params = [(mu, s_i0,
    k_pl), ...] from the rest state: returns the list of (u, gate, (mu, s_i0,
    k_pl)) for the initial state, every Newton stage and every converged state,
    and the converged trajectories."""
    if u0 is None:
        u0 = cell.initial_state()
    snaps = []
    trajs = []
    for (mu, s_i0, k_pl) in params:
        u = u0.copy()
        g0 = cell.gate_at(u, cell.split(u)[2])
        snaps.append((u.copy(), g0, (mu, s_i0, k_pl)))
        traj = [u.copy()]
        for _ in range(n_steps):
            rec = []
            u, info = cell.step(u, dt, mu, s_i0, k_pl, record=rec)
            snaps += [(x, g, (mu, s_i0, k_pl)) for (x, g) in rec]
            traj.append(u.copy())
        trajs.append(np.array(traj))
    return snaps, trajs


# -------------------------------------------------------------------- POD
def weights(cell):
    """Inner-product weights of the full state: V per c and phi value, A per
    face value."""
    N = cell.N
    w = np.full(cell.n_unknowns, cell.V)
    w[2 * N:] = cell.A
    return w


def pod(S, w, r, rel_tol=1e-10):
    """W-orthonormal POD modes (columns) of the snapshot columns S: the left
    singular vectors of W^(1/2) S, mapped back by W^(-1/2); at most r modes,
    none below rel_tol of the largest singular value."""
    sw = np.sqrt(w)[:, None]
    Uw, sv, _ = np.linalg.svd(sw * S, full_matrices=False)
    if sv.size == 0 or sv[0] == 0:
        return np.zeros((S.shape[0], 0)), sv
    k = int(min(r, np.count_nonzero(sv > rel_tol * sv[0])))
    return Uw[:, :k] / sw, sv


# ---------------------------------------------------------------- EI-Greedy
def ei_greedy(T, M, rel_tol=1e-12):
    """EI-Greedy on the training columns T (L x K): returns the basis Q (L x m)
    and the points P (m,), m <= M.  Q[P, :] is unit lower triangular."""
    R = np.array(T, dtype=np.float64, copy=True)
    L = R.shape[0]
    scale = np.max(np.abs(T)) if T.size else 0.0
    Q, P = [], []
    for _ in range(M):
        if R.shape[1] == 0:
            break
        err = np.max(np.abs(R), axis=0)
        k = int(np.argmax(err))
        if err[k] <= rel_tol * scale:
            break
        r = R[:, k]
        p = int(np.argmax(np.abs(r)))
        q = r / r[p]
        Q.append(q)
        P.append(p)
        R = R - np.outer(q, R[p, :])
    if not Q:
        return np.zeros((L, 0)), np.zeros(0, np.int64)
    return np.array(Q).T, np.array(P, dtype=np.int64)


def ei_interpolate(Q, P, values_at_points):
    """I[O] = Q (Q[P,:])^-1 O[P]."""
    return Q @ sla.solve_triangular(Q[P, :], values_at_points, lower=True, unit_diagonal=True)


# ------------------------------------------------------------ build / solve
class ROM:
    """Reduced model data (all FP64 arrays)."""


def build(cell, snaps, dims, pod_tol=1e-10, ei_tol=1e-12):
    """Reduced model from snapshots.  dims = (n_c, n_phi, M_bv, M_1c), n_c
    bounding the c and the n block each; POD
    modes below pod_tol of the largest singular value and EI steps whose
    largest error is below ei_tol of the training set's largest entry are not
    taken."""
    N, F_ = cell.N, cell.F_pl
    n = cell.n_unknowns
    w = weights(cell)
    X = np.array([s[0] for s in snaps]).T                      # n x K
    cidx = np.arange(N)
    pidx = N + np.arange(N)
    nidx = 2 * N + np.arange(F_)
    Vc, svc = pod(X[cidx], w[cidx], dims[0], pod_tol)
    Vn, svn = pod(X[nidx], w[nidx], dims[0], pod_tol)
    Vp, svp = pod(X[pidx], w[pidx], dims[1], pod_tol)
    rc = Vc.shape[1] + Vn.shape[1]
    rp = Vp.shape[1]
    U = np.zeros((n, rc + rp))
    U[cidx, :Vc.shape[1]] = Vc
    U[nidx, Vc.shape[1]:rc] = Vn
    U[pidx, rc:] = Vp
    rom_nc, rom_nn = Vc.shape[1], Vn.shape[1]
    # training sets of the interpolated sub-operators
    Tbv, T1c = [], []
    for (u, g, prm) in snaps:
        so = suboperators(cell, u, g)
        for k in ("bv", "ce", "pl"):
            if np.any(so[k] != 0):
                Tbv.append(so[k])
        if np.any(so["c1"] != 0):
            T1c.append(so["c1"])
    Tbv = np.array(Tbv).T if Tbv else np.zeros((n, 0))
    T1c = np.array(T1c).T if T1c else np.zeros((n, 0))
    Qbv, Pbv = ei_greedy(Tbv, dims[2], ei_tol)
    Q1c, P1c = ei_greedy(T1c, dims[3], ei_tol)
    D = np.ones(n)
    D[2 * N:] = cell.A
    UD = U * D[:, None]                                         # D U (rows weighted)
    rom = ROM()
    rom.cell = cell
    rom.U, rom.rc, rom.rp = U, rc, rp
    rom.nc, rom.nn = rom_nc, rom_nn
    rom.sv_c, rom.sv_phi = svc, svp
    rom.Ms = UD.T @ (storage_diag(cell)[:, None] * U)
    lin_cols = suboperators(cell, U.T, np.zeros(F_), linear_only=True)["lin"].T  # columns A_lin(U e_j)
    rom.Alin = UD.T @ lin_cols
    rom.bbnd = UD.T @ suboperators(cell, np.zeros(n), np.zeros(F_), linear_only=True)["bnd"]
    rom.Qbv, rom.Pbv, rom.Q1c, rom.P1c = Qbv, Pbv, Q1c, P1c
    rom.Pbv_proj = (UD.T @ Qbv) @ np.linalg.inv(Qbv[Pbv, :]) if len(Pbv) else np.zeros((rc + rp, 0))
    rom.P1c_proj = (UD.T @ Q1c) @ np.linalg.inv(Q1c[P1c, :]) if len(P1c) else np.zeros((rc + rp, 0))
    last = np.arange(N).reshape(cell.shape)[-1].ravel()
    rom.s_cp = U[N + last, :].mean(axis=0)
    gvox = np.nonzero(cell.flat == G)[0]
    rom.s_ac = U[gvox, :].mean(axis=0) if len(gvox) else np.zeros(rc + rp)
    rom.a0 = U.T @ (w * cell.initial_state())                   # W-orthonormal columns
    rom.closure_faces = closure_plating_faces(cell, Pbv)
    rom.closure = stencil_closure(cell, np.concatenate([Pbv, P1c]))
    rom.Uloc = U[rom.closure, :]
    rom.us_loc = cell.unknown_scale()[rom.closure]
    return rom


def error_estimate(rom, rom_val, A, A_val, theta=0.0):
    """Hierarchical a-posteriori error estimate of Sec. workflow:MOR (Eqs.
    ap4:saturation and ap4:estimate): per time step n,
        e_c[n]   = ||c~_n - c^_n|| / (1 - theta),
        e_phi[n] = ||phi~_n - phi^_n|| / (1 - theta),
    where (c~, phi~) = U a is the reconstruction of the reduced model and
    (c^, phi^) = U^ a^ that of a larger validation model (V~ within V^ and
    larger interpolation bases) over the same steps, and || || is the L^2
    norm of the voxel grid (weight V per voxel value: the inner product the
    POD uses).  Under the saturation assumption with constant theta in [0, 1)
    these bound the reduced model's errors against the full-order solution.
    e_n is the same difference of the plated-Li inventory (weight A per face
    value), a state the paper's estimate does not have.  A and A_val are the
    coefficient trajectories, shapes (steps, N_r) and (steps, N_r^)."""
    if not 0.0 <= theta < 1.0:
        raise ValueError("theta must lie in [0, 1)")
    cell = rom.cell
    N = cell.N
    w = weights(cell)
    D = np.atleast_2d(A) @ rom.U.T - np.atleast_2d(A_val) @ rom_val.U.T   # steps x unknowns
    s = 1.0 / (1.0 - theta)
    blocks = {"c": slice(0, N), "phi": slice(N, 2 * N), "n": slice(2 * N, None)}
    return {k: s * np.sqrt(np.sum(w[b] * D[:, b] ** 2, axis=1)) for k, b in blocks.items()}


def stencil_closure(cell, points):
    """Degrees of freedom on which the residual rows `points` depend: the
    columns of those rows in the full-order Jacobian pattern."""
    rows, cols, _ = cell._pattern()
    sel = np.isin(rows, np.asarray(points))
    return np.unique(cols[sel])


def closure_plating_faces(cell, points):
    """Plating faces whose current enters some EI point's row (their gates
    matter to the reduced model)."""
    N = cell.N
    pts = np.asarray(points)
    vox = np.unique(np.concatenate([pts[pts < N], pts[(pts >= N) & (pts < 2 * N)] - N]))
    faces = pts[pts >= 2 * N] - 2 * N
    sel = np.isin(cell.pf_g, vox) | np.isin(cell.pf_e, vox)
    sel[faces] = True
    return np.nonzero(sel)[0]


def reduced_residual(rom, a, a_old, dt, mu, s_i0, k_pl, gate):
    cell = rom.cell
    u = rom.U @ a
    so = suboperators(cell, u, gate)
    f_bv = s_i0 * so["bv"][rom.Pbv] + so["ce"][rom.Pbv] + k_pl * so["pl"][rom.Pbv]
    f_1c = so["c1"][rom.P1c]
    return (rom.Ms @ (a - a_old) / dt + rom.Alin @ a + mu * rom.bbnd
            + rom.Pbv_proj @ f_bv + rom.P1c_proj @ f_1c)


def reduced_jacobian(rom, a, dt, s_i0, k_pl, gate):
    cell = rom.cell
    u = rom.U @ a
    J = sub_jacobians(cell, u, gate)
    Jbv = (s_i0 * J["bv"] + J["ce"] + k_pl * J["pl"])[rom.Pbv, :] @ rom.U
    J1c = J["c1"][rom.P1c, :] @ rom.U
    return rom.Ms / dt + rom.Alin + rom.Pbv_proj @ Jbv + rom.P1c_proj @ J1c


def equilibrated_solve(J, b):
    """x = J^-1 b with rows, then columns scaled to unit max-norm before the
    LU (library); the scaling leaves the solution unchanged and removes the
    ill-conditioning of the mixed concentration/potential/face units."""
    r = 1.0 / np.max(np.abs(J), axis=1)
    Jr = J * r[:, None]
    c = 1.0 / np.max(np.abs(Jr), axis=0)
    return c * np.linalg.solve(Jr * c[None, :], r * b)


class _NoConvergence(RuntimeError):
    pass


def _step(rom, a_old, mu, s_i0, k_pl, dt, tol, maxit):
    """One implicit Euler step of the reduced model from a_old: the plating
    active-set passes, each a reduced Newton iteration.  Returns (a, Newton
    iterations, gate flips); raises _NoConvergence."""
    cell = rom.cell
    N = cell.N
    its = flips = 0
    u_old = rom.U @ a_old
    n_old = u_old[2 * N:]
    gate = cell.gate_at(u_old, n_old)
    for npass in range(1, MAX_PASSES + 1):
        a = a_old.copy()
        ok = False
        dv_prev = np.inf
        for it in range(1, maxit + 1):
            r = reduced_residual(rom, a, a_old, dt, mu, s_i0, k_pl, gate)
            Jr = reduced_jacobian(rom, a, dt, s_i0, k_pl, gate)
            d = equilibrated_solve(Jr, -r)
            ud = rom.Uloc @ d
            du = np.abs(ud) / rom.us_loc
            dn = np.max(du) if len(du) else 0.0
            if not np.isfinite(dn):
                break
            # the step length as the full-order Newton takes it: the closure's
            # voxel unknowns (c, phi) in their scales, its plated inventories
            # relative to max(n_c, |n|) of the current reconstruction.  The
            # reduced iteration also stops in these scales: a plated layer of
            # ~1e3 n_c (Sec. workflow:degradation_modeling) strips at currents
            # whose exp sensitivity turns the rounding of the reconstruction
            # (~1e-16 of phi in FP64) into updates above 1e-12 n_c
            vox = rom.closure < 2 * N
            du_cap = du.copy()
            if np.any(~vox):
                n_cur = (rom.Uloc @ a)[~vox]
                du_cap[~vox] = np.abs(ud[~vox]) / np.maximum(cell.nc, np.abs(n_cur))
            dv = np.max(du_cap) if len(du_cap) else 0.0
            lam = 1.0 if dv <= DELTA_MAX else DELTA_MAX / dv
            a = a + lam * d
            its += 1
            # converged below tol, or at a full step below TOL_FLOOR that no longer
            # halves the previous update (the rounding floor of the reconstruction;
            # Newton's own convergence is quadratic)
            if lam * dv <= tol or (lam == 1.0 and dv <= TOL_FLOOR and it >= 2 and dv >= 0.5 * dv_prev):
                ok = True
                break
            dv_prev = dv
        if not ok:
            raise _NoConvergence("oracle reduced Newton did not converge")
        g2 = cell.gate_at(rom.U @ a, n_old)
        cf = rom.closure_faces
        nflip = int(np.count_nonzero(g2[cf] != gate[cf]))
        if nflip == 0 or npass == MAX_PASSES:
            break
        flips += nflip
        gate = g2
    return a, its, flips


def solve(rom, mu, s_i0, k_pl, dt, n_steps, tol=TOL_NEWTON, maxit=30, max_halvings=0):
    """Reduced trajectory from a0: returns dict with a (n_steps+1, N_r),
    V_cell and s_ac per step (index 0 = initial), newton iterations and
    gate flips.  A step that fails is retaken from the state before it as
    2^h steps of dt / 2^h, h = 1 .. max_halvings (the full-order step's dt
    halving); RuntimeError when the smallest substeps fail too."""
    a = rom.a0.copy()
    A_traj = [a.copy()]
    its_total = 0
    flips_total = 0
    for _ in range(n_steps):
        a_old = a.copy()
        for h in range(0, max_halvings + 1):
            try:
                a = a_old.copy()
                for _k in range(2 ** h):
                    a, its, flips = _step(rom, a, mu, s_i0, k_pl, dt / 2 ** h, tol, maxit)
                    its_total += its
                    flips_total += flips
                break
            except _NoConvergence:
                if h == max_halvings:
                    raise RuntimeError("oracle reduced Newton did not converge")
        A_traj.append(a.copy())
    A_traj = np.array(A_traj)
    return dict(a=A_traj, V_cell=A_traj @ rom.s_cp, s_ac=A_traj @ rom.s_ac,
                newton_its=its_total, flips=flips_total)
