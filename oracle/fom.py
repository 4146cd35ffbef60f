"""Full-order oracle (test infrastructure only; see package header).

What it computes
----------------
The implicit Euler system of Eq. (ap4:detailed) for the cell-centred finite
volume discretisation of Sec. 2.4 on a uniform voxel grid, with the
interface conditions of Eq. (interfaceCond) used as the numerical flux on
phase-interface faces (Sec. 2.4, first paragraph).

Unknowns: u = [c (N), phi (N), n (F)] with N voxels in [t][y][z] order (z
fastest) and F plating faces (every graphite-electrolyte face, ordered by the
graphite voxel's linear index and then by direction -t, +t, -y, +y, -z, +z).

Residual rows (units: mol/s, A, mol/(m^2 s)):

* R_c(v) = V (c_v - c_old,v)/dt + sum of Li outflows  (E, G, K voxels; Eqs.
  cgr and cel).  L, CN, CP voxels carry no concentration: R_c(v) = c_v.
* R_phi(v) = sum of current outflows (Eqs. phigr, phiel).
* R_n(f) = (n_f - n_old,f)/dt + i_pl,f / F  (plated-Li inventory per face).

Face fluxes from voxel a to its neighbour b (Delta = (.)_b - (.)_a, A = h^2):

* E-E (Eqs. cel, phiel with dmu/dc = RT/c * TDF, TDF = 1):
      j = -kappa dphi/h - kappa (t+ - 1) (RT/F) TDF dc / (cbar h),
      cbar = (c_a + c_b)/2,   N = -D_E dc/h + (t+/F) j.
* G-G, K-K (Eqs. cgr, phigr): N = -D_s dc/h, j = -sigma dphi/h.
* Any other pair of electronic conductors (L, CN, CP, G-CN, K-CP, ...):
  N = 0, j = -sigma_h dphi/h with the harmonic mean sigma_h (Table
  interfaceCond, "N = 0, j = cont.").
* Solid-electrolyte faces (Eq. interfaceCond, normal from solid to E):
  current density i from the solid into E;
      R_c(E) -= A i/F,  R_phi(E) -= A i,  R_phi(s) += A i,
      R_c(s) += A i_bv/F for s in {G, K}.
  G-E and K-E: Eq. (ise_gr)  i_bv = 2 i00 s_i0 sqrt(c_s c_E) sinh(F eta/(2RT)),
      eta = Phi_s - U0(c_s/cmax) - phi_E.
  L-E: Eq. (ise_li)  i = 2 i00_L sinh(F (Phi_L - phi_E)/(2RT)).
  G-E faces also carry plating/stripping, Eq. (iplel) with the overpotential
  of Eq. (ap2:theo:overpot:eq2) and the regulariser f_pre of Sec. 2.3:
      i_pl = g_f k_pl i00_Pl sqrt(c_E) (f_pre(n+) e^{F eta_p/(2RT)}
             - e^{-F eta_p/(2RT)}),   eta_p = Phi_G - phi_E,
      f_pre(n) = n^4/(n_c^4 + n^4),  n_c = 0.48 nm / V_m,Li,
  entering R_phi(G), R_c(E), R_phi(E) and R_n(f) (not R_c(G)).
* C-E faces: no flux (Table interfaceCond; its "N=-1" entry is read as the
  "N=0, j=0" printed for the same pair).
* Outer faces: t = 0 face of a CN voxel: Dirichlet Phi = 0 through a
  half-voxel ghost, outflow 2 A sigma_CN Phi / h; t = nt-1 face of a CP voxel:
  uniform outflow A I_app (I_app > 0 delithiates the anode); all other outer
  faces carry no flux.

Clamps: c is replaced by max(c, clamp_rel * c_ref) inside sqrt and 1/cbar.

Gate g_f (plating active set, the build's reading of "plating occurs when the
overpotential is negative", Sec. 2.3): g_f = 1 if n_old,f > 1e-9 n_c or
eta_p < 0 at the state where the gate is taken, else 0.  The gate is frozen during one
Newton solve; after convergence it is re-taken at the converged state and
the step is re-solved from u_old if any face flipped (at most 3 passes).

Parity status: pinned by tests/test_oracle_fom.py (closed forms T1, T2, T4,
T5, T6, rest-state invariance T3, Li conservation T7, affine-in-current T9,
mirror symmetry T10, and the complex-step Jacobian against central
differences T8) and tests/test_oracle_pins.py (the cathode's Butler-Volmer
face in closed form and its small-current linearisation).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synthetic.geometry import E, G, K, L, CN, CP

# direction order: (axis, step)
DIRS = ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))
_CONDUCTORS = (G, K, L, CN, CP)
DELTA_MAX = 0.25
N_GATE_REL = 1e-9
_FORBIDDEN = {(G, K), (G, CP), (K, CN), (CN, CP), (K, L)}


def ocp(x, a):
    """Open-circuit potential U0(x) = a0 + a1 x + a2 e^{-a3 x} + a4 tanh((x-a5)/a6).

    The paper treats U0 as a concentration dependent material property
    (Sec. 2.2, after Eq. ise_gr) without giving it; the form and its
    coefficients are the project's placeholders from the parameter table."""
    return a[0] + a[1] * x + a[2] * np.exp(-a[3] * x) + a[4] * np.tanh((x - a[5]) / a[6])


class GeometryError(ValueError):
    pass


class Cell:
    """Voxel cell: labels (nt, ny, nz) uint8, voxel edge h (m), parameter dict."""

    def __init__(self, labels, h, params):
        lab = np.ascontiguousarray(labels, dtype=np.uint8)
        if lab.ndim != 3:
            raise GeometryError("labels must be 3-D")
        self.lab = lab
        self.shape = lab.shape
        nt, ny, nz = lab.shape
        self.N = N = lab.size
        self.h = float(h)
        self.A = self.h ** 2
        self.V = self.h ** 3
        self.p = p = params
        self.RT = p["R"] * p["T"]
        self.f2 = p["F"] / (2.0 * self.RT)          # F/(2RT)
        flat = lab.ravel()
        self.flat = flat
        idx = np.arange(N).reshape(lab.shape)

        sigma = np.zeros(6)
        sigma[G] = p["G"]["sigma"]; sigma[K] = p["K"]["sigma"]; sigma[L] = p["L"]["sigma"]
        sigma[CN] = p["CN"]["sigma"]; sigma[CP] = p["CP"]["sigma"]
        self.sigma = sigma

        # per-voxel concentration reference (scaling, clamps)
        cref = np.ones(6)
        cref[E] = p["E"]["c0"]; cref[G] = p["G"]["cmax"]; cref[K] = p["K"]["cmax"]
        self.cref_v = cref[flat]
        self.diffusive = (flat == E) | (flat == G) | (flat == K)

        # ---- face classification (a -> b along +axis) ----
        ee_a, ee_b = [], []
        sd_a, sd_b, sd_D, sd_s = [], [], [], []
        cd_a, cd_b, cd_s = [], [], []
        itf = {G: ([], []), K: ([], []), L: ([], [])}
        Dph = np.zeros(6); Dph[G] = p["G"]["D"]; Dph[K] = p["K"]["D"]
        for ax in range(3):
            sl_lo = [slice(None)] * 3; sl_hi = [slice(None)] * 3
            sl_lo[ax] = slice(0, -1); sl_hi[ax] = slice(1, None)
            la = lab[tuple(sl_lo)].ravel(); lb = lab[tuple(sl_hi)].ravel()
            ia = idx[tuple(sl_lo)].ravel(); ib = idx[tuple(sl_hi)].ravel()
            for (x, y) in _FORBIDDEN:
                bad = ((la == x) & (lb == y)) | ((la == y) & (lb == x))
                if bad.any():
                    raise GeometryError("forbidden contact between phases %d and %d" % (x, y))
            m = (la == E) & (lb == E)
            ee_a.append(ia[m]); ee_b.append(ib[m])
            m = (la == lb) & ((la == G) | (la == K))
            sd_a.append(ia[m]); sd_b.append(ib[m]); sd_D.append(Dph[la[m]]); sd_s.append(sigma[la[m]])
            ca = np.isin(la, _CONDUCTORS); cb = np.isin(lb, _CONDUCTORS)
            m = ca & cb & ~((la == lb) & ((la == G) | (la == K)))
            sa_, sb_ = sigma[la[m]], sigma[lb[m]]
            cd_a.append(ia[m]); cd_b.append(ib[m]); cd_s.append(2.0 * sa_ * sb_ / (sa_ + sb_))
            for s in (G, K, L):
                m1 = (la == s) & (lb == E)
                m2 = (la == E) & (lb == s)
                itf[s][0].append(np.concatenate([ia[m1], ib[m2]]))
                itf[s][1].append(np.concatenate([ib[m1], ia[m2]]))
        cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0, np.int64)
        # each collector present must touch electrode solid, else its potential
        # floats and the applied current has no path (singular system)
        for cc_, sol in ((CN, (G, L)), (CP, (K, L))):
            if np.any(flat == cc_):
                touch = False
                for ax in range(3):
                    sl_lo = [slice(None)] * 3; sl_hi = [slice(None)] * 3
                    sl_lo[ax] = slice(0, -1); sl_hi[ax] = slice(1, None)
                    la = lab[tuple(sl_lo)]; lb = lab[tuple(sl_hi)]
                    touch |= bool(np.any(((la == cc_) & np.isin(lb, sol)) | ((lb == cc_) & np.isin(la, sol))))
                if not touch:
                    raise GeometryError("collector %d touches no electrode solid" % cc_)
        self.ee = (cat(ee_a), cat(ee_b))
        self.sd = (cat(sd_a), cat(sd_b), cat(sd_D), cat(sd_s))
        self.cd = (cat(cd_a), cat(cd_b), cat(cd_s))
        self.kitf = (cat(itf[K][0]), cat(itf[K][1]))
        self.litf = (cat(itf[L][0]), cat(itf[L][1]))

        # ---- plating faces: every G-E face, ordered by G voxel then direction ----
        pg, pe = [], []
        gvox = np.nonzero(flat == G)[0]
        coords = np.stack(np.unravel_index(gvox, lab.shape), axis=1)
        per_dir = []
        for d, (ax, st) in enumerate(DIRS):
            nb = coords.copy(); nb[:, ax] += st
            ok = (nb[:, ax] >= 0) & (nb[:, ax] < lab.shape[ax])
            nbi = np.full(len(gvox), -1, np.int64)
            nbi[ok] = np.ravel_multi_index(tuple(nb[ok].T), lab.shape)
            isE = np.zeros(len(gvox), bool)
            isE[ok] = flat[nbi[ok]] == E
            per_dir.append((nbi, isE))
        # interleave: for each G voxel in order, directions 0..5
        mask = np.stack([per_dir[d][1] for d in range(6)], axis=1)      # (nG, 6)
        nbrs = np.stack([per_dir[d][0] for d in range(6)], axis=1)
        gi, di = np.nonzero(mask)                                        # row-major: G voxel, then dir
        self.pf_g = gvox[gi]
        self.pf_e = nbrs[gi, di]
        self.pf_dir = di
        self.F_pl = len(self.pf_g)
        self.n_unknowns = 2 * N + self.F_pl

        # boundaries
        t0 = idx[0].ravel(); self.bc_dir = t0[flat[t0] == CN]
        t1 = idx[-1].ravel(); self.bc_neu = t1[flat[t1] == CP]

        # incidence matrices for the antisymmetric bulk fluxes
        def inc(a, b):
            nf = len(a)
            rows = np.concatenate([a, b]); cols = np.concatenate([np.arange(nf), np.arange(nf)])
            vals = np.concatenate([np.ones(nf), -np.ones(nf)])
            return sp.csr_matrix((vals, (rows, cols)), shape=(N, nf))
        def pick(a):
            return sp.csr_matrix((np.ones(len(a)), (a, np.arange(len(a)))), shape=(N, len(a)))
        self.S_pg, self.S_pe = pick(self.pf_g), pick(self.pf_e)
        self.S_ks, self.S_ke = pick(self.kitf[0]), pick(self.kitf[1])
        self.S_ls, self.S_le = pick(self.litf[0]), pick(self.litf[1])
        self.M_ee = inc(*self.ee)
        self.M_sd = inc(self.sd[0], self.sd[1])
        self.M_cd = inc(self.cd[0], self.cd[1])

        # 1C current density (A/m^2): graphite capacity over one hour per cross-section
        nG = int(np.count_nonzero(flat == G))
        self.i_1c = (p["F"] * self.V * p["G"]["cmax"] * (1.0 - p["G"]["x0"]) * nG / 3600.0
                     / (ny * nz * self.A))
        self.nc = p["Pl"]["layer_m"] / p["Pl"]["Vm_Li"]

    # ------------------------------------------------------------------ state
    def initial_state(self):
        """Rest state: table concentrations and equilibrium potentials."""
        p = self.p
        N, flat = self.N, self.flat
        c = np.zeros(N); phi = np.zeros(N)
        xg, xk = p["G"]["x0"], p["K"]["x0"]
        c[flat == E] = p["E"]["c0"]
        c[flat == G] = xg * p["G"]["cmax"]
        c[flat == K] = xk * p["K"]["cmax"]
        phiE = -ocp(np.float64(xg * p["G"]["cmax"]) / p["G"]["cmax"], p["G"]["ocp"])
        phiK = phiE + ocp(np.float64(xk * p["K"]["cmax"]) / p["K"]["cmax"], p["K"]["ocp"])
        phi[flat == E] = phiE
        phi[flat == K] = phiK
        phi[flat == L] = phiE
        phi[flat == G] = 0.0
        phi[flat == CN] = 0.0
        phi[flat == CP] = phiK if np.any(flat == K) else phiE
        return np.concatenate([c, phi, np.zeros(self.F_pl)])

    def split(self, u):
        N = self.N
        return u[..., :N], u[..., N:2 * N], u[..., 2 * N:]

    # --------------------------------------------------------------- residual
    def residual(self, u, u_old, dt, I_app, gate, s_i0=1.0, k_pl=1.0):
        """R(u) for one state (n,) or a batch (B, n); real or complex dtype."""
        single = u.ndim == 1
        U = np.atleast_2d(u)
        p = self.p
        N, h, A, V = self.N, self.h, self.A, self.V
        F = p["F"]
        c, phi, n = U[:, :N], U[:, N:2 * N], U[:, 2 * N:]
        c_old, phi_old, n_old = self.split(u_old)
        Rc = np.zeros_like(c); Rp = np.zeros_like(phi)
        dif = self.diffusive
        Rc[:, dif] = V * (c[:, dif] - c_old[dif]) / dt
        Rc[:, ~dif] = c[:, ~dif]

        def clamp(x, lo):
            return np.where(x.real < lo, lo, x)

        cr = p["clamp_rel"]
        # E-E faces
        a, b = self.ee
        if len(a):
            ca = clamp(c[:, a], cr * p["E"]["c0"]); cb = clamp(c[:, b], cr * p["E"]["c0"])
            dc = c[:, b] - c[:, a]; dp = phi[:, b] - phi[:, a]
            cbar = 0.5 * (ca + cb)
            kap, tp = p["E"]["kappa"], p["E"]["tplus"]
            j = -kap * dp / h - kap * (tp - 1.0) * (self.RT / F) * p["E"]["tdf"] * dc / (cbar * h)
            Nf = -p["E"]["D"] * dc / h + (tp / F) * j
            Rc += (self.M_ee @ (A * Nf).T).T
            Rp += (self.M_ee @ (A * j).T).T
        # same-phase intercalation solids
        a, b, Ds, ss = self.sd
        if len(a):
            Nf = -Ds * (c[:, b] - c[:, a]) / h
            j = -ss * (phi[:, b] - phi[:, a]) / h
            Rc += (self.M_sd @ (A * Nf).T).T
            Rp += (self.M_sd @ (A * j).T).T
        # conduction-only pairs
        a, b, sh = self.cd
        if len(a):
            j = -sh * (phi[:, b] - phi[:, a]) / h
            Rp += (self.M_cd @ (A * j).T).T

        def scatter(R, S, vals):
            R += (S @ vals.T).T

        f2 = self.f2
        # graphite-electrolyte: Butler-Volmer + plating
        g, e = self.pf_g, self.pf_e
        Rn = np.zeros_like(n)
        if len(g):
            cg = clamp(c[:, g], cr * p["G"]["cmax"]); ce = clamp(c[:, e], cr * p["E"]["c0"])
            eta = phi[:, g] - ocp(cg / p["G"]["cmax"], p["G"]["ocp"]) - phi[:, e]
            ibv = 2.0 * p["G"]["i00"] * s_i0 * np.sqrt(cg * ce) * np.sinh(f2 * eta)
            etap = phi[:, g] - phi[:, e]
            npos = np.where(n.real > 0, n, 0.0)
            fpre = npos ** 4 / (self.nc ** 4 + npos ** 4)
            ipl = gate * k_pl * p["Pl"]["i00"] * np.sqrt(ce) * (fpre * np.exp(f2 * etap)
                                                                 - np.exp(-f2 * etap))
            scatter(Rc, self.S_pg, A * ibv / F)
            scatter(Rp, self.S_pg, A * (ibv + ipl))
            scatter(Rc, self.S_pe, -A * (ibv + ipl) / F)
            scatter(Rp, self.S_pe, -A * (ibv + ipl))
            Rn = (n - n_old) / dt + ipl / F
        # cathode-electrolyte: Butler-Volmer
        s, e = self.kitf
        if len(s):
            cs = clamp(c[:, s], cr * p["K"]["cmax"]); ce = clamp(c[:, e], cr * p["E"]["c0"])
            eta = phi[:, s] - ocp(cs / p["K"]["cmax"], p["K"]["ocp"]) - phi[:, e]
            ibv = 2.0 * p["K"]["i00"] * s_i0 * np.sqrt(cs * ce) * np.sinh(f2 * eta)
            scatter(Rc, self.S_ks, A * ibv / F)
            scatter(Rp, self.S_ks, A * ibv)
            scatter(Rc, self.S_ke, -A * ibv / F)
            scatter(Rp, self.S_ke, -A * ibv)
        # Li foil-electrolyte: counter-electrode kinetics
        s, e = self.litf
        if len(s):
            ice = 2.0 * p["L"]["i00"] * np.sinh(f2 * (phi[:, s] - phi[:, e]))
            scatter(Rp, self.S_ls, A * ice)
            scatter(Rc, self.S_le, -A * ice / F)
            scatter(Rp, self.S_le, -A * ice)
        # outer boundaries
        if len(self.bc_dir):
            Rp[:, self.bc_dir] += 2.0 * A * p["CN"]["sigma"] * phi[:, self.bc_dir] / h
        if len(self.bc_neu):
            Rp[:, self.bc_neu] += A * I_app
        R = np.concatenate([Rc, Rp, Rn], axis=1)
        return R[0] if single else R

    # ------------------------------------------------------- scales / norms
    def unknown_scale(self):
        return np.concatenate([self.cref_v, np.ones(self.N), np.full(self.F_pl, self.nc)])

    def residual_scale(self, dt):
        rc = np.where(self.diffusive, self.V * self.cref_v / dt, 1.0)
        return np.concatenate([rc, np.full(self.N, self.A * 1.0), np.full(self.F_pl, self.nc / dt)])

    def gate_at(self, u, n_old):
        """Active set: g = 1 where plated Li is present (n_old > N_GATE_REL n_c)
        or eta_p = Phi_G - phi_E < 0.  An inventory below 1e-9 of the
        critical layer counts as none (f_pre ~ 1e-36 there): the rule must
        not switch on rounding noise of a reconstructed state."""
        c, phi, n = self.split(u)
        etap = phi[self.pf_g] - phi[self.pf_e]
        return ((n_old > N_GATE_REL * self.nc) | (etap < 0)).astype(np.float64)

    # --------------------------------------------------------------- Jacobian
    def _pattern(self):
        if hasattr(self, "_pat"):
            return self._pat
        N, F_ = self.N, self.F_pl
        shp = self.shape
        tt, yy, zz = np.unravel_index(np.arange(N), shp)
        rows, cols = [], []
        vox_nb = [np.arange(N)]
        for ax, st in DIRS:
            co = [tt.copy(), yy.copy(), zz.copy()]
            co[ax] = co[ax] + st
            ok = (co[ax] >= 0) & (co[ax] < shp[ax])
            nb = np.full(N, -1, np.int64)
            nb[ok] = np.ravel_multi_index((co[0][ok], co[1][ok], co[2][ok]), shp)
            vox_nb.append(nb)
        for nb in vox_nb:
            v = np.nonzero(nb >= 0)[0]; w = nb[v]
            for fr in range(2):
                for fc in range(2):
                    rows.append(fr * N + v); cols.append(fc * N + w)
        f = np.arange(F_)
        for vv in (self.pf_g, self.pf_e):
            for fr in range(2):
                rows.append(fr * N + vv); cols.append(2 * N + f)
                rows.append(2 * N + f); cols.append(fr * N + vv)
        rows.append(2 * N + f); cols.append(2 * N + f)
        rows = np.concatenate(rows); cols = np.concatenate(cols)
        # colours: voxel (t%3, y%3, z%3) per field; faces by doubled midpoint mod 4
        col27 = (tt % 3) + 3 * (yy % 3) + 9 * (zz % 3)
        color = np.empty(2 * N + F_, np.int64)
        color[:N] = col27; color[N:2 * N] = 27 + col27
        if F_:
            m = np.stack([tt[self.pf_g] + tt[self.pf_e], yy[self.pf_g] + yy[self.pf_e],
                          zz[self.pf_g] + zz[self.pf_e]], axis=1)
            ax = np.array([d[0] for d in DIRS])[self.pf_dir]
            code = np.zeros(F_, np.int64)
            for a in range(3):
                sel = ax == a
                o1, o2 = [i for i in range(3) if i != a]
                code[sel] = (a * 8 + 4 * (m[sel, a] % 4 == 3) + 2 * (m[sel, o1] % 4 == 2)
                             + (m[sel, o2] % 4 == 2))
            color[2 * N:] = 54 + code
        self._pat = (rows, cols, color)
        return self._pat

    def jacobian(self, u, u_old, dt, I_app, gate, s_i0=1.0, k_pl=1.0):
        """Exact Jacobian (CSR) by complex-step differentiation of the residual,
        one batched evaluation per colour of a distance-2 colouring."""
        rows, cols, color = self._pattern()
        n = self.n_unknowns
        hstep = 1e-20 * self.unknown_scale()
        ncol = int(color.max()) + 1
        P = np.zeros((ncol, n), dtype=complex)
        P[color, np.arange(n)] = 1j * hstep
        Rz = self.residual(u[None, :] + P, u_old, dt, I_app, gate, s_i0, k_pl)
        vals = Rz.imag[color[cols], rows] / hstep[cols]
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    # ----------------------------------------------------------------- Newton
    def solve_linear(self, J, b, dt):
        """Sparse direct solve of J x = b (SciPy SuperLU).  Columns are scaled
        by the unknown scales and rows by the resulting diagonal magnitude, so
        that the 0.01 diagonal-pivot threshold keeps the symmetric
        minimum-degree ordering's pivots."""
        us = self.unknown_scale()
        Jc = (J @ sp.diags(us)).tocsr()
        dr = np.abs(Jc.diagonal())
        Js = (sp.diags(1.0 / dr) @ Jc).tocsc()
        lu = spla.splu(Js, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.01,
                       options=dict(SymmetricMode=True))
        return us * lu.solve(b / dr)

    def newton(self, u0, u_old, dt, I_app, gate, s_i0=1.0, k_pl=1.0, tol=1e-12, maxit=40, record=None):
        """Newton's method with sparse direct LU (SciPy SuperLU) for the linear
        correction equations (the paper's BEST solver used AMG there, Sec. 2.4).

        Step length: lam = min(1, DELTA_MAX / m) with DELTA_MAX = 0.25 and m
        the larger of the max-norm of the voxel unknowns' update (c, phi: the
        arguments of the exponentials) scaled by (c_ref, 1 V) and the largest
        plated-inventory update relative to max(n_c, |n|) at the current
        iterate (a thick layer may change by a quarter of itself, a thin one
        by a quarter of n_c).  Stops after the first applied update with
        lam * ||delta||_s <= tol, ||.||_s the max-norm of every unknown scaled
        by (c_ref, 1 V, n_c).
        With a list `record`, every iterate (after each update) is appended
        together with the gate it was computed with."""
        u = u0.copy()
        us = self.unknown_scale()
        for it in range(1, maxit + 1):
            R = self.residual(u, u_old, dt, I_app, gate, s_i0, k_pl)
            J = self.jacobian(u, u_old, dt, I_app, gate, s_i0, k_pl)
            d = self.solve_linear(J, -R, dt)
            dn = np.max(np.abs(d) / us)
            if not np.isfinite(dn):
                return u, it, False
            dv = np.max(np.abs(d[:2 * self.N]) / us[:2 * self.N])
            if self.F_pl:
                n_cur = u[2 * self.N:].real
                dv = max(dv, float(np.max(np.abs(d[2 * self.N:]) / np.maximum(self.nc, np.abs(n_cur)))))
            lam = 1.0 if dv <= DELTA_MAX else DELTA_MAX / dv
            u = u + lam * d
            if record is not None:
                record.append((u.copy(), np.array(gate, dtype=np.float64)))
            if lam * dn <= tol:
                return u, it, True
        return u, maxit, False

    def step(self, u_old, dt, I_app, s_i0=1.0, k_pl=1.0, tol=1e-12, max_passes=3, record=None):
        """One implicit Euler step of Eq. (ap4:detailed) with the plating
        active-set passes.  Returns (u_new, info dict).  `record` collects
        the Newton stages (see newton)."""
        n_old = self.split(u_old)[2]
        gate = self.gate_at(u_old, n_old)
        its = 0
        flips = 0
        for npass in range(1, max_passes + 1):
            u, it, ok = self.newton(u_old, u_old, dt, I_app, gate, s_i0, k_pl, tol, record=record)
            its += it
            if not ok:
                raise RuntimeError("oracle Newton did not converge")
            g2 = self.gate_at(u, n_old)
            nflip = int(np.count_nonzero(g2 != gate))
            if nflip == 0 or npass == max_passes:
                break
            flips += nflip
            gate = g2
        unresolved = nflip if nflip and npass == max_passes else 0
        info = dict(newton_its=its, passes=npass, flips=flips, unresolved_flips=unresolved, gate=gate)
        info.update(self.functionals(u))
        return u, info

    # ----------------------------------------------------------- adaptive dt
    def local_error(self, u_new, u_start, u_hist, dt, dt_hist):
        """Local error estimate of the implicit Euler step from u_start (time
        t) to u_new (t + dt), with u_hist the state at t - dt_hist, in the
        max-norm scaled by the unknown scales.  For a smooth solution the
        implicit Euler step errs by (dt^2/2) u'' and the linear extrapolation
        u_pred = u_start + (dt/dt_hist)(u_start - u_hist) by -dt(dt +
        dt_hist)/2 u'', so u_new - u_pred = dt(2 dt + dt_hist)/2 u'' and the
        step's local error is dt/(2 dt + dt_hist) (u_new - u_pred) to leading
        order."""
        u_pred = u_start + (dt / dt_hist) * (u_start - u_hist)
        return float(np.max(np.abs(u_new - u_pred) / self.unknown_scale())) * dt / (2.0 * dt + dt_hist)

    def step_adaptive(self, u_start, u_hist, dt_hist, dt_try, I_app, tol, dt_min=1e-3, dt_max=60.0,
                      s_i0=1.0, k_pl=1.0, max_rejects=10):
        """One accepted step of adaptive size (Sec. workflow:discretization
        adapts the time step; the controller is the build's).  Without a
        history (u_hist None) the step of size dt_try is accepted as is.
        Otherwise a step with local error estimate e > tol is rejected and
        retried with dt * clamp(0.9 sqrt(tol / e), 0.2, 2) (first order
        method: exponent 1/2), down to dt_min, at most max_rejects times; the
        accepted step proposes the next size by the same factor, within
        [dt_min, dt_max].  Returns (u_new, info) with dt_used, dt_next, err,
        rejects."""
        dt = min(max(dt_try, dt_min), dt_max)
        rejects = 0
        while True:
            u, info = self.step(u_start, dt, I_app, s_i0, k_pl)
            if u_hist is None:
                info.update(dt_used=dt, dt_next=dt, err=0.0, rejects=0)
                return u, info
            e = self.local_error(u, u_start, u_hist, dt, dt_hist)
            fac = 2.0 if e == 0.0 else min(2.0, max(0.2, 0.9 * np.sqrt(tol / e)))
            if e <= tol or dt <= dt_min or rejects >= max_rejects:
                info.update(dt_used=dt, dt_next=min(max(dt * fac, dt_min), dt_max), err=e, rejects=rejects)
                return u, info
            rejects += 1
            dt = max(dt * fac, dt_min)

    # ------------------------------------------------------------ functionals
    def functionals(self, u):
        """Linear outputs (Sec. 2.5, s_cp and s_ac) and Li inventories."""
        c, phi, n = self.split(u)
        flat = self.flat
        nt, ny, nz = self.shape
        Vcell = float(np.mean(phi.reshape(self.shape)[-1]))
        g = flat == G
        mean_cG = float(np.mean(c[g])) if g.any() else 0.0
        dif = self.diffusive
        li_total = self.V * float(np.sum(c[dif])) + self.A * float(np.sum(n))
        li_anode = self.V * float(np.sum(c[g])) + self.A * float(np.sum(n))
        return dict(V_cell=Vcell, mean_c_solid=mean_cG, Li_total=li_total,
                    Li_anode=li_anode, Li_plated=self.A * float(np.sum(n)))
