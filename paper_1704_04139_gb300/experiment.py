"""The paper's model-reduction experiment (Sec. results) at reduced size, on
the GPU through the C-ABI.

Protocol, as the paper states it:

* a graphite | separator | Li-foil half cell with plated lithium seeded by
  the germ-grain model (germs of intensity 0.01 per square micrometre on the
  separator-anode plane, grains of radius 2.2 um, the plated layer one voxel
  thick: an inventory of h / V_m,Li on each grain face) and a high lithium
  concentration in the graphite (x = 0.75, the paper's "about 75 % state of
  charge" plateau);
* 60 s of constant-current delithiation at current densities mu in
  P = [2.5, 250] A/m^2 (C/10 to 10C in the paper's cell);
* snapshots from full-order runs at min P, max P and their mean; POD to a
  relative tolerance of 1e-7 of the largest singular value and EI-Greedy to
  1e-10 of the largest training entry (the stripping currents dominate that
  entry by ~1e3 over the Butler-Volmer terms, so this is ~1e-7 of those; at
  1e-7 of the largest entry the reduced potential misses the full-order one by
  5 % even at a training current); the reduced model keeps 97 % of
  the basis vectors and interpolation points of each space, the validation
  model of the error estimator all of them;
* the reduced model against the full-order model at 10 random mu in P plus
  the three training values: the relative model-reduction error, L-inf in
  time of the L^2 norm of the voxel grid, for concentration and potential; the
  hierarchical error estimate (theta = 0) and its over- and under-estimation
  factors; the estimate on 100 further mu; timings and the speedup.

The sizes are reduced (h = 1 um instead of 0.44 um, a smaller box) and the
time step is fixed at dt = 1 s for both models (the reduced model steps with a
fixed dt); the adaptive step of the full-order model is shown separately on the
largest current, across the stripping -> intercalation transition.

Inputs are synthetic stand-ins for the paper's GEOSTOCH anode (Boolean
spheres) and its parameter table (synthetic/params.json with x_G0 = 0.75).
"""
import copy
import math
import time

import numpy as np

P_MIN, P_MAX = 2.5, 250.0                    # A/m^2, the paper's parameter domain
PAPER_VALIDATION_DIMS = (183, 40, 69, 952, 1027)   # the paper's validation model (c, plated Li, phi, BV, 1/c)
# bounds of the reduced-size experiment's validation model: the paper's mode counts, at most 400 points per
# interpolated operator (each EI-Greedy step is a pass over the whole training matrix)
STUDY_DIMS = (183, 40, 69, 400, 400)


def half_cell_inputs(params, ny=32, nz=32, n_anode=48, n_sep=12, n_foil=2, porosity=0.35,
                     radius=("uniform", 2, 4), seed=61, x0=0.75, h=1e-6):
    """Labels, the experiment's parameter table and the germ-grain plating
    mask (over (voxel, direction) pairs)."""
    import synthetic as syn
    from synthetic.plating import germ_grain
    lab = syn.half_cell(ny, nz, n_anode, n_sep, n_foil, porosity, radius, seed)
    prm = copy.deepcopy(params)
    prm["G"]["x0"] = x0
    mask, hits = germ_grain(lab, h, 1 + n_anode, seed=seed)
    return lab, prm, mask, hits


def initial_state(cell, prm, mask, h=1e-6):
    """Rest state at x_G0 with the plated inventory h / V_m,Li on the grain
    faces (the one-voxel plated layer as a face inventory)."""
    u = cell.state()
    g, e, d = cell.plating_faces()
    shape = mask.shape[:3]
    t, y, z = np.unravel_index(g, shape)
    on = mask[t, y, z, d]
    u[2 * cell.N + np.nonzero(on)[0]] = h / prm["Pl"]["Vm_Li"]
    return u, int(np.count_nonzero(on))


def _field_norms(x, w, N):
    """W-norms of the c, phi and n blocks of the state(s) x (..., n)."""
    out = []
    for sl in (slice(0, N), slice(N, 2 * N), slice(2 * N, None)):
        out.append(np.sqrt(np.sum(w[sl] * x[..., sl] ** 2, axis=-1)))
    return out


def run_study(B, params, dt=1.0, steps=60, n_test=10, n_more=100, seed=62, sizes=None, opts=None,
              adaptive_tol=1e-3):
    """The experiment (module docstring); returns a JSON-able dict."""
    sizes = sizes or {}
    h = 1e-6
    lab, prm, mask, hits = half_cell_inputs(params, **sizes)
    if opts is None:
        opts = B.default_opts(precision=B.PREC_MIXED, newton_tol=1e-10, krylov_rtol=1e-5, max_halvings=3)
    cell = B.Cell(lab, h, prm, opts)
    u0, n_plated = initial_state(cell, prm, mask, h)
    cell.set_state(u0)
    N, n = cell.N, cell.n
    w = np.full(n, h ** 3)
    w[2 * N:] = h ** 2
    train = [(P_MIN, 1.0, 1.0), (P_MAX, 1.0, 1.0), (0.5 * (P_MIN + P_MAX), 1.0, 1.0)]
    t0 = time.perf_counter()
    red, val = B.Rom.build_pair(cell, train, dt, steps, STUDY_DIMS, frac=0.97, pod_tol=1e-7,
                                ei_tol=1e-10)
    build_s = time.perf_counter() - t0
    nc, nn, nphi = val.block_dims()
    cell.set_state(u0)
    rng = np.random.default_rng(seed)
    mus = [float(x) for x in rng.uniform(P_MIN, P_MAX, n_test)] + [t[0] for t in train]
    prm_i = [(mu, 1.0, 1.0) for mu in mus]
    red.solve(prm_i[:2], 2, dt)
    t0 = time.perf_counter()
    rt = red.solve_traj(prm_i, steps, dt)
    rom_wall = time.perf_counter() - t0
    U = red.basis(n)
    est = red.estimate(val, prm_i, steps, dt, 0.0)
    rows = []
    fom_wall = 0.0
    for k, mu in enumerate(mus):
        cell.set_state(u0)
        e_c, e_p, n_c, n_p, V = [], [], [], [], []
        for step in range(steps + 1):
            if step > 0:
                t1 = time.perf_counter()
                V.append(cell.step(dt, mu)["V_cell"])
                fom_wall += time.perf_counter() - t1
            u = cell.state()
            d = U @ rt["a"][k, step] - u
            dc, dp, _ = _field_norms(d, w, N)
            uc, up, _ = _field_norms(u, w, N)
            e_c.append(dc); e_p.append(dp); n_c.append(uc); n_p.append(up)
        e_c, e_p, n_c, n_p = map(np.array, (e_c, e_p, n_c, n_p))
        ec_max, ep_max = float(e_c.max()), float(e_p.max())
        es_c, es_p = float(np.max(est["est"][k, :, 0])), float(np.max(est["est"][k, :, 1]))
        rows.append({"mu": mu, "training": k >= n_test,
                     "rel_err": {"c": ec_max / float(n_c.max()), "phi": ep_max / float(n_p.max())},
                     "rel_est": {"c": es_c / float(np.max(est["norm_val"][k, :, 0])),
                                 "phi": es_p / float(np.max(est["norm_val"][k, :, 1]))},
                     "effectivity": {"c": es_c / ec_max if ec_max > 0 else None,
                                     "phi": es_p / ep_max if ep_max > 0 else None},
                     "V_fom": V, "V_rom": [float(x) for x in rt["V"][k, 1:]]})
    # the estimator on n_more further current densities
    more = [(float(x), 1.0, 1.0) for x in np.random.default_rng(seed + 1).uniform(P_MIN, P_MAX, n_more)]
    em = red.estimate(val, more, steps, dt, 0.0)
    rel_more = {f: float(np.max(np.max(em["est"][:, :, i], axis=1) / np.max(em["norm_val"][:, :, i], axis=1)))
                for i, f in enumerate(("c", "phi"))}
    # the full-order model with the adaptive step at the largest current
    cell.set_state(u0)
    t, dt_try, steps_a, rejects, trace = 0.0, 0.5, 0, 0, []
    while t < steps * dt - 1e-12:
        a = cell.step_adaptive(min(dt_try, steps * dt - t), P_MAX, adaptive_tol, dt_min=1e-3, dt_max=5.0)
        t += a["dt_used"]
        steps_a += 1
        rejects += a["rejects"]
        trace.append((t, a["dt_used"], a["V_cell"]))
        dt_try = a["dt_next"]
    tr = np.array(trace)
    late = tr[tr[:, 0] > 2.0] if np.any(tr[:, 0] > 2.0) else tr
    k_min = int(np.argmin(late[:, 1]))
    eff = [r["effectivity"] for r in rows]
    res = {
        "workload": "half cell %dx%dx%d voxels (h = 1 um; anode %d | separator %d | Li foil %d + collectors), "
                    "germ-grain plated Li on %d faces, x_G0 = 0.75, delithiation 60 s at dt = %g s"
                    % (lab.shape[1], lab.shape[2], lab.shape[0], sizes.get("n_anode", 48), sizes.get("n_sep", 12),
                       sizes.get("n_foil", 2), n_plated, dt),
        "voxels": int(N), "plating_faces": int(cell.F), "germs": int(len(hits)),
        "dims": {"validation": {"blocks_c_n_phi": [nc, nn, nphi], "ei_bv": val.n_bv, "ei_1c": val.n_1c},
                 "reduced": {"blocks_c_n_phi": list(red.block_dims()), "ei_bv": red.n_bv, "ei_1c": red.n_1c}},
        "max_rel_err": {f: max(r["rel_err"][f] for r in rows) for f in ("c", "phi")},
        "max_rel_est": {f: max(r["rel_est"][f] for r in rows) for f in ("c", "phi")},
        "estimator_over_factor": {f: max((e[f] for e in eff if e[f] and e[f] >= 1), default=None)
                                  for f in ("c", "phi")},
        "estimator_under_factor": {f: max((1.0 / e[f] for e in eff if e[f] and e[f] < 1), default=None)
                                   for f in ("c", "phi")},
        "max_rel_est_100_more": rel_more,
        "timing_s": {"full_order_per_simulation": fom_wall / len(mus), "reduced_batch_of_13": rom_wall,
                     "reduced_per_simulation_in_batch": rom_wall / len(mus),
                     "build_pair_from_one_snapshot_set": build_s},
        "speedup_per_simulation": (fom_wall / len(mus)) / (rom_wall / len(mus)),
        "failed": {"reduced": rt["failed"], "estimate": est["failed"] + em["failed"]},
        "adaptive_full_order_at_max_current": {"tol": adaptive_tol, "steps": steps_a, "rejects": rejects,
                                               "dt_min": float(tr[:, 1].min()), "dt_max": float(tr[:, 1].max()),
                                               "t_of_smallest_step_after_2s": float(late[k_min, 0]),
                                               "trace_t_dt_V": [[float(x) for x in r] for r in trace]},
        "rows": rows,
    }
    red.close()
    val.close()
    cell.close()
    return res
