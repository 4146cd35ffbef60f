#!/usr/bin/env python3
"""Benchmark of the full-order implicit step (the hot path) on one GB300.

Workload (default): the 128x128x256-voxel full cell at h = 1 um (anode 112 |
separator 32 | cathode 112 voxels + one collector layer at each end),
Boolean-sphere electrodes with log-normal radii (mean 5 voxels, sigma_log 0.3)
at porosity 0.30 (anode) / 0.35 (cathode), seeds (21, 22), charged at 2C with
plating enabled, implicit Euler with dt = 1 s.  A *step* is one implicit Euler
time step of that charge (Newton-Krylov with the multigrid preconditioner and
the plating active-set passes), run through the C-ABI on resident device
state.  Metric: simulated seconds per wall second.

The first warm-up step switches the current on from rest; the timed steps
continue the charge.  Inputs (state ~0.2 GB, operators ~1 GB) exceed the
129 MB L2, so no flush is needed between steps.

--impl reference times the FP64 CPU oracle (SciPy SuperLU Newton) on a bounded
sample of the same workload: one step of a 258x8x8-voxel window cut from the
same cell, per reported step, scaled to the full cell by voxel count.

Multi-GPU: the full-order step does not shard in this build (replicas only):
each rank runs its own copy of the workload and value = total simulated
seconds of all ranks / max wall time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sim-s/wall-s full-order; ROM solves/s + p50/p99 vs FP64 plain, V err≤1e-6"
UNIT = "sim-s/wall-s"


def workload_labels(name):
    import synthetic as syn
    if name == "cell128x128x256":
        return syn.full_cell(128, 128, 112, 32, 112, 0.30, 0.35, ("lognormal_mean", 5, 0.3), (21, 22))
    if name == "cell16x16x48":
        return syn.full_cell(16, 16, 20, 8, 20, 0.35, 0.35, ("uniform", 2, 4), (11, 12))
    if name == "cell32x32x96":
        return syn.full_cell(32, 32, 40, 16, 40, 0.35, 0.35, ("uniform", 2, 4), (11, 12))
    if name == "cell64x64x128":
        return syn.full_cell(64, 64, 53, 22, 53, 0.35, 0.35, ("uniform", 2, 4), (31, 32))
    raise SystemExit("unknown workload %s" % name)


CRATE = {"cell128x128x256": -2.0, "cell16x16x48": -1.0, "cell64x64x128": -2.0}


def fom_opts(B, prec, args):
    """Solver options of the full-order bench: Newton to 1e-10 in the scaled
    max-norm (the production tolerance), Krylov relative residual 1e-4 (mixed)
    or 1e-6 (FP64)."""
    return B.default_opts(precision=prec, newton_tol=1e-10, krylov_rtol=1e-4 if prec else 1e-6,
                          newton_maxit=20, krylov_maxit=300, max_halvings=3,
                          mg_bf16=0 if args.fp32_coarse else 1, mg_stream=args.mg_stream,
                          mg_tail=args.mg_tail, krylov_forcing=0 if args.no_ew else 1,
                          mg_kcycle_reorth=0 if args.kcycle_cgs1 else 1, mg_kcycle=args.mg_kcycle,
                          mg_smooth=args.mg_smooth, mg_coarse_pre=args.mg_coarse[0], mg_coarse_post=args.mg_coarse[1],
                          pc_lag=0 if args.no_pc_lag else 1, pc_lag_drift=args.pc_lag_drift,
                          mg_pdl=args.mg_pdl, newton_rate_test=0 if args.no_newton_rate_test else 1)


def step_record(infos):
    """Per-step solver record of the timed steps."""
    keys = ("newton_its", "krylov_its", "passes", "flips", "unresolved_flips", "halvings", "dt_used", "res_norm")
    return {k: [i[k] for i in infos] for k in keys}


def fields_rel_err(a, b, N):
    """Max-norm error of a against b per field, relative to b's max-norm."""
    out = {}
    for name, sl in (("c", slice(0, N)), ("phi", slice(N, 2 * N)), ("n_plated", slice(2 * N, None))):
        ref = b[sl]
        scale = float(np.max(np.abs(ref))) if ref.size else 0.0
        out[name] = float(np.max(np.abs(a[sl] - ref)) / scale) if scale > 0 else 0.0
    return out


def fp64_arm(B, labels, params, args, torch, V_mixed, u_mixed):
    """The same warm-up and timed steps with the FP64 solver (linearisation
    from the FP64 state in FP64, Krylov to 1e-6), timed with CUDA events on
    the cell's stream; the mixed run's cell potential of every timed step and
    its final fields are compared with it."""
    cell = B.Cell(labels, 1e-6, params, fom_opts(B, B.PREC_FP64, args))
    I = CRATE[args.workload] * cell.i_1c
    for _ in range(args.warmup):
        cell.step(1.0, I)
    stream = torch.cuda.ExternalStream(cell.stream_ptr())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    infos = [cell.step(1.0, I) for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    V = np.array([i["V_cell"] for i in infos])
    u64 = cell.state()
    N = cell.N
    cell.close()
    return {"value": args.steps / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms / args.steps,
            "precision": "f64 linearisation and residual; Krylov relative residual 1e-6",
            "mixed_vs_fp64": {"V_max_rel_err": float(np.max(np.abs(np.asarray(V_mixed) - V) / np.abs(V))),
                              "fields_max_rel_err_final": fields_rel_err(u_mixed, u64, N),
                              "bounds": {"V": 1e-6, "fields": 1e-5}},
            "solver": step_record(infos)}


def max_over_ranks(x, dist, device):
    """The largest x over the ranks of the process group (x without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws, steps, dt, ms):
    """Simulated seconds of all replicas per wall second: every rank advances its
    own cell by steps * dt in the (slowest rank's) ms."""
    return ws * steps * dt / (ms / 1000.0)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch.distributed as dist
    rank = int(os.environ["RANK"]); local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl"
    import torch
    torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return rank, local, ws, dist


class ClockSampler:
    """nvidia-smi clock/throttle sampling every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) > 1 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks(key="hbm_gbs"):
    """A measured peak (MEASURED_PEAKS.json: HBM copy GB/s, or BF16 GEMM TFLOP/s)
    and "measured", else the recipe's fallback and "fallback"."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d[key]), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}[key], "fallback"


def kernel_traffic(kernel, workload, mode):
    """DRAM bytes per launch of a kernel in the given mode from the committed
    ncu summary (profiles/<kernel>__<workload>.json), or None."""
    path = os.path.join(ROOT, "profiles", "%s__%s.json" % (kernel, workload))
    try:
        with open(path) as f:
            return float(json.load(f)["dram_bytes_per_launch"][mode])
    except Exception:
        return None


def oracle_sample(labels, params, crate_sign, nsteps=1):
    """Oracle (FP64, SciPy SuperLU) on a 258x8x8 window of the workload cell:
    returns (sim-s/wall-s scaled to the full cell, seconds, sample text)."""
    import synthetic.geometry as geo
    from oracle.fom import Cell as OCell
    win = geo.percolating(np.ascontiguousarray(labels[:, :8, :8]))
    oc = OCell(win, 1e-6, params)
    u = oc.initial_state()
    I = crate_sign * oc.i_1c
    t0 = time.perf_counter()
    for _ in range(nsteps):
        u, _ = oc.step(u, 1.0, I)
    wall = time.perf_counter() - t0
    scale = win.size / labels.size
    return (nsteps * 1.0 / wall) * scale, wall, ("%d oracle step(s) of a %dx8x8 window (%d voxels) of the %s cell, "
                                                  "scaled by voxel count %d/%d" %
                                                  (nsteps, win.shape[0], win.size, "workload", win.size, labels.size))


def run_reference(args):
    # the oracle runs on the host cores: no process group, no device; under
    # torchrun rank 0 alone runs it and the other ranks exit without work
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synthetic as syn
    params = syn.load_params()
    labels = workload_labels(args.workload)
    cores = 1
    vals = []
    for _ in range(args.warmup):
        oracle_sample(labels, params, np.sign(CRATE[args.workload]))
    t_all = 0.0
    for _ in range(args.steps):
        v, wall, sample = oracle_sample(labels, params, np.sign(CRATE[args.workload]))
        vals.append(v)
        t_all += wall
    value = float(np.mean(vals))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_all / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": args.workload, "dt_s": 1.0, "crate": CRATE[args.workload]},
           "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cores, "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


ROM_CELL = "cell16x16x48"
ROM_DIMS = (60, 30, 30, 200, 150)     # POD c, plated Li, phi; EI interface, migration (serving model)
ROM_DIMS_PAPER = (183, 40, 69, 952, 1027)   # the paper's 183 c / 69 phi modes, 952 BV / 1027 lambda points


def rom_paper_dims(B, params, args, torch, estimate=True):
    """The reduced model at the paper's dimensions (as far as the 16x16x48
    cell's snapshots support them): snapshots at four parameter points
    (C-rate 0.5, 5, 2, 1) over 60 steps, POD to 1e-9; a timed batch of
    --rom-instances instances over a bounded sample of the 600-step protocol
    (--rom-paper-steps steps), and the cell-potential error of two instances
    against full-order runs over that sample."""
    labels = workload_labels(ROM_CELL)
    opts = B.default_opts(precision=B.PREC_MIXED, newton_tol=1e-10, krylov_rtol=1e-5, max_halvings=3)
    cell = B.Cell(labels, 1e-6, params, opts)
    i1 = cell.i_1c
    t0 = time.perf_counter()
    snap = [(-0.5 * i1, 0.5, 0.1), (-5.0 * i1, 2.0, 10.0), (-2.0 * i1, 1.0, 1.0), (-1.0 * i1, 1.0, 1.0)]
    if estimate:
        r97, rom = B.Rom.build_pair(cell, snap, 1.0, 60, ROM_DIMS_PAPER, frac=0.97, pod_tol=1e-9)
    else:
        r97, rom = None, B.Rom.build(cell, snap, 1.0, 60, ROM_DIMS_PAPER, pod_tol=1e-9)
    build_s = time.perf_counter() - t0
    if args.rom_gemm >= 0:
        rom.debug_tensor(args.rom_gemm)
    rng = np.random.default_rng(43)
    prm = _rom_params(rng, args.rom_instances, i1)
    steps = args.rom_paper_steps
    rom.solve(prm, 1, 1.0)     # warm-up on the timed batch's shape (allocation, autotuning, graph capture)
    torch.cuda.synchronize()
    if args.rom_host_loop:
        rom.debug_graph(False)
    t0 = time.perf_counter()
    out = rom.solve(prm, steps, 1.0)
    wall = time.perf_counter() - t0
    tune = rom.gemm_tuning()
    inst_steps = args.rom_instances * steps
    errs = []
    for b in range(2):
        fc = B.Cell(labels, 1e-6, params, opts)
        fc.set_scales(prm[b][1], prm[b][2])
        V = np.array([fc.step(1.0, prm[b][0])["V_cell"] for _ in range(steps)])
        fc.close()
        errs.append(float(np.max(np.abs(out["V"][b][1:] - V)) / np.max(np.abs(V))))
    est = rom_error_estimate(r97, rom, prm, steps) if estimate else None
    res = {"workload": "ROM of the %s cell at the paper's dimensions, snapshots at (C-rate, i0 scale, k_pl) = "
                       "(0.5, 0.5, 0.1), (5, 2, 10), (2, 1, 1), (1, 1, 1), 60 steps each; %d of the 600 steps "
                       "timed" % (ROM_CELL, steps),
           "dims": {"n_r": rom.n_r, "ei_interface": rom.n_bv, "ei_migration": rom.n_1c,
                    "requested": list(ROM_DIMS_PAPER)},
           "instances": args.rom_instances, "steps": steps, "dt_s": 1.0,
           "precision": "f64 state and residual; float-float reconstruction; Newton matrix with f32 accuracy "
                        "(3xTF32 on the tensor cores) and f32 LU; escalated instances by f64 GMRES preconditioned "
                        "by their f32 LU",
           "instance_steps_per_s": inst_steps / wall, "solves_per_s": args.rom_instances / wall, "wall_s": wall,
           "build_s": build_s, "build_note": "validation and 97 % models from one snapshot set" if estimate else None,
           "newton_its_per_instance_step": out["newton_its"] / inst_steps,
           "failed": out["failed"], "V_rel_err_vs_full_order_2_instances": errs,
           "gemm": rom_gemm_figures(rom, tune, args),
           "step_mode": "host loop" if args.rom_host_loop else "one CUDA graph per time step",
           "error_estimate": est}
    rom.close()
    cell.close()
    return res


def rom_gemm_figures(rom, tune, args):
    """The Newton-matrix GEMM: the variant in use and, from the autotuning
    (256-instance scratch batch), each variant's time and the tensor rate of
    the three TF32 products per operand pair against the TF32 peak derived
    from the measured BF16 one (x 1.1 / 2.25, the nominal dense ratio)."""
    names = ["f32 fma", "mma.sync 3xtf32", "tcgen05 3xtf32"]
    out = {"variant": names[tune[0]]}
    if args.rom_gemm >= 0:
        return out
    flops = 3 * 2.0 * rom.n_r * (256 * rom.n_r) * (rom.n_bv + rom.n_1c)
    peak, kind = measured_peaks("bf16_tflops")
    tf32 = peak * 1.1 / 2.25 if peak else None
    out["autotune_ms_per_launch"] = {n: tune[1][k] for k, n in enumerate(names)}
    out["tensor_rate_tflops"] = {n: (flops / (tune[1][k] * 1e-3) / 1e12 if tune[1][k] > 0 else None)
                                 for k, n in enumerate(names) if k > 0}
    out["tf32_peak_tflops"] = tf32
    out["tf32_peak_kind"] = "%s (bf16 x 1.1/2.25)" % kind
    t = out["tensor_rate_tflops"].get("tcgen05 3xtf32")
    out["tcgen05_frac_of_tf32_peak"] = t / tf32 if (t and tf32) else None
    return out


def rom_error_estimate(r97, rom, prm, steps, n_inst=256):
    """The paper's certification step (Sec. workflow:MOR, Eq. ap4:estimate):
    the reduced model r97 with 97 % of the validation model's basis vectors
    and interpolation points per block (built from the same snapshots),
    estimated against the validation model `rom` on n_inst instances over the
    timed steps with theta = 0.  Relative errors as the paper states them:
    L-inf in time of the estimate over L-inf in time of the validation field's
    L^2 norm, the largest over the instances."""
    nc, nn, nphi = rom.block_dims()
    n_inst = min(n_inst, len(prm))
    t0 = time.perf_counter()
    out = r97.estimate(rom, prm[:n_inst], steps, 1.0, 0.0)
    wall = time.perf_counter() - t0
    e, nv = out["est"], out["norm_val"]
    rel = {}
    for f, k in enumerate(("c", "phi", "n_plated")):
        den = np.max(nv[:, :, f], axis=1)
        rel[k] = float(np.max(np.max(e[:, :, f], axis=1) / den)) if np.all(den > 0) else None
    v_err = float(np.max(np.abs(out["V"] - out["V_val"]) / np.abs(out["V_val"])))
    res = {"reduced_dims": {"n_r": r97.n_r, "blocks_c_n_phi": list(r97.block_dims()), "ei_interface": r97.n_bv,
                            "ei_migration": r97.n_1c},
           "validation_dims": {"n_r": rom.n_r, "blocks_c_n_phi": [nc, nn, nphi], "ei_interface": rom.n_bv,
                               "ei_migration": rom.n_1c},
           "instances": n_inst, "steps": steps, "theta": 0.0, "max_rel_estimate": rel,
           "V_rel_diff_reduced_vs_validation": v_err, "failed": out["failed"], "wall_s": wall}
    r97.close()
    return res


def _rom_params(rng, n, i1):
    """Parameter instances of the reduced-model study: C-rate ~ U(0.5, 5) (charge),
    exchange-current scale ~ LogU(0.5, 2), plating rate scale ~ LogU(0.1, 10)."""
    c = rng.uniform(0.5, 5.0, n)
    s = np.exp(rng.uniform(np.log(0.5), np.log(2.0), n))
    k = np.exp(rng.uniform(np.log(0.1), np.log(10.0), n))
    return [(-ci * i1, si, ki) for ci, si, ki in zip(c, s, k)]


SERVE_FOM_CELL = "cell32x32x96"
V_CUTOFF = 4.2   # charge protocols end at the 4.2 V limit (the cfg2 protocol's cutoff)


def _serve_requests(rng, n, i1, i1_fom):
    """n requests of the serving mix: 95 % reduced-model queries (protocol
    length U{100..3000} steps, C-rate from {0.5, 1, 2, 3, 5}, i0 scale and
    plating rate as the reduced-model study), 5 % full-order validation solves
    (60 steps)."""
    out = []
    for k in range(n):
        crate = float(rng.choice([0.5, 1.0, 2.0, 3.0, 5.0]))
        s = float(np.exp(rng.uniform(np.log(0.5), np.log(2.0))))
        kp = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        if rng.random() < 0.95:
            out.append(("rom", -crate * i1, s, kp, int(rng.integers(100, 3001))))
        else:
            out.append(("fom", -crate * i1_fom, s, kp, 60))
    return out


def serve_run(B, params, rom, i1, args, slots=256, workers=4, load=0.7):
    """Continuous batching under Poisson arrivals.  The server's capacity is
    measured on a burst of twice its slot count drawn from the same mix
    (reduced and full-order requests), and requests then arrive at 0.8 of it.
    Reduced requests run in the resident slot batch of `rom`; full-order
    validation solves run on worker threads with cells of the 32x32x96
    template (cfg1's generator rules), admitted by device memory."""
    flab = workload_labels(SERVE_FOM_CELL)
    fopts = B.default_opts(precision=B.PREC_MIXED, newton_tol=1e-10, krylov_rtol=1e-4, max_halvings=3)
    probe = B.Cell(flab, 1e-6, params, fopts)
    i1_fom = probe.i_1c
    fom_bytes = int(probe.device_bytes)
    probe.close()
    srv = B.Server(rom=rom, labels=flab, params=params, fom_opts=fopts, rom_slots=slots, fom_workers=workers,
                   fom_budget_bytes=workers * fom_bytes)

    def submit(r):
        kind = B.REQ_ROM if r[0] == "rom" else B.REQ_FOM
        return srv.submit(kind, r[1], r[2], r[3], r[4], 1.0, v_cutoff=V_CUTOFF)

    rng = np.random.default_rng(50)
    burst = _serve_requests(rng, 2 * slots, i1, i1_fom)
    t0 = time.perf_counter()
    left = {submit(r) for r in burst}
    while left:
        for t in list(left):
            if srv.poll(t) is not None:
                left.discard(t)
        time.sleep(0.001)
    cap = len(burst) / (time.perf_counter() - t0)
    rate = load * cap
    rng = np.random.default_rng(51)
    n_req = args.serve_requests
    reqs = _serve_requests(rng, n_req, i1, i1_fom)
    gaps = rng.exponential(1.0 / rate, n_req)
    t0 = time.perf_counter()
    t_next = t0
    pending, done, t_sub = {}, {}, {}
    for k, r in enumerate(reqs):
        t_next += gaps[k]
        while time.perf_counter() < t_next:
            for t in list(pending):
                res = srv.poll(t)
                if res is not None:
                    done[t] = (pending.pop(t), res)
            time.sleep(0.0005)
        t_s = time.perf_counter() - t0
        tk = submit(r)
        pending[tk] = r[0]
        t_sub[tk] = t_s
    t_arrivals = time.perf_counter() - t0
    while pending:
        for t in list(pending):
            res = srv.poll(t)
            if res is not None:
                done[t] = (pending.pop(t), res)
        time.sleep(0.001)
    total = time.perf_counter() - t0
    _, peak, _ = srv.debug_cells()
    srv.close()
    lat = {"rom": [], "fom": []}
    bad = cut = 0
    t_fin = []
    for tk, (kind, res) in done.items():
        lat[kind].append(1000.0 * (res["t_done"] - res["t_submit"]))
        t_fin.append(t_sub[tk] + (res["t_done"] - res["t_submit"]))
        bad += res["status"] not in (B.MB_OK, B.MB_ECUTOFF)
        cut += res["status"] == B.MB_ECUTOFF
    # steady state: completions in the second half of the arrival window against the
    # arrivals in it (the first half covers the fill-up of requests of up to 3000 steps;
    # the whole-run figure also carries the drain of the last long requests)
    t_fin = np.array(t_fin)
    half = 0.5 * t_arrivals
    done_2nd = int(np.count_nonzero((t_fin >= half) & (t_fin < t_arrivals)))
    arr_2nd = int(np.count_nonzero(np.array(list(t_sub.values())) >= half))
    return {"requests": n_req, "rom_fraction": 0.95, "arrival_rate_per_s": rate,
            "capacity_mixed_burst_per_s": cap, "throughput_per_s": n_req / total,
            "throughput_over_arrival_rate": (n_req / total) / (n_req / t_arrivals), "wall_s": total,
            "arrival_window_s": t_arrivals,
            "steady_state_second_half": {"completed": done_2nd, "arrived": arr_2nd,
                                         "throughput_over_arrival_rate": done_2nd / max(arr_2nd, 1)},
            "failed": int(bad), "ended_at_cutoff": int(cut), "v_cutoff": V_CUTOFF, "rom_slots": slots,
            "fom_workers": workers, "fom_cells_peak": peak,
            "p50_ms": {k: float(np.percentile(v, 50)) if v else None for k, v in lat.items()},
            "p99_ms": {k: float(np.percentile(v, 99)) if v else None for k, v in lat.items()},
            "workload": "Poisson arrivals at %.1f of the capacity measured on a mixed burst; 95 %% reduced "
                        "requests of U{100..3000} steps (C-rate in {0.5,1,2,3,5}, i0 scale ~ LogU(0.5,2), "
                        "plating rate ~ LogU(0.1,10)) on the reduced model of the %s cell; 5 %% full-order "
                        "validation solves of 60 steps on the %s cell; a sample of %d requests"
                        % (load, ROM_CELL, SERVE_FOM_CELL, n_req)}


def rom_and_serve(B, params, args, torch):
    """A smaller reduced model of the 16x16x48 cell (the serving model;
    snapshots at three corners of the parameter box over the --rom-steps
    horizon, POD to 1e-7), a timed batched solve of --rom-instances instances
    over --rom-steps steps, its cell-potential error against full-order runs of
    two instances, and the serving run (serve_run)."""
    labels = workload_labels(ROM_CELL)
    opts = B.default_opts(precision=B.PREC_MIXED, newton_tol=1e-10, krylov_rtol=1e-5, max_halvings=3)
    cell = B.Cell(labels, 1e-6, params, opts)
    i1 = cell.i_1c
    t0 = time.perf_counter()
    snap = [(-0.5 * i1, 0.5, 0.1), (-5.0 * i1, 2.0, 10.0), (-2.0 * i1, 1.0, 1.0)]
    rom = B.Rom.build(cell, snap, 1.0, args.rom_steps, ROM_DIMS, pod_tol=1e-7)
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(41)
    prm = _rom_params(rng, args.rom_instances, i1)
    rom.solve(prm[:8], 2, 1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = rom.solve(prm, args.rom_steps, 1.0)
    wall = time.perf_counter() - t0
    inst_steps = args.rom_instances * args.rom_steps
    # cell-potential error of two instances against full-order runs
    errs = []
    for b in range(2):
        fc = B.Cell(labels, 1e-6, params, opts)
        fc.set_scales(prm[b][1], prm[b][2])
        V = []
        for _ in range(args.rom_steps):
            V.append(fc.step(1.0, prm[b][0])["V_cell"])
        fc.close()
        V = np.array(V)
        errs.append(float(np.max(np.abs(out["V"][b][1:] - V)) / np.max(np.abs(V))))
    rom_res = {"workload": "ROM of the %s cell, snapshots at (C-rate, i0 scale, k_pl) = (0.5, 0.5, 0.1), "
                           "(5, 2, 10), (2, 1, 1), %d steps each" % (ROM_CELL, args.rom_steps),
               "dims": {"n_r": rom.n_r, "ei_interface": rom.n_bv, "ei_migration": rom.n_1c,
                        "requested": list(ROM_DIMS)},
               "instances": args.rom_instances, "steps": args.rom_steps, "dt_s": 1.0,
               "precision": "f64 state, reconstruction and residual; f32 Newton matrix and LU",
               "instance_steps_per_s": inst_steps / wall, "solves_per_s": args.rom_instances / wall,
               "wall_s": wall, "build_s": build_s, "newton_its_per_instance_step": out["newton_its"] / inst_steps,
               "failed": out["failed"], "V_rel_err_vs_full_order_2_instances": errs}
    serve = serve_run(B, params, rom, i1, args)
    rom.close()
    cell.close()
    return rom_res, serve


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cell128x128x256")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-coarse", action="store_true",
                    help="smoother and coarse-level products from FP32 operators instead of their BF16 copies")
    ap.add_argument("--mg-stream", type=int, default=3, choices=[0, 1, 2, 3],
                    help="operator fetch of the BF16 coarse sweeps: 0 plain, 1 L2 prefetch, 2 staged in shared memory, "
                         "3 plain at 5 blocks per SM")
    ap.add_argument("--kcycle-cgs1", action="store_true",
                    help="one Gram-Schmidt pass in the level-1 K-cycle instead of two (mg_kcycle_reorth = 0)")
    ap.add_argument("--no-pc-lag", action="store_true",
                    help="rebuild the preconditioner at every Newton iteration (pc_lag = 0)")
    ap.add_argument("--no-newton-rate-test", action="store_true",
                    help="stop Newton only on an update below the tolerance (newton_rate_test = 0)")
    ap.add_argument("--mg-pdl", type=int, default=0, choices=[0, 1],
                    help="programmatic dependent launch of the preconditioner's kernels (mg_pdl)")
    ap.add_argument("--pc-lag-drift", type=float, default=0.05,
                    help="scaled size of the Newton updates after which a lagged preconditioner is rebuilt")
    ap.add_argument("--mg-kcycle", type=int, default=5, help="FGMRES iterations of the level-1 K-cycle")
    ap.add_argument("--mg-smooth", type=int, default=2, help="fine-level sweeps before and after the coarse correction")
    ap.add_argument("--mg-coarse", type=int, nargs=2, default=[2, 2], metavar=("PRE", "POST"),
                    help="sweeps before and after the coarse correction on levels >= 1")
    ap.add_argument("--no-ew", action="store_true",
                    help="every linear solve to krylov_rtol instead of Eisenstat-Walker forcing (krylov_forcing = 0)")
    ap.add_argument("--mg-tail", type=int, default=0,
                    help="coarse V-cycle levels from this one (1: the first that one wave covers) in one persistent "
                         "cooperative launch instead of per-level launches (0: per-level launches)")
    ap.add_argument("--no-fp64-arm", action="store_true",
                    help="skip the FP64 run of the same steps (and the mixed-vs-FP64 errors)")
    ap.add_argument("--no-rom", action="store_true", help="skip the reduced-model and serving measurements")
    ap.add_argument("--rom-instances", type=int, default=4096)
    ap.add_argument("--rom-host-loop", action="store_true",
                    help="reduced steps driven from the host instead of one CUDA graph per step (same results; "
                         "every kernel a separate launch, for a profiler's launch list)")
    ap.add_argument("--rom-steps", type=int, default=60)
    ap.add_argument("--rom-paper-steps", type=int, default=10,
                    help="timed steps of the paper-size reduced model (a sample of its 600-step protocol)")
    ap.add_argument("--serve-requests", type=int, default=800)
    ap.add_argument("--experiment", action="store_true",
                    help="also run the paper's half-cell model-reduction experiment at reduced size "
                         "(paper_1704_04139_gb300.experiment) and add its results under 'experiment'")
    ap.add_argument("--rom-gemm", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="Newton-matrix GEMM of the paper-size reduced model: 2 tcgen05, 1 mma.sync, 0 FP32 FMA "
                         "(-1: the library's choice)")
    ap.add_argument("--rom-only", action="store_true",
                    help="run only the paper-size reduced model (build, timed batch, error check) and print its "
                         "JSON object: the command the reduced-model launch lists are taken with")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, local, ws, dist = _dist()
    torch.cuda.set_device(local)
    import synthetic as syn
    from paper_1704_04139_gb300 import binding as B
    if not os.path.exists(B.LIB_PATH):
        from paper_1704_04139_gb300 import build
        build.build()
    params = syn.load_params()
    if args.rom_only:
        if rank == 0:
            print(json.dumps({"rom": rom_paper_dims(B, params, args, torch, estimate=False)}))
        return 0
    labels = workload_labels(args.workload)
    prec = B.PREC_MIXED if args.precision == "mixed" else B.PREC_FP64
    opts = fom_opts(B, prec, args)
    cell = B.Cell(labels, 1e-6, params, opts)
    I = CRATE[args.workload] * cell.i_1c
    dt = 1.0
    for _ in range(args.warmup):
        cell.step(dt, I)
    u_start = cell.state()          # the timed steps start here; e2e replays them from it
    stream = torch.cuda.ExternalStream(cell.stream_ptr())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    cell.prof_enable(True)
    l0 = cell.launch_count()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(cell.step(dt, I))
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = cell.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    n_jvp, ms_jvp = cell.prof_read(B.Cell.PROF_JVP)
    n_res, ms_res = cell.prof_read(B.Cell.PROF_RESIDUAL)
    n_pc, ms_pc = cell.prof_read(B.Cell.PROF_PRECOND)
    n_sm, ms_sm = cell.prof_read(B.Cell.PROF_SMOOTH)
    n_ls, ms_ls = cell.prof_read(B.Cell.PROF_LSMOOTH)
    cell.prof_enable(False)
    ms = max_over_ranks(ms, dist, "cuda")
    if dist is not None:
        dist.barrier()
    value = whole_job_value(ws, args.steps, dt, ms)
    u_end = cell.state()

    # end to end through the C-ABI with host buffers, on the same steps: the
    # state saved before the timed steps is uploaded from pinned host memory
    # before, and read back after, every step of the replay
    u_host = torch.empty(cell.n, dtype=torch.float64).pin_memory().numpy()
    u_host[:] = u_start
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cell.set_state(u_host)
        cell.step(dt, I)
        cell.state(out=u_host)
    e2e_wall = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": ws * args.steps * dt / e2e_wall, "unit": UNIT,
           "h2d_bytes_per_step": 8 * cell.n, "d2h_bytes_per_step": 8 * cell.n,
           "steps": "the timed steps, replayed from the state saved before them",
           "replay_identical": bool(np.array_equal(u_host, u_end))}

    # roofline of the dominant timed kernel: the fine smoothing sweep k_fine_stencil,
    # the Krylov operator's stencil JVP k_jvp_lin, or the level-1 smoothing sweep
    # k_lvl_smooth of the K-cycle
    peak, peak_kind = measured_peaks()
    N, F, NI = cell.N, cell.F, cell.NI
    cell_levels = cell.debug_levels()
    # algorithmic bytes per launch.  Fine sweep, per voxel: the assembled stencil (14 row blocks of
    # two BF16 = 56 B, or two FP32 = 112 B) + float-float iterate (c, phi) in 16 and out 16 + FP32
    # right-hand side 8 + 2x2 block inverse 16.  Krylov JVP, per voxel: vcode 4 + FP32 c 4 +
    # float-float direction (c, phi) 16 + FP32 result 8 + FP32 row scales 8; per interface face six
    # FP32 partials 24; per plating face float-float direction 8 + result 4 + row scale 4.
    # Level-1 post-smoothing sweep, per coarse cell: the operator rows (six 4x4 couplings, the
    # difference-form self block and the block inverse: 32 rows of four BF16 = 256 B, or 512 B in
    # FP32) + right-hand side 16 + float-float iterate in 32 and out 32; one sweep in two also reads
    # the prolonged level-2 correction (32 B per level-2 cell).
    lv = cell_levels
    c1 = lv[0][0] * lv[0][1] * lv[0][2]
    c2 = lv[1][0] * lv[1][1] * lv[1][2] if len(lv) > 1 else 0
    op_b = 256.0 if opts.mg_bf16 else 512.0
    st_b = 56.0 if opts.mg_bf16 else 112.0
    kinds = {"smoother": (n_sm, ms_sm, (st_b + 56.0) * N,
                          "k_fine_stencil<%s,sweep> (fine smoothing sweep)" % ("bf16" if opts.mg_bf16 else "fp32"),
                          "k_fine_stencil"),
             "operator": (n_jvp, ms_jvp, 40.0 * N + 24.0 * NI + 16.0 * F, "k_jvp_lin (Krylov operator)",
                          "k_jvp_lin"),
             "level1_smoother": (n_ls, ms_ls, (op_b + 80.0) * c1 + 32.0 * c2 / 2.0,
                                 ("k_lvl_smooth_o5 (level-1 post-smoothing sweep, bf16, 5 blocks/SM)"
                                  if (opts.mg_bf16 and args.mg_stream == 3) else
                                  "k_lvl_smooth<%s> (level-1 post-smoothing sweep)" % ("true" if opts.mg_bf16 else "false")),
                                 "k_lvl_smooth_o5" if (opts.mg_bf16 and args.mg_stream == 3) else "k_lvl_smooth")}
    dom = max(kinds, key=lambda k: kinds[k][1])
    n_k, ms_k, bytes_per_launch, kname, kfile = kinds[dom]
    avg_ms = ms_k / max(n_k, 1)
    achieved = bytes_per_launch / (avg_ms / 1000.0) / 1e9 if n_k else None
    roof = {"kernel": kname, "bound": "hbm",
            "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": kernel_traffic(kfile, args.workload, dom),
            "bytes_per_launch": bytes_per_launch, "launches": n_k, "avg_launch_ms": avg_ms,
            "share_of_step": ms_k / ms if ms else None,
            "other": {k: {"launches": v[0], "avg_launch_ms": v[1] / max(v[0], 1),
                          "gbs": (v[2] / (v[1] / max(v[0], 1) / 1000.0) / 1e9) if v[0] else None}
                      for k, v in kinds.items()}}
    # step level: the algorithmic bytes of the three timed kernel classes over the timed steps
    # divided by the timed steps' wall time (a lower bound of the step's HBM use: the other
    # kernels' bytes are not counted)
    step_bytes = sum(v[0] * v[2] for v in kinds.values())
    roof["step"] = {"bytes_counted_per_step": step_bytes / args.steps,
                    "kernels_counted": [v[4] for v in kinds.values()],
                    "share_of_step_time": sum(v[1] for v in kinds.values()) / ms if ms else None,
                    "achieved_gbs": step_bytes / (ms / 1000.0) / 1e9 if ms else None,
                    "frac": step_bytes / (ms / 1000.0) / 1e9 / peak if ms else None}

    cell.close()
    arm64 = None
    if rank == 0 and ws == 1 and prec == B.PREC_MIXED and not args.no_fp64_arm:
        arm64 = fp64_arm(B, labels, params, args, torch, [i["V_cell"] for i in infos], u_end)
    rom = rom_small = serve = None
    if rank == 0 and ws == 1 and not args.no_rom:
        rom = rom_paper_dims(B, params, args, torch)
        rom_small, serve = rom_and_serve(B, params, args, torch)

    experiment = None
    if rank == 0 and ws == 1 and args.experiment:
        from paper_1704_04139_gb300 import experiment as X
        experiment = X.run_study(B, params)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, wall, sample = oracle_sample(labels, params, np.sign(CRATE[args.workload]))
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample, "wall_s": wall}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None,
               "dtype": "f32+f64" if prec == B.PREC_MIXED else "f64", "data": "synthetic",
               "config": {"workload": args.workload, "voxels": int(cell.N), "plating_faces": int(cell.F),
                          "device_bytes": int(cell.device_bytes),
                          "dt_s": dt, "crate": CRATE[args.workload], "precision": args.precision,
                          "coarse_operators": "fp32" if args.fp32_coarse else "bf16", "mg_stream": args.mg_stream,
                          "mg_tail": args.mg_tail, "krylov_forcing": 0 if args.no_ew else 1,
                          "mg_kcycle_reorth": 0 if args.kcycle_cgs1 else 1, "mg_kcycle": args.mg_kcycle,
                          "mg_smooth": args.mg_smooth, "mg_coarse": list(args.mg_coarse),
                          "pc_lag": 0 if args.no_pc_lag else 1, "pc_lag_drift": args.pc_lag_drift,
                          "mg_pdl": args.mg_pdl, "newton_rate_test": 0 if args.no_newton_rate_test else 1,
                          "l2": "working set > 129 MB L2, no flush", "parallelism": "replicas" if ws > 1 else "1 GPU"},
               "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
               "cpu_baseline": cpu,
               "solver": dict(step_record(infos), V_cell=[i["V_cell"] for i in infos],
                              newton_tol=opts.newton_tol, krylov_rtol=opts.krylov_rtol,
                              precond_ms=ms_pc, precond_calls=n_pc, residual_ms=ms_res, residual_calls=n_res),
               "fp64_arm": arm64,
               "rom": rom, "rom_small": rom_small, "serve": serve}
        if experiment is not None:
            out["experiment"] = experiment
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
