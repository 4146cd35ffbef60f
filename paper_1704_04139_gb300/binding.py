"""ctypes binding of libmb (include/mb.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback.  If
libmb.so has not been built, importing the library raises ``RuntimeError``.
Device-pointer variants accept torch CUDA tensors (their data_ptr is passed
with torch's current stream).
"""
import ctypes as C
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmb.so")

MB_OK, MB_EINVAL, MB_ENOMEM, MB_EBADGEOM, MB_ENOCONV, MB_ECUTOFF, MB_ETIMEOUT, MB_EPENDING, MB_ECUDA = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
PREC_FP64, PREC_MIXED = 0, 1


class MBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libmb error %d: %s" % (code, msg))
        self.code = code


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "F", "R", "T", "clamp_rel", "E_c0", "E_D", "E_kappa", "E_tplus", "E_tdf",
        "G_cmax", "G_D", "G_sigma", "G_i00", "G_x0")] + [("G_ocp", C.c_double * 7)] + [
        (n, C.c_double) for n in ("K_cmax", "K_D", "K_sigma", "K_i00", "K_x0")] + [
        ("K_ocp", C.c_double * 7)] + [(n, C.c_double) for n in (
            "L_sigma", "L_i00", "CN_sigma", "CP_sigma", "Pl_i00", "Pl_layer_m", "Pl_Vm_Li")]


class SolverOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("newton_tol", C.c_double), ("newton_maxit", C.c_int),
                ("gmres_m", C.c_int), ("krylov_maxit", C.c_int), ("krylov_rtol", C.c_double),
                ("max_passes", C.c_int), ("max_halvings", C.c_int), ("mg_coarse_cells", C.c_int),
                ("mg_smooth", C.c_int), ("mg_kcycle", C.c_int), ("mg_coarse_pre", C.c_int),
                ("mg_coarse_post", C.c_int), ("mg_bf16", C.c_int), ("mg_stream", C.c_int),
                ("pass_start", C.c_int), ("mg_kcycle_reorth", C.c_int), ("krylov_forcing", C.c_int),
                ("mg_tail", C.c_int), ("pc_lag", C.c_int), ("pc_lag_drift", C.c_double), ("mg_pdl", C.c_int),
                ("newton_rate_test", C.c_int)]


class StepInfo(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("krylov_its", C.c_int), ("passes", C.c_int),
                ("flips", C.c_int), ("unresolved_flips", C.c_int), ("halvings", C.c_int),
                ("dt_used", C.c_double),
                ("V_cell", C.c_double), ("mean_c_solid", C.c_double), ("Li_total", C.c_double),
                ("Li_anode", C.c_double), ("Li_plated", C.c_double), ("res_norm", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdaptOpts(C.Structure):
    _fields_ = [("tol", C.c_double), ("dt_min", C.c_double), ("dt_max", C.c_double), ("max_rejects", C.c_int)]


class AdaptInfo(C.Structure):
    _fields_ = [("dt_used", C.c_double), ("dt_next", C.c_double), ("err", C.c_double), ("rejects", C.c_int)]


class CellInfo(C.Structure):
    _fields_ = [("n_vox", C.c_int64), ("n_faces", C.c_int64), ("n_unknowns", C.c_int64),
                ("nt", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("i_1c", C.c_double), ("count", C.c_int64 * 6), ("device_bytes", C.c_int64),
                ("n_iface", C.c_int64)]


_lib = None
P_u8 = C.POINTER(C.c_uint8)
P_d = C.POINTER(C.c_double)
P_i32 = C.POINTER(C.c_int32)
VP = C.c_void_p


class RomData(C.Structure):
    _fields_ = [("n_r", C.c_int), ("n_bv", C.c_int), ("n_1c", C.c_int), ("U", VP), ("p_bv", VP), ("p_1c", VP),
                ("Ms", VP), ("Alin", VP), ("bbnd", VP), ("Pbv", VP), ("P1c", VP), ("s_cp", VP), ("s_ac", VP),
                ("a0", VP)]


class RomParams(C.Structure):
    _fields_ = [("I_app", C.c_double), ("s_i0", C.c_double), ("k_pl", C.c_double)]


class RomBuildOpts(C.Structure):
    _fields_ = [("n_params", C.c_int), ("params", VP), ("dt", C.c_double), ("n_steps", C.c_int),
                ("n_c", C.c_int), ("n_n", C.c_int), ("n_phi", C.c_int), ("m_bv", C.c_int), ("m_1c", C.c_int),
                ("pod_tol", C.c_double), ("ei_tol", C.c_double)]


class ServeOpts(C.Structure):
    _fields_ = [("rom", VP), ("fom_labels", VP), ("nt", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double), ("params", VP), ("fom_opts", VP), ("rom_slots", C.c_int),
                ("fom_budget_bytes", C.c_int64), ("fom_workers", C.c_int)]




class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("n_steps", C.c_int), ("t_submit", C.c_double), ("t_start", C.c_double),
                ("t_done", C.c_double), ("V", VP), ("s_ac", VP)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("prm", RomParams), ("n_steps", C.c_int), ("dt", C.c_double),
                ("v_cutoff", C.c_double)]


class RomInfo(C.Structure):
    _fields_ = [("newton_its", C.c_int64), ("flips", C.c_int64), ("failed", C.c_int)]


def _declare(lib):
    def fn(name, res, args):
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    fn("mb_last_error", C.c_char_p, [])
    fn("mb_opts_default", None, [C.POINTER(SolverOpts)])
    fn("mb_cell_create", C.c_int, [VP, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(Params),
                                   C.POINTER(SolverOpts), C.POINTER(VP)])
    fn("mb_cell_destroy", C.c_int, [VP])
    fn("mb_cell_info_get", C.c_int, [VP, C.POINTER(CellInfo)])
    fn("mb_cell_set_scales", C.c_int, [VP, C.c_double, C.c_double])
    fn("mb_cell_set_opts", C.c_int, [VP, C.POINTER(SolverOpts)])
    fn("mb_plating_faces", C.c_int, [VP, VP, VP, VP])
    fn("mb_state_get", C.c_int, [VP, VP])
    fn("mb_state_set", C.c_int, [VP, VP])
    fn("mb_step_adaptive", C.c_int, [VP, C.c_double, C.c_double, C.POINTER(AdaptOpts), C.POINTER(AdaptInfo),
                                     C.POINTER(StepInfo)])
    fn("mb_adapt_reset", C.c_int, [VP])
    fn("mb_step", C.c_int, [VP, C.c_double, C.c_double, C.POINTER(StepInfo)])
    fn("mb_residual", C.c_int, [VP, VP, VP, VP, C.c_double, C.c_double, VP])
    fn("mb_residual_dev", C.c_int, [VP, VP, VP, VP, C.c_double, C.c_double, VP, VP])
    fn("mb_residual_dev_noalloc", C.c_int, [VP, VP, VP, C.c_double, C.c_double, VP, VP])
    fn("mb_rom_create", C.c_int, [VP, C.POINTER(RomData), C.POINTER(VP)])
    fn("mb_rom_destroy", C.c_int, [VP])
    fn("mb_rom_build_pair", C.c_int, [VP, C.POINTER(RomBuildOpts), C.c_double, C.POINTER(VP), C.POINTER(VP)])
    fn("mb_rom_build", C.c_int, [VP, C.POINTER(RomBuildOpts), C.POINTER(VP)])
    fn("mb_serve_create", C.c_int, [C.POINTER(ServeOpts), C.POINTER(VP)])
    fn("mb_serve_submit", C.c_int, [VP, C.POINTER(Request), C.POINTER(C.c_uint64)])
    fn("mb_serve_poll", C.c_int, [VP, C.c_uint64, C.POINTER(Result)])
    fn("mb_serve_destroy", C.c_int, [VP])
    fn("mb_debug_serve_cells", C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64)])
    fn("mb_rom_dims", C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)])
    fn("mb_rom_solve_batch", C.c_int, [VP, C.c_int, C.POINTER(RomParams), C.c_int, C.c_double, VP, VP, VP,
                                        C.POINTER(RomInfo)])
    fn("mb_rom_solve_batch_traj", C.c_int, [VP, C.c_int, C.POINTER(RomParams), C.c_int, C.c_double, VP, VP, VP,
                                             C.POINTER(RomInfo)])
    fn("mb_rom_basis", C.c_int, [VP, VP])
    fn("mb_rom_estimate_batch", C.c_int, [VP, VP, C.c_double, C.c_int, C.POINTER(RomParams), C.c_int, C.c_double,
                                          VP, VP, VP, VP, C.POINTER(RomInfo)])
    fn("mb_rom_block_dims", C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)])
    fn("mb_jvp", C.c_int, [VP, VP, VP, C.c_double, VP, VP])
    fn("mb_jvp_dev", C.c_int, [VP, VP, VP, C.c_double, VP, VP, VP])
    fn("mb_jvp_f32_dev", C.c_int, [VP, VP, VP, C.c_double, VP, VP, VP])
    fn("mb_prof_enable", C.c_int, [VP, C.c_int])
    fn("mb_prof_read", C.c_int, [VP, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)])
    fn("mb_prof_reset", C.c_int, [VP])
    fn("mb_launch_count", C.c_int, [VP, C.POINTER(C.c_int64)])
    fn("mb_cell_stream", C.c_int, [VP, C.POINTER(VP)])
    # inspection hooks (include/mb_debug.h)
    fn("mb_debug_precond", C.c_int, [VP, VP, VP, C.c_double, VP, VP])
    fn("mb_debug_levels", C.c_int, [VP, C.POINTER(C.c_int)])
    fn("mb_debug_level_dims", C.c_int, [VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)])
    fn("mb_debug_level_op", C.c_int, [VP, C.c_int, VP, VP, VP])
    fn("mb_debug_fine", C.c_int, [VP, VP, VP, VP])
    fn("mb_debug_fine_stencil", C.c_int, [VP, VP])
    fn("mb_debug_rom_jac", C.c_int, [C.c_int, C.c_int, C.c_int, VP, VP, VP, VP, VP, C.c_int, VP])
    fn("mb_debug_rom_graph", C.c_int, [VP, C.c_int])
    fn("mb_debug_rom_tensor", C.c_int, [VP, C.c_int])
    fn("mb_debug_rom_gemm_tuning", C.c_int, [VP, C.POINTER(C.c_int), C.POINTER(C.c_float)])
    fn("mb_debug_rom_slot", C.c_int, [VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_float),
                                      C.POINTER(C.c_int)])
    fn("mb_debug_rom_refine", C.c_int, [VP, C.c_int])
    fn("mb_debug_rom_lu", C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, VP, VP, VP])
    fn("mb_debug_residual_split", C.c_int, [VP, VP, VP, VP, C.c_double, C.c_double, VP])
    fn("mb_debug_symeig", C.c_int, [C.c_int, VP, VP, VP])
    return lib


def lib():
    """Load libmb.so (built by ``paper_1704_04139_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmb.so is not built (run paper_1704_04139_gb300/build.py); "
                               "there is no CPU fallback")
        _lib = _declare(C.CDLL(LIB_PATH))
    return _lib


def _check(rc):
    if rc != MB_OK:
        raise MBError(rc, lib().mb_last_error().decode())
    return rc


def params_from_dict(d):
    p = Params()
    p.F, p.R, p.T, p.clamp_rel = d["F"], d["R"], d["T"], d["clamp_rel"]
    e = d["E"]; p.E_c0, p.E_D, p.E_kappa, p.E_tplus, p.E_tdf = e["c0"], e["D"], e["kappa"], e["tplus"], e["tdf"]
    g = d["G"]; p.G_cmax, p.G_D, p.G_sigma, p.G_i00, p.G_x0 = g["cmax"], g["D"], g["sigma"], g["i00"], g["x0"]
    p.G_ocp[:] = g["ocp"]
    k = d["K"]; p.K_cmax, p.K_D, p.K_sigma, p.K_i00, p.K_x0 = k["cmax"], k["D"], k["sigma"], k["i00"], k["x0"]
    p.K_ocp[:] = k["ocp"]
    p.L_sigma, p.L_i00 = d["L"]["sigma"], d["L"]["i00"]
    p.CN_sigma, p.CP_sigma = d["CN"]["sigma"], d["CP"]["sigma"]
    p.Pl_i00, p.Pl_layer_m, p.Pl_Vm_Li = d["Pl"]["i00"], d["Pl"]["layer_m"], d["Pl"]["Vm_Li"]
    return p


def default_opts(**kw):
    o = SolverOpts()
    lib().mb_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(a):
    return a.ctypes.data_as(VP)


def _stream_of(t):
    import torch
    return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


class Cell:
    """A voxel cell resident on the current CUDA device (mb_cell)."""

    def __init__(self, labels, h, params, opts=None):
        labels = np.ascontiguousarray(labels, dtype=np.uint8)
        nt, ny, nz = labels.shape
        self._p = params_from_dict(params) if isinstance(params, dict) else params
        self._o = opts if opts is not None else default_opts()
        h_ = VP()
        _check(lib().mb_cell_create(_ptr(labels), nt, ny, nz, float(h), C.byref(self._p),
                                    C.byref(self._o), C.byref(h_)))
        self.h = h_
        info = CellInfo()
        _check(lib().mb_cell_info_get(self.h, C.byref(info)))
        self.info = info
        self.shape = (nt, ny, nz)
        self.N = info.n_vox
        self.F = info.n_faces
        self.NI = info.n_iface
        self.device_bytes = info.device_bytes
        self.n = info.n_unknowns
        self.i_1c = info.i_1c

    def close(self):
        if getattr(self, "h", None):
            lib().mb_cell_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_scales(self, s_i0=1.0, k_pl=1.0):
        _check(lib().mb_cell_set_scales(self.h, float(s_i0), float(k_pl)))

    def set_opts(self, opts):
        self._o = opts
        _check(lib().mb_cell_set_opts(self.h, C.byref(opts)))

    def plating_faces(self):
        g = np.zeros(self.F, np.int32); e = np.zeros(self.F, np.int32); d = np.zeros(self.F, np.int32)
        _check(lib().mb_plating_faces(self.h, _ptr(g), _ptr(e), _ptr(d)))
        return g, e, d

    def state(self, out=None):
        """The FP64 state; into `out` (a contiguous float64 array of n entries,
        e.g. in pinned memory) when given."""
        u = np.empty(self.n) if out is None else out
        assert u.dtype == np.float64 and u.shape == (self.n,) and u.flags["C_CONTIGUOUS"]
        _check(lib().mb_state_get(self.h, _ptr(u)))
        return u

    def set_state(self, u):
        u = np.ascontiguousarray(u, dtype=np.float64)
        assert u.shape == (self.n,)
        _check(lib().mb_state_set(self.h, _ptr(u)))

    def step(self, dt, I_app):
        info = StepInfo()
        _check(lib().mb_step(self.h, float(dt), float(I_app), C.byref(info)))
        return info.as_dict()

    def step_adaptive(self, dt_try, I_app, tol, dt_min=1e-3, dt_max=60.0, max_rejects=10):
        """One accepted adaptive step (mb_step_adaptive): the step info dict
        plus dt_used, dt_next, err and rejects."""
        o = AdaptOpts(float(tol), float(dt_min), float(dt_max), int(max_rejects))
        ai = AdaptInfo()
        info = StepInfo()
        _check(lib().mb_step_adaptive(self.h, float(dt_try), float(I_app), C.byref(o), C.byref(ai), C.byref(info)))
        out = info.as_dict()
        out.update(dt_used=ai.dt_used, dt_next=ai.dt_next, err=ai.err, rejects=ai.rejects)
        return out

    def adapt_reset(self):
        _check(lib().mb_adapt_reset(self.h))

    def residual(self, u, u_old, dt, I_app, gate=None):
        u = np.ascontiguousarray(u, np.float64); uo = np.ascontiguousarray(u_old, np.float64)
        r = np.empty(self.n)
        g = None if gate is None else np.ascontiguousarray(gate, np.uint8)
        _check(lib().mb_residual(self.h, _ptr(u), _ptr(uo), None if g is None else _ptr(g),
                                 float(dt), float(I_app), _ptr(r)))
        return r

    def debug_residual_split(self, u, u_old, dt, I_app, gate):
        u = np.ascontiguousarray(u, np.float64); uo = np.ascontiguousarray(u_old, np.float64)
        r = np.empty(self.n)
        g = np.ascontiguousarray(gate, np.uint8)
        _check(lib().mb_debug_residual_split(self.h, _ptr(u), _ptr(uo), _ptr(g), float(dt), float(I_app), _ptr(r)))
        return r

    def jvp(self, u, v, dt, gate=None):
        u = np.ascontiguousarray(u, np.float64); v = np.ascontiguousarray(v, np.float64)
        out = np.empty(self.n)
        g = None if gate is None else np.ascontiguousarray(gate, np.uint8)
        _check(lib().mb_jvp(self.h, _ptr(u), None if g is None else _ptr(g), float(dt), _ptr(v), _ptr(out)))
        return out

    # kernel timing (CUDA events on the launching stream) and launch counting
    PROF_JVP, PROF_RESIDUAL, PROF_PRECOND, PROF_SMOOTH, PROF_LSMOOTH = 0, 1, 2, 3, 4

    def prof_enable(self, on=True):
        _check(lib().mb_prof_enable(self.h, 1 if on else 0))

    def prof_read(self, kind):
        n = C.c_int64(); ms = C.c_double()
        _check(lib().mb_prof_read(self.h, int(kind), C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def stream_ptr(self):
        s = VP()
        _check(lib().mb_cell_stream(self.h, C.byref(s)))
        return s.value or 0

    def launch_count(self):
        n = C.c_int64()
        _check(lib().mb_launch_count(self.h, C.byref(n)))
        return n.value

    # inspection hooks of the preconditioner (tests)
    def debug_precond(self, u, gate, dt, r):
        u = np.ascontiguousarray(u, np.float64); r = np.ascontiguousarray(r, np.float64)
        g = np.ascontiguousarray(gate, np.uint8)
        z = np.empty(self.n)
        _check(lib().mb_debug_precond(self.h, _ptr(u), _ptr(g), float(dt), _ptr(r), _ptr(z)))
        return z

    def debug_levels(self):
        n = C.c_int()
        _check(lib().mb_debug_levels(self.h, C.byref(n)))
        out = []
        for l in range(1, n.value + 1):
            a, b, c = C.c_int(), C.c_int(), C.c_int()
            _check(lib().mb_debug_level_dims(self.h, l, C.byref(a), C.byref(b), C.byref(c)))
            out.append((a.value, b.value, c.value))
        return out

    def debug_level_op(self, level):
        dims = self.debug_levels()[level - 1]
        cells = dims[0] * dims[1] * dims[2]
        aself = np.empty((cells, 4, 4), np.float32); off = np.empty((cells, 6, 4, 4), np.float32)
        mask = np.empty(cells, np.uint8)
        _check(lib().mb_debug_level_op(self.h, level, _ptr(aself), _ptr(off), _ptr(mask)))
        return dims, aself, off, mask

    def debug_fine(self):
        dinv = np.empty((self.N, 2, 2), np.float32); fc = np.empty((max(self.F, 1), 8), np.float32)
        rowdiag = np.empty(self.n, np.float32)
        _check(lib().mb_debug_fine(self.h, _ptr(dinv), _ptr(fc), _ptr(rowdiag)))
        return dinv, fc[:self.F], rowdiag

    def debug_fine_stencil(self):
        out = np.empty((14, self.N, 2), np.float32)
        _check(lib().mb_debug_fine_stencil(self.h, _ptr(out)))
        return out

    # device-pointer variants (torch CUDA tensors)
    def residual_dev(self, u, u_old, dt, I_app, r, gate=None):
        _check(lib().mb_residual_dev(self.h, VP(u.data_ptr()), VP(u_old.data_ptr()),
                                     None if gate is None else VP(gate.data_ptr()), float(dt),
                                     float(I_app), VP(r.data_ptr()), _stream_of(u)))

    def residual_dev_noalloc(self, u, u_old, dt, I_app, r):
        _check(lib().mb_residual_dev_noalloc(self.h, VP(u.data_ptr()), VP(u_old.data_ptr()), float(dt),
                                             float(I_app), VP(r.data_ptr()), _stream_of(u)))

    def jvp_dev(self, u, v, dt, out, gate=None):
        _check(lib().mb_jvp_dev(self.h, VP(u.data_ptr()), None if gate is None else VP(gate.data_ptr()),
                                float(dt), VP(v.data_ptr()), VP(out.data_ptr()), _stream_of(u)))

    def jvp_f32_dev(self, u, v, dt, out, gate):
        _check(lib().mb_jvp_f32_dev(self.h, VP(u.data_ptr()), VP(gate.data_ptr()), float(dt),
                                    VP(v.data_ptr()), VP(out.data_ptr()), _stream_of(u)))


class Rom:
    """Reduced model of a cell (mb_rom_create): arrays in the layout of
    include/mb.h (row-major FP64; points as residual-row indices)."""

    @classmethod
    def build(cls, cell, params, dt, n_steps, dims, pod_tol=1e-7, ei_tol=1e-12):
        """mb_rom_build: params = [(I_app, s_i0, k_pl), ...], dims = (n_c, n_n, n_phi, m_bv, m_1c)."""
        prm = (RomParams * len(params))(*[RomParams(*map(float, p)) for p in params])
        o = RomBuildOpts(len(params), C.cast(prm, VP), float(dt), int(n_steps), *[int(x) for x in dims],
                         float(pod_tol), float(ei_tol))
        h = VP()
        _check(lib().mb_rom_build(cell.h, C.byref(o), C.byref(h)))
        self = cls.__new__(cls)
        self.h = h
        self.cell = cell
        self._keep = []
        nr, nb, n1 = C.c_int(), C.c_int(), C.c_int()
        _check(lib().mb_rom_dims(h, C.byref(nr), C.byref(nb), C.byref(n1)))
        self.n_r, self.n_bv, self.n_1c = nr.value, nb.value, n1.value
        return self

    @classmethod
    def build_pair(cls, cell, params, dt, n_steps, dims, frac=0.97, pod_tol=1e-7, ei_tol=1e-12):
        """mb_rom_build_pair: (reduced, validation) models from one snapshot set,
        the reduced one keeping ceil(frac x) of each validation space."""
        prm = (RomParams * len(params))(*[RomParams(*map(float, p)) for p in params])
        o = RomBuildOpts(len(params), C.cast(prm, VP), float(dt), int(n_steps), *[int(x) for x in dims],
                         float(pod_tol), float(ei_tol))
        hr, hv = VP(), VP()
        _check(lib().mb_rom_build_pair(cell.h, C.byref(o), float(frac), C.byref(hr), C.byref(hv)))
        out = []
        for h in (hr, hv):
            self = cls.__new__(cls)
            self.h = h
            self.cell = cell
            self._keep = []
            nr, nb, n1 = C.c_int(), C.c_int(), C.c_int()
            _check(lib().mb_rom_dims(h, C.byref(nr), C.byref(nb), C.byref(n1)))
            self.n_r, self.n_bv, self.n_1c = nr.value, nb.value, n1.value
            out.append(self)
        return out[0], out[1]

    def __init__(self, cell, U, p_bv, p_1c, Ms, Alin, bbnd, Pbv, P1c, s_cp, s_ac, a0):
        f64 = lambda a: np.ascontiguousarray(a, np.float64)
        i64 = lambda a: np.ascontiguousarray(a, np.int64)
        self._keep = [f64(U), i64(p_bv), i64(p_1c), f64(Ms), f64(Alin), f64(bbnd), f64(Pbv), f64(P1c),
                      f64(s_cp), f64(s_ac), f64(a0)]
        U_, pb, pc, Ms_, Al, bb, Pb, Pc, sc, sa, a0_ = self._keep
        self.n_r = U_.shape[1]
        d = RomData(self.n_r, len(pb), len(pc), _ptr(U_), _ptr(pb), _ptr(pc), _ptr(Ms_), _ptr(Al), _ptr(bb),
                    _ptr(Pb), _ptr(Pc), _ptr(sc), _ptr(sa), _ptr(a0_))
        h = VP()
        _check(lib().mb_rom_create(cell.h, C.byref(d), C.byref(h)))
        self.h = h
        self.cell = cell

    def solve(self, params, n_steps, dt):
        """params: sequence of (I_app, s_i0, k_pl).  Returns dict V (B, n_steps+1),
        s_ac, a (B, n_r) and the Newton/flip/failure counts."""
        B = len(params)
        prm = (RomParams * B)(*[RomParams(*map(float, p)) for p in params])
        V = np.empty((B, n_steps + 1))
        S = np.empty((B, n_steps + 1))
        A = np.empty((B, self.n_r))
        info = RomInfo()
        rc = lib().mb_rom_solve_batch(self.h, B, prm, int(n_steps), float(dt), _ptr(V), _ptr(S), _ptr(A),
                                      C.byref(info))
        out = dict(V=V, s_ac=S, a=A, newton_its=int(info.newton_its), flips=int(info.flips),
                   failed=int(info.failed))
        if rc != 0 and rc != -4:
            _check(rc)
        out["ok"] = rc == 0
        return out

    def solve_traj(self, params, n_steps, dt):
        """As solve, with the coefficients of every step: a (B, n_steps+1, n_r)."""
        B = len(params)
        prm = (RomParams * B)(*[RomParams(*map(float, p)) for p in params])
        V = np.empty((B, n_steps + 1))
        S = np.empty((B, n_steps + 1))
        A = np.empty((B, n_steps + 1, self.n_r))
        info = RomInfo()
        rc = lib().mb_rom_solve_batch_traj(self.h, B, prm, int(n_steps), float(dt), _ptr(V), _ptr(S), _ptr(A),
                                           C.byref(info))
        if rc != 0 and rc != -4:
            _check(rc)
        return dict(V=V, s_ac=S, a=A, newton_its=int(info.newton_its), failed=int(info.failed), ok=rc == 0)

    def basis(self, n):
        """The reduced basis U (n, n_r) in the full state layout."""
        U = np.empty((n, self.n_r))
        _check(lib().mb_rom_basis(self.h, _ptr(U)))
        return U

    def estimate(self, val, params, n_steps, dt, theta=0.0):
        """Hierarchical error estimate against the validation model `val`
        (mb_rom_estimate_batch).  Returns dict est (B, n_steps+1, 3: c, phi,
        n), V and V_val (B, n_steps+1) and the counts."""
        B = len(params)
        prm = (RomParams * B)(*[RomParams(*map(float, p)) for p in params])
        est = np.empty((B, n_steps + 1, 3))
        nrm = np.empty((B, n_steps + 1, 3))
        V = np.empty((B, n_steps + 1))
        Vv = np.empty((B, n_steps + 1))
        info = RomInfo()
        rc = lib().mb_rom_estimate_batch(self.h, val.h, float(theta), B, prm, int(n_steps), float(dt), _ptr(V),
                                         _ptr(Vv), _ptr(est), _ptr(nrm), C.byref(info))
        if rc != 0 and rc != -4:
            _check(rc)
        return dict(est=est, norm_val=nrm, V=V, V_val=Vv, newton_its=int(info.newton_its),
                    failed=int(info.failed), ok=rc == 0)

    def block_dims(self):
        """(n_c, n_n, n_phi): reduced modes by field."""
        a, b_, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().mb_rom_block_dims(self.h, C.byref(a), C.byref(b_), C.byref(c)))
        return a.value, b_.value, c.value

    def debug_refine(self, on):
        """Escalated instances by GMRES preconditioned with the FP32 LU (on, the default) or the FP64 LU (off)."""
        _check(lib().mb_debug_rom_refine(self.h, 1 if on else 0))

    def debug_graph(self, on):
        _check(lib().mb_debug_rom_graph(self.h, int(bool(on))))

    def debug_tensor(self, on):
        """Fix the Newton-matrix GEMM variant: 2 tcgen05, 1 mma.sync (both 3xTF32), 0 FP32 FMA
        (default: autotuned per batch shape)."""
        _check(lib().mb_debug_rom_tensor(self.h, int(on)))

    def debug_slot(self, b):
        """(failed 0/1 limit/2 non-finite, iterations of the last pass, last scaled update norm, escalated)."""
        f, it, e = C.c_int(), C.c_int(), C.c_int()
        nrm = C.c_float()
        _check(lib().mb_debug_rom_slot(self.h, int(b), C.byref(f), C.byref(it), C.byref(nrm), C.byref(e)))
        return f.value, it.value, nrm.value, e.value

    def gemm_tuning(self):
        """(variant in use, ms per launch of variants 0, 1, 2 at the last autotuning; -1 = not timed)."""
        ch = C.c_int()
        ms = (C.c_float * 3)()
        _check(lib().mb_debug_rom_gemm_tuning(self.h, C.byref(ch), ms))
        return ch.value, [float(x) for x in ms]

    def close(self):
        if getattr(self, "h", None):
            lib().mb_rom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


REQ_ROM, REQ_FOM = 0, 1


class Server:
    """Serving loop (mb_serve_*): reduced-model requests in a resident slot
    batch, full-order requests on worker threads."""

    def __init__(self, rom=None, labels=None, h=1e-6, params=None, fom_opts=None, rom_slots=64,
                 fom_budget_bytes=8 << 30, fom_workers=1):
        self._keep = []
        lab = None
        nt = ny = nz = 0
        prm_p = None
        fo_p = None
        if labels is not None:
            lab = np.ascontiguousarray(labels, np.uint8)
            nt, ny, nz = lab.shape
            pr = params_from_dict(params) if isinstance(params, dict) else params
            self._keep += [lab, pr]
            prm_p = C.cast(C.pointer(pr), VP)
            if fom_opts is not None:
                self._keep.append(fom_opts)
                fo_p = C.cast(C.pointer(fom_opts), VP)
        o = ServeOpts(rom.h if rom is not None else None, _ptr(lab) if lab is not None else None, nt, ny, nz,
                      float(h), prm_p, fo_p, int(rom_slots), int(fom_budget_bytes), int(fom_workers))
        hnd = VP()
        _check(lib().mb_serve_create(C.byref(o), C.byref(hnd)))
        self.h = hnd
        self._n = {}

    def submit(self, kind, I_app, s_i0, k_pl, n_steps, dt, v_cutoff=0.0):
        r = Request(int(kind), RomParams(float(I_app), float(s_i0), float(k_pl)), int(n_steps), float(dt),
                    float(v_cutoff))
        t = C.c_uint64()
        _check(lib().mb_serve_submit(self.h, C.byref(r), C.byref(t)))
        self._n[t.value] = int(n_steps)
        return t.value

    def poll(self, ticket):
        """None while pending, else dict(status, V, s_ac, t_submit, t_start, t_done)."""
        n = self._n[ticket]
        V = np.full(n + 1, np.nan)
        S = np.full(n + 1, np.nan)
        res = Result(0, 0, 0.0, 0.0, 0.0, _ptr(V), _ptr(S))
        rc = lib().mb_serve_poll(self.h, C.c_uint64(ticket), C.byref(res))
        if rc == -7:
            return None
        _check(rc)
        del self._n[ticket]
        return dict(status=res.status, n_steps=res.n_steps, V=V, s_ac=S, t_submit=res.t_submit,
                    t_start=res.t_start, t_done=res.t_done)

    def debug_cells(self):
        """(alive, peak, cell_bytes) of the server's full-order cells."""
        a, p, cb = C.c_int(), C.c_int(), C.c_int64()
        _check(lib().mb_debug_serve_cells(self.h, C.byref(a), C.byref(p), C.byref(cb)))
        return a.value, p.value, cb.value

    def close(self):
        if getattr(self, "h", None):
            lib().mb_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_rom_jac(P, GU, Ms, Alin, dt_inv, tc=True):
    """The reduced model's Newton-matrix kernel on given arrays: J[b] = P GU[b] +
    Ms dt_inv[b] + Alin (GU shape (B, M, Nr)); tc: 2 the tcgen05 kernel (TMEM
    accumulator), 1 (or True) the mma.sync tensor-core kernel, 0 FP32 FMA."""
    P = np.ascontiguousarray(P, dtype=np.float32)
    Nr, M = P.shape
    B = len(dt_inv)
    gu = np.ascontiguousarray(np.transpose(np.asarray(GU, dtype=np.float32), (1, 0, 2)).reshape(M, B * Nr))
    ms = np.ascontiguousarray(Ms, dtype=np.float32)
    al = np.ascontiguousarray(Alin, dtype=np.float32)
    dti = np.ascontiguousarray(dt_inv, dtype=np.float64)
    J = np.empty((B, Nr, Nr), dtype=np.float32)
    _check(lib().mb_debug_rom_jac(Nr, M, B, _ptr(P), _ptr(gu), _ptr(ms), _ptr(al), _ptr(dti), int(tc), _ptr(J)))
    return J


def debug_symeig(A):
    """The offline build's symmetric eigensolver on a host matrix: (w, V)
    with A = V diag(w) V^T, eigenvalues unordered."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    _check(lib().mb_debug_symeig(n, _ptr(A), _ptr(w), _ptr(V)))
    return w, V


def debug_rom_lu(J, r, fp64=True, in_place=False):
    """The reduced model's Newton-step LU kernel: delta[b] = -J[b]^-1 r[b] (J shape (B, Nr, Nr))."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    B, Nr = r.shape
    delta = np.empty((B, Nr))
    _check(lib().mb_debug_rom_lu(Nr, B, 1 if fp64 else 0, 1 if in_place else 0, _ptr(J), _ptr(r), _ptr(delta)))
    return delta

