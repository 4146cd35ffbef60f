"""The C-ABI library loads and exports every entry point include/mb.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mb_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1704_04139_gb300 import build, binding
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    return binding.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mb_cell_create", "mb_step", "mb_residual", "mb_jvp", "mb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(libpath):
    from paper_1704_04139_gb300 import binding
    lib = binding.lib()
    for n in declared_functions():
        f = getattr(lib, n)
        assert f.restype is not None or n == "mb_opts_default", n


def test_default_options_roundtrip(libpath):
    """The library's defaults are the ones include/mb.h documents."""
    from paper_1704_04139_gb300 import binding
    o = binding.default_opts()
    assert o.precision == binding.PREC_FP64 and o.gmres_m > 0 and o.newton_tol > 0
    want = dict(mg_kcycle=5, mg_coarse_pre=2, mg_coarse_post=2, mg_bf16=1, mg_stream=3, pass_start=1,
                mg_kcycle_reorth=1, krylov_forcing=1, mg_tail=0, pc_lag=1, mg_pdl=0, newton_rate_test=1)
    for k, v in want.items():
        assert getattr(o, k) == v, k
    assert o.pc_lag_drift == 0.05


@pytest.mark.parametrize("field,bad", [("mg_stream", 4), ("mg_tail", 17), ("mg_tail", -1), ("pc_lag", 2),
                                       ("pc_lag_drift", -0.1), ("pc_lag_drift", float("nan")), ("mg_pdl", 2),
                                       ("newton_rate_test", 2), ("krylov_forcing", 2), ("mg_kcycle", 0),
                                       ("mg_kcycle", 17), ("gmres_m", 64), ("newton_tol", 0.0),
                                       ("mg_coarse_pre", 5), ("precision", 2)])
def test_create_rejects_bad_options_without_gpu(libpath, field, bad):
    """Every option is range-checked before any device call."""
    import numpy as np
    import synthetic
    from paper_1704_04139_gb300 import binding
    p = binding.params_from_dict(synthetic.load_params())
    lab = synthetic.slab_1d([4, 1, 0, 2, 5], 2, 2)
    o = binding.default_opts(**{field: bad})
    h = ctypes.c_void_p()
    rc = binding.lib().mb_cell_create(lab.ctypes.data_as(ctypes.c_void_p), lab.shape[0], 2, 2, 1e-6,
                                      ctypes.byref(p), ctypes.byref(o), ctypes.byref(h))
    assert rc == binding.MB_EINVAL
    assert b"solver options" in binding.lib().mb_last_error()


def test_create_rejects_bad_arguments_without_gpu(libpath):
    """Argument checks run before any device call."""
    import numpy as np
    import synthetic
    from paper_1704_04139_gb300 import binding
    p = binding.params_from_dict(synthetic.load_params())
    lab = np.zeros((2, 2, 2), np.uint8)
    lab[0, 0, 0] = 9
    h = ctypes.c_void_p()
    rc = binding.lib().mb_cell_create(lab.ctypes.data_as(ctypes.c_void_p), 2, 2, 2, 1e-6,
                                      ctypes.byref(p), None, ctypes.byref(h))
    assert rc == binding.MB_EINVAL
    assert b"labels" in binding.lib().mb_last_error()


@pytest.mark.parametrize("kind", ["random", "repeated", "gram", "diagonal", "tiny"])
def test_host_eigensolver(libpath, kind):
    """The offline build's symmetric eigensolver (host code) against the
    definition A V = V diag(w), V^T V = I, and against LAPACK's eigenvalues
    (numpy.linalg.eigvalsh), to a few ulps of ||A||: random matrices, a
    spectrum with repeated eigenvalues, a rank-deficient Gram matrix whose
    singular values span 12 decades (the POD's input), diagonal input (no
    reflector, no rotation) and n = 1, 2."""
    import numpy as np
    from paper_1704_04139_gb300 import binding
    rng = np.random.default_rng(5)
    cases = []
    if kind == "random":
        for n in (3, 17, 96):
            X = rng.standard_normal((n, n))
            cases.append(X + X.T)
    elif kind == "repeated":
        Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
        cases.append((Q * np.repeat([3.0, -1.0, 0.0, 2.0], 10)) @ Q.T)
    elif kind == "gram":
        S = rng.standard_normal((600, 30)) @ rng.standard_normal((30, 120)) * np.logspace(0, -12, 120)
        cases.append(S.T @ S)
    elif kind == "diagonal":
        cases.append(np.diag(rng.standard_normal(12)))
    else:
        cases += [np.array([[2.5]]), np.array([[1.0, 2.0], [2.0, -1.0]])]
    for A in cases:
        n = A.shape[0]
        w, V = binding.debug_symeig(A)
        scale = np.max(np.abs(A))
        assert np.max(np.abs(A @ V - V * w)) <= 1e-13 * n * scale
        assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-13 * n
        assert np.max(np.abs(np.sort(w) - np.linalg.eigvalsh(A))) <= 1e-14 * n * scale


def test_host_eigensolver_rejects_bad_arguments(libpath):
    import numpy as np
    from paper_1704_04139_gb300 import binding
    w = np.zeros(1)
    rc = binding.lib().mb_debug_symeig(0, w.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                       w.ctypes.data_as(ctypes.c_void_p))
    assert rc == binding.MB_EINVAL


@pytest.mark.parametrize("name,args", [
    ("mb_cell_destroy", (None,)), ("mb_cell_info_get", (None, None)), ("mb_cell_set_scales", (None, 1.0, 1.0)),
    ("mb_cell_set_opts", (None, None)), ("mb_state_get", (None, None)), ("mb_state_set", (None, None)),
    ("mb_step", (None, 1.0, 0.0, None)), ("mb_adapt_reset", (None,)),
    ("mb_residual", (None, None, None, None, 1.0, 0.0, None)),
    ("mb_rom_solve_batch", (None, 1, None, 1, 1.0, None, None, None, None)), ("mb_rom_dims", (None, None, None, None)),
    ("mb_rom_destroy", (None,)), ("mb_rom_basis", (None, None)), ("mb_serve_create", (None, None)),
    ("mb_serve_submit", (None, None, None)), ("mb_serve_poll", (None, 0, None)), ("mb_serve_destroy", (None,)),
    ("mb_prof_enable", (None, 1)), ("mb_launch_count", (None, None)), ("mb_cell_stream", (None, None)),
    ("mb_residual_dev_noalloc", (None, None, None, 1.0, 0.0, None, None))])
def test_null_arguments_are_rejected_with_a_message(libpath, name, args):
    """A null handle or pointer gives MB_EINVAL and a message naming the call,
    before any device work."""
    from paper_1704_04139_gb300 import binding
    rc = getattr(binding.lib(), name)(*args)
    assert rc == binding.MB_EINVAL
    assert binding.lib().mb_last_error().decode().startswith(name)
