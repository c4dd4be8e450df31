"""ctypes binding of libmasw (the C ABI declared in ``include/masw.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library. Functions carry the C names without the ``masw_`` prefix. Inputs
and outputs may be numpy arrays (host memory) or torch tensors (host or
device); device pointers and the current torch stream are passed straight
through. Loading fails loudly when the library is missing and cannot be
built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, EADMIT, ECUDA, ETIMEOUT, EAGAIN = 0, 1, 2, 3, 4, 5, 6
FOUND, NO_ROOT = 0, 1
HOST, DEVICE = 0, 1
MISFIT_PAPER, MISFIT_LSQ = 0, 1
MAX_LAYERS = 128

_lib = None


class MaswError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (code {code})")


class ModelsDesc(ctypes.Structure):
    _fields_ = [("n_models", ctypes.c_int32), ("n_layers", ctypes.c_void_p),
                ("h", ctypes.c_void_p), ("alpha", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("rho", ctypes.c_void_p), ("n_lambda", ctypes.c_void_p),
                ("lambda_", ctypes.c_void_p), ("mem_space", ctypes.c_int32)]


class GridDesc(ctypes.Structure):
    _fields_ = [("c0", ctypes.c_double), ("dc", ctypes.c_double), ("n_c", ctypes.c_int32)]


class Plan(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("cpl", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("ordered", ctypes.c_int32), ("stage_layers", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("count_block", ctypes.c_int32), ("count_split", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


def library_path() -> str:
    return _build.SO


def load():
    """Load libmasw.so, building it first when a source is newer."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmasw not found at {path}")
    lib = ctypes.CDLL(path)
    p, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "masw_model_batch_create": [ctypes.POINTER(ModelsDesc), ctypes.POINTER(GridDesc), p,
                                    ctypes.POINTER(p)],
        "masw_model_batch_destroy": [p],
        "masw_model_batch_update": [p, p, p, p, p, i32],
        "masw_batch_info": [p, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i32)],
        "masw_dispersion": [p, p, p, p, i32],
        "masw_dispersion_plain": [p, p, p, p, i32],
        "masw_dispersion_changes": [p, i32, p, p, p, p, i32],
        "masw_dispersion_leaky": [p, p, p, p, i32],
        "masw_mode_count": [p, i32, p, p, p, p],
        "masw_set_route": [p, i32],
        "masw_test_fail_alloc": [i32],
        "masw_misfit": [p, p, i32, d, p],
        "masw_misfit_grad": [p, p, i32, d, p, p, p],
        "masw_roots": [p, p],
        "masw_root_grad": [p, p, ctypes.POINTER(i64)],
        "masw_det_eval": [p, i32, p, p, p, p],
        "masw_get_plan": [p, ctypes.POINTER(Plan)],
        "masw_set_plan": [p, ctypes.POINTER(Plan)],
        "masw_autotune": [p, i32, ctypes.POINTER(Plan)],
        "masw_last_scan_ms": [p, ctypes.POINTER(ctypes.c_float)],
        "masw_fp64_peak": [p, ctypes.POINTER(d)],
        "masw_sm_count": [ctypes.POINTER(i32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.masw_strerror.argtypes = [ctypes.c_int]
    lib.masw_strerror.restype = ctypes.c_char_p
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().masw_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != OK:
        raise MaswError(rc, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data_as(ctypes.c_void_p)


def _space(x) -> int:
    return DEVICE if (_is_torch(x) and x.is_cuda) else HOST


def _stream_handle(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


# ------------------------------------------------------------ C names

def model_batch_create(n_layers, h, alpha, beta, rho, n_lambda, lam, grid, stream=None):
    """masw_model_batch_create; returns an opaque handle (int)."""
    lib = load()
    space = _space(h if h is not None else beta)
    keep = [n_layers, h, alpha, beta, rho, n_lambda, lam]
    desc = ModelsDesc(int(len(n_layers)), _ptr(n_layers), _ptr(h), _ptr(alpha), _ptr(beta),
                      _ptr(rho), _ptr(n_lambda), _ptr(lam), space)
    g = GridDesc(float(grid[0]), float(grid[1]), int(grid[2]))
    out = ctypes.c_void_p()
    _check(lib.masw_model_batch_create(ctypes.byref(desc), ctypes.byref(g), _stream_handle(stream),
                                       ctypes.byref(out)), "masw_model_batch_create")
    del keep
    return out.value


def model_batch_destroy(handle):
    _check(load().masw_model_batch_destroy(ctypes.c_void_p(handle)), "masw_model_batch_destroy")


def model_batch_update(handle, h, alpha, beta, rho):
    _check(load().masw_model_batch_update(ctypes.c_void_p(handle), _ptr(h), _ptr(alpha),
                                          _ptr(beta), _ptr(rho), _space(beta)),
           "masw_model_batch_update")


def model_batch_update_beta_h(handle, h, beta):
    """masw_model_batch_update_beta_h: new beta and h, Poisson ratio and
    density held."""
    f = load().masw_model_batch_update_beta_h
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(handle), _ptr(h), _ptr(beta)), "masw_model_batch_update_beta_h")


def batch_info(handle):
    n_items, n_models, max_layers = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().masw_batch_info(ctypes.c_void_p(handle), ctypes.byref(n_items),
                                  ctypes.byref(n_models), ctypes.byref(max_layers)),
           "masw_batch_info")
    return n_items.value, n_models.value, max_layers.value


def dispersion(handle, ct, ct_idx, status):
    space = _space(next(x for x in (ct, ct_idx, status) if x is not None))
    _check(load().masw_dispersion(ctypes.c_void_p(handle), _ptr(ct), _ptr(ct_idx), _ptr(status),
                                  space), "masw_dispersion")


def dispersion_plain(handle, ct, ct_idx, status):
    space = _space(next(x for x in (ct, ct_idx, status) if x is not None))
    _check(load().masw_dispersion_plain(ctypes.c_void_p(handle), _ptr(ct), _ptr(ct_idx),
                                        _ptr(status), space), "masw_dispersion_plain")


MAX_CHANGES = 15


def dispersion_changes(handle, max_changes, ct, ct_idx, status, delta_count):
    """Algorithm 1 continued: the first max_changes sign changes per item
    with the change in K's negative-eigenvalue count across each
    (masw_dispersion_changes); outputs [n_items * max_changes]."""
    space = _space(next(x for x in (ct, ct_idx, status, delta_count) if x is not None))
    _check(load().masw_dispersion_changes(ctypes.c_void_p(handle), int(max_changes), _ptr(ct),
                                          _ptr(ct_idx), _ptr(status), _ptr(delta_count), space),
           "masw_dispersion_changes")


def dispersion_leaky(handle, ct, ct_idx, status):
    """Algorithm 1 over the whole grid with the sign of Re det K (complex
    half-space block at and above its shear speed; masw_dispersion_leaky)."""
    space = _space(next(x for x in (ct, ct_idx, status) if x is not None))
    _check(load().masw_dispersion_leaky(ctypes.c_void_p(handle), _ptr(ct), _ptr(ct_idx),
                                        _ptr(status), space), "masw_dispersion_leaky")


def misfit(handle, ce, kind, sigma, out):
    _check(load().masw_misfit(ctypes.c_void_p(handle), _ptr(ce), int(kind), float(sigma),
                              _ptr(out)), "masw_misfit")


def misfit_curves(handle, ce, kind, sigma, out, ct, ct_idx, status):
    """masw_misfit_curves: Algorithm 1 + Algorithm 2 with the curves and the
    misfit returned together (each buffer host or device)."""
    f = load().masw_misfit_curves
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(handle), _ptr(ce), int(kind), float(sigma), _ptr(out), _ptr(ct),
             _ptr(ct_idx), _ptr(status)), "masw_misfit_curves")


def misfit_grad(handle, ce, kind, sigma, out, grad_beta, grad_h):
    _check(load().masw_misfit_grad(ctypes.c_void_p(handle), _ptr(ce), int(kind), float(sigma),
                                   _ptr(out), _ptr(grad_beta), _ptr(grad_h)), "masw_misfit_grad")


def roots(handle, croot):
    _check(load().masw_roots(ctypes.c_void_p(handle), _ptr(croot)), "masw_roots")


def root_grad(handle, rows=None) -> int:
    total = ctypes.c_int64()
    _check(load().masw_root_grad(ctypes.c_void_p(handle), _ptr(rows), ctypes.byref(total)),
           "masw_root_grad")
    return total.value


def det_eval(handle, item, c, sign, log_abs):
    _check(load().masw_det_eval(ctypes.c_void_p(handle), int(len(item)), _ptr(item), _ptr(c),
                                _ptr(sign), _ptr(log_abs)), "masw_det_eval")


def mode_count(handle, item, c, s, j0):
    """Wittrick-Williams counts (s, J0) at arbitrary points (masw_mode_count)."""
    _check(load().masw_mode_count(ctypes.c_void_p(handle), int(len(item)), _ptr(item), _ptr(c),
                                  _ptr(s), _ptr(j0)), "masw_mode_count")


def test_fail_alloc(k: int):
    """Test hook: the k-th next device allocation fails (masw_test_fail_alloc)."""
    _check(load().masw_test_fail_alloc(int(k)), "masw_test_fail_alloc")


def set_route(handle, route: int):
    """Test routing through the slower paths (masw_set_route)."""
    _check(load().masw_set_route(ctypes.c_void_p(handle), int(route)), "masw_set_route")


def get_plan(handle) -> Plan:
    p = Plan()
    _check(load().masw_get_plan(ctypes.c_void_p(handle), ctypes.byref(p)), "masw_get_plan")
    return p


def set_plan(handle, plan: Plan):
    _check(load().masw_set_plan(ctypes.c_void_p(handle), ctypes.byref(plan)), "masw_set_plan")


def autotune(handle, reps: int = 2) -> Plan:
    p = Plan()
    _check(load().masw_autotune(ctypes.c_void_p(handle), int(reps), ctypes.byref(p)),
           "masw_autotune")
    return p


def last_scan_ms(handle) -> float:
    ms = ctypes.c_float()
    _check(load().masw_last_scan_ms(ctypes.c_void_p(handle), ctypes.byref(ms)), "masw_last_scan_ms")
    return ms.value


def last_scan_phases(handle):
    f = load().masw_last_scan_phases
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    f.restype = ctypes.c_int
    ms = (ctypes.c_float * 3)()
    _check(f(ctypes.c_void_p(handle), ms), "masw_last_scan_phases")
    return [ms[0], ms[1], ms[2]]


def last_count_phases(handle):
    """(FP32 counting search, FP64 certificate, fallback chain on the second
    stream or 0) device ms of the last scan (masw_last_count_phases; split
    counting plan, no graph)."""
    f = load().masw_last_count_phases
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]
    f.restype = ctypes.c_int
    ms = (ctypes.c_float * 3)()
    _check(f(ctypes.c_void_p(handle), ms), "masw_last_count_phases")
    return [ms[0], ms[1], ms[2]]


def last_scan_screen(handle, n32):
    f = load().masw_last_scan_screen
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(handle), _ptr(n32)), "masw_last_scan_screen")


def last_scan_unresolved(handle) -> int:
    f = load().masw_last_scan_unresolved
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    n = ctypes.c_int32()
    _check(f(ctypes.c_void_p(handle), ctypes.byref(n)), "masw_last_scan_unresolved")
    return n.value


def last_changes_linear(handle) -> int:
    f = load().masw_last_changes_linear
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    n = ctypes.c_int32()
    _check(f(ctypes.c_void_p(handle), ctypes.byref(n)), "masw_last_changes_linear")
    return n.value


def last_scan_fallback(handle) -> int:
    f = load().masw_last_scan_fallback
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]
    f.restype = ctypes.c_int
    n = ctypes.c_int32()
    _check(f(ctypes.c_void_p(handle), ctypes.byref(n)), "masw_last_scan_fallback")
    return n.value


def exp_check(x, stream=None):
    """(library e^x, CUDA exp(x)) at host points x <= 0 (masw_exp_check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y_lib = np.empty_like(x)
    y_cuda = np.empty_like(x)
    f = load().masw_exp_check
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(x.size, _ptr(x), _ptr(y_lib), _ptr(y_cuda), _stream_handle(stream)), "masw_exp_check")
    return y_lib, y_cuda


def sincos_check(x, stream=None):
    """(library sin, cos, CUDA sin, cos) at host points 0 <= x <= 5 pi / 4
    (masw_sincos_check)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    outs = [np.empty_like(x) for _ in range(4)]
    f = load().masw_sincos_check
    f.argtypes = [ctypes.c_int32] + [ctypes.c_void_p] * 6
    f.restype = ctypes.c_int
    _check(f(x.size, _ptr(x), *[_ptr(o) for o in outs], _stream_handle(stream)),
           "masw_sincos_check")
    return tuple(outs)


def element_check(handle, item, layer, c, dd_trig=False):
    """(fp64, df): the element's denominator and six numerators (7 per point)
    from the FP64 element and the double-float one (masw_element_check;
    dd_trig: the leaky continuation's, trigonometric branch in double-float)."""
    item = np.ascontiguousarray(item, dtype=np.int32)
    layer = np.ascontiguousarray(layer, dtype=np.int32)
    c = np.ascontiguousarray(c, dtype=np.float64)
    fp = np.empty((item.size, 7))
    df = np.empty((item.size, 7))
    f = load().masw_element_check
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int32] + [ctypes.c_void_p] * 2
    f.restype = ctypes.c_int
    _check(f(ctypes.c_void_p(handle), item.size, _ptr(item), _ptr(layer), _ptr(c),
             int(bool(dd_trig)), _ptr(fp), _ptr(df)), "masw_element_check")
    return fp, df


def fp64_peak(stream=None) -> float:
    f = ctypes.c_double()
    _check(load().masw_fp64_peak(_stream_handle(stream), ctypes.byref(f)), "masw_fp64_peak")
    return f.value


def sm_count() -> int:
    n = ctypes.c_int32()
    _check(load().masw_sm_count(ctypes.byref(n)), "masw_sm_count")
    return n.value


# ------------------------------------------------------- convenience

class Batch:
    """Owning wrapper of a masw_batch built from a ``workloads.Models``.

    ``device=True`` uploads the model arrays as torch CUDA tensors first
    (exercising the device-pointer path of the ABI)."""

    def __init__(self, models, grid, stream=None, device: bool = False):
        arrs = [np.ascontiguousarray(models.n_layers, dtype=np.int32),
                np.ascontiguousarray(models.h, dtype=np.float64),
                np.ascontiguousarray(models.alpha, dtype=np.float64),
                np.ascontiguousarray(models.beta, dtype=np.float64),
                np.ascontiguousarray(models.rho, dtype=np.float64),
                np.ascontiguousarray(models.n_lambda, dtype=np.int32),
                np.ascontiguousarray(models.lam, dtype=np.float64)]
        if device:
            import torch
            arrs = [torch.from_numpy(a).cuda() for a in arrs]
        g = (grid.c0, grid.dc, grid.n_c) if hasattr(grid, "c0") else tuple(grid)
        self.handle = model_batch_create(*arrs, g, stream=stream)
        self.n_items, self.n_models, self.max_layers = batch_info(self.handle)
        self.models = models
        self.grid = g

    def close(self):
        if self.handle:
            model_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # host-output helpers
    def dispersion(self, plain: bool = False):
        ct = np.empty(self.n_items)
        idx = np.empty(self.n_items, dtype=np.int32)
        st = np.empty(self.n_items, dtype=np.int32)
        (dispersion_plain if plain else dispersion)(self.handle, ct, idx, st)
        return ct, idx, st

    def changes(self, max_changes: int):
        """(ct, idx, status, delta_count), each of shape (n_items, max_changes)."""
        shape = (self.n_items, int(max_changes))
        ct = np.empty(shape)
        idx = np.empty(shape, dtype=np.int32)
        st = np.empty(shape, dtype=np.int32)
        dl = np.empty(shape, dtype=np.int32)
        dispersion_changes(self.handle, max_changes, ct, idx, st, dl)
        return ct, idx, st, dl

    def leaky(self):
        """(ct, idx, status) of the whole-grid scan with the sign of Re det K."""
        ct = np.empty(self.n_items)
        idx = np.empty(self.n_items, dtype=np.int32)
        st = np.empty(self.n_items, dtype=np.int32)
        dispersion_leaky(self.handle, ct, idx, st)
        return ct, idx, st

    def roots(self):
        out = np.empty(self.n_items)
        roots(self.handle, out)
        return out

    def root_grad(self):
        n = root_grad(self.handle, None)
        rows = np.empty(max(n, 1))
        root_grad(self.handle, rows)
        return rows[:n]

    def misfit(self, ce, kind=MISFIT_LSQ, sigma=2.0):
        out = np.empty(self.n_models)
        misfit(self.handle, np.ascontiguousarray(ce, dtype=np.float64), kind, sigma, out)
        return out

    def misfit_curves(self, ce, kind=MISFIT_LSQ, sigma=2.0):
        """(misfit, ct, idx, status) from one evaluation."""
        out = np.empty(self.n_models)
        ct = np.empty(self.n_items)
        idx = np.empty(self.n_items, dtype=np.int32)
        st = np.empty(self.n_items, dtype=np.int32)
        misfit_curves(self.handle, np.ascontiguousarray(ce, dtype=np.float64), kind, sigma, out,
                      ct, idx, st)
        return out, ct, idx, st

    def misfit_grad(self, ce, kind=MISFIT_LSQ, sigma=2.0):
        n_rec = int(np.sum(self.models.n_layers) + self.n_models)
        out = np.empty(self.n_models)
        gb = np.empty(n_rec)
        gh = np.empty(max(n_rec - self.n_models, 1))
        misfit_grad(self.handle, np.ascontiguousarray(ce, dtype=np.float64), kind, sigma, out, gb, gh)
        return out, gb, gh[:n_rec - self.n_models]

    def det_eval(self, item, c):
        item = np.ascontiguousarray(item, dtype=np.int32)
        c = np.ascontiguousarray(c, dtype=np.float64)
        sign = np.empty(item.size, dtype=np.int32)
        la = np.empty(item.size)
        det_eval(self.handle, item, c, sign, la)
        return sign, la

    def set_route(self, route: int):
        set_route(self.handle, route)

    def mode_count(self, item, c):
        """(s, J0) at the points: negative eigenvalues of K and clamped-layer modes."""
        item = np.ascontiguousarray(item, dtype=np.int32)
        c = np.ascontiguousarray(c, dtype=np.float64)
        s = np.empty(item.size, dtype=np.int32)
        j0 = np.empty(item.size, dtype=np.int32)
        mode_count(self.handle, item, c, s, j0)
        return s, j0

    def update(self, h, alpha, beta, rho):
        model_batch_update(self.handle, *(np.ascontiguousarray(x, dtype=np.float64)
                                          if not _is_torch(x) else x for x in (h, alpha, beta, rho)))

    def plan(self) -> Plan:
        return get_plan(self.handle)

    def set_plan(self, **kw):
        p = get_plan(self.handle)
        for k, v in kw.items():
            setattr(p, k, int(v))
        set_plan(self.handle, p)

    def autotune(self, reps: int = 2) -> Plan:
        return autotune(self.handle, reps)

    def last_scan_ms(self) -> float:
        return last_scan_ms(self.handle)

    def last_scan_unresolved(self) -> int:
        return last_scan_unresolved(self.handle)

    def last_scan_fallback(self) -> int:
        return last_scan_fallback(self.handle)

    def last_changes_linear(self) -> int:
        return last_changes_linear(self.handle)


# ------------------------------------------------------------ no allocation

ETOOBIG = 7
NOALLOC_MAX_MODELS, NOALLOC_MAX_RECORDS, NOALLOC_MAX_ITEMS = 1024, 16384, 65536


def dispersion_noalloc(n_layers, h, alpha, beta, rho, n_lambda, lam, grid, ct, ct_idx, status,
                       stream=None):
    """masw_dispersion_noalloc: Algorithm 1 without any allocation by the
    library, for callers whose GPU memory comes from someone else. Model
    arrays host or device (all in the same space); ct, ct_idx, status must be
    device tensors. Raises MaswError (code ETOOBIG beyond the fixed limits)."""
    lib = load()
    f = lib.masw_dispersion_noalloc
    f.argtypes = [ctypes.POINTER(ModelsDesc), ctypes.POINTER(GridDesc), ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    spaces = {_space(x) for x in (n_layers, h, alpha, beta, rho, n_lambda, lam) if x is not None}
    if len(spaces) != 1:
        raise ValueError("dispersion_noalloc: model arrays must all be host or all be device")
    space = spaces.pop()
    desc = ModelsDesc(int(len(n_layers)), _ptr(n_layers), _ptr(h), _ptr(alpha), _ptr(beta),
                      _ptr(rho), _ptr(n_lambda), _ptr(lam), space)
    g = GridDesc(float(grid[0]), float(grid[1]), int(grid[2]))
    _check(f(ctypes.byref(desc), ctypes.byref(g), _stream_handle(stream), _ptr(ct), _ptr(ct_idx),
             _ptr(status)), "masw_dispersion_noalloc")
