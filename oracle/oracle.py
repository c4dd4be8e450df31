"""ctypes binding of the CPU FP64 oracle (``masw_oracle.c``).

TEST INFRASTRUCTURE ONLY. The test suite, the package smoke check and the
benchmark's CPU-baseline leg call it; the product path (``libmasw``) never
does, and the two share no code.

Each wrapper takes numpy arrays and returns numpy arrays; the arithmetic
lives in C. See ``masw_oracle.c`` for the passage of the paper each routine
follows (Algorithm 1 scan, Section 2.1 stiffness matrix method, Algorithm 2
misfit) and for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "masw_oracle.c")
_HDR = os.path.join(_HERE, "masw_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libmasw_oracle.so")

OK = 0
NO_ROOT = 1
EINVAL = -1
MAX_KH = 300.0  # domain of the plain hyperbolic functions: k h <= MAX_KH in every layer
ENOMEM = -2
MAX_LAYERS = 256

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction) and return
    the path of the shared library."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= newest:
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_BUILD)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    lib.oracle_grid_velocity.restype = d
    lib.oracle_grid_velocity.argtypes = [d, d, i]
    lib.oracle_layer_stiffness.restype = None
    lib.oracle_layer_stiffness.argtypes = [d, d, d, d, d, d, p]
    lib.oracle_halfspace_stiffness.restype = None
    lib.oracle_halfspace_stiffness.argtypes = [d, d, d, d, d, p]
    lib.oracle_assemble.restype = None
    lib.oracle_assemble.argtypes = [i, p, p, p, p, d, d, p]
    lib.oracle_lu_det.restype = None
    lib.oracle_lu_det.argtypes = [i, p, p, p]
    lib.oracle_det.restype = i
    lib.oracle_det.argtypes = [i, p, p, p, p, d, d, p, p]
    lib.oracle_scan_limit.restype = i
    lib.oracle_scan_limit.argtypes = [d, d, d, i]
    lib.oracle_scan.restype = i
    lib.oracle_scan.argtypes = [i, p, p, p, p, d, d, d, i, p, p]
    lib.oracle_scan_changes.restype = i
    lib.oracle_scan_changes.argtypes = [i, p, p, p, p, d, d, d, i, i, p, p]
    lib.oracle_dispersion.restype = i
    lib.oracle_dispersion.argtypes = [i, p, p, p, p, p, p, p, d, d, i, p, p, p, i]
    lib.oracle_refine.restype = i
    lib.oracle_refine.argtypes = [i, p, p, p, p, d, d, d, d, p]
    lib.oracle_root.restype = i
    lib.oracle_root.argtypes = [i, p, p, p, p, d, d, d, i, i, d, p]
    lib.oracle_root_grad_fd.restype = i
    lib.oracle_root_grad_fd.argtypes = [i, p, p, p, p, d, d, d, i, i, d, d, p, p]
    lib.oracle_det_leaky.restype = i
    lib.oracle_det_leaky.argtypes = [i, p, p, p, p, d, d, p, p]
    lib.oracle_scan_leaky.restype = i
    lib.oracle_scan_leaky.argtypes = [i, p, p, p, p, d, d, d, i, p, p]
    lib.oracle_halfspace_stiffness_complex.restype = None
    lib.oracle_halfspace_stiffness_complex.argtypes = [d, d, d, d, d, p]
    lib.oracle_assemble_complex.restype = None
    lib.oracle_assemble_complex.argtypes = [i, p, p, p, p, d, d, p]
    lib.oracle_lu_det_complex.restype = None
    lib.oracle_lu_det_complex.argtypes = [i, p, p, p]
    lib.oracle_det_sign_banded.restype = i
    lib.oracle_det_sign_banded.argtypes = [i, p, p, p, p, d, d, p]
    lib.oracle_scan_banded.restype = i
    lib.oracle_scan_banded.argtypes = [i, p, p, p, p, d, d, d, i, p, p]
    lib.oracle_dispersion_banded.restype = i
    lib.oracle_dispersion_banded.argtypes = [i, p, p, p, p, p, p, p, d, d, i, p, p, p, i]
    lib.oracle_misfit_paper.restype = d
    lib.oracle_misfit_paper.argtypes = [i, p, p]
    lib.oracle_misfit_lsq.restype = d
    lib.oracle_misfit_lsq.argtypes = [i, p, p, d]
    _lib = lib
    return lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def grid_velocity(c0: float, dc: float, n: int) -> float:
    """V[n] = c0 + n*dc rounded once."""
    return _load().oracle_grid_velocity(c0, dc, n)


def layer_stiffness(k, c, h, alpha, beta, rho) -> np.ndarray:
    """4x4 layer stiffness (DOFs ux_top, uz_top, ux_bot, uz_bot)."""
    out = np.empty(16)
    _load().oracle_layer_stiffness(k, c, h, alpha, beta, rho, _ptr(out))
    return out.reshape(4, 4)


def halfspace_stiffness(k, c, alpha, beta, rho) -> np.ndarray:
    """2x2 half-space stiffness for c < beta."""
    out = np.empty(4)
    _load().oracle_halfspace_stiffness(k, c, alpha, beta, rho, _ptr(out))
    return out.reshape(2, 2)


def assemble(h, alpha, beta, rho, k, c) -> np.ndarray:
    """Dense global stiffness 2(N+1) x 2(N+1)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    N = h.size
    n = 2 * (N + 1)
    K = np.empty((n, n))
    _load().oracle_assemble(N, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), k, c, _ptr(K))
    return K


def lu_det(A) -> tuple[int, float]:
    """(sign, ln|det|) of a dense square matrix by LU with partial pivoting."""
    A = _f64(np.array(A, dtype=np.float64, copy=True))
    n = A.shape[0]
    sg = ctypes.c_int()
    la = ctypes.c_double()
    _load().oracle_lu_det(n, _ptr(A), ctypes.byref(sg), ctypes.byref(la))
    return sg.value, la.value


def det(h, alpha, beta, rho, k, c) -> tuple[int, float]:
    """(sign, ln|det K|) of the global stiffness at (k, c)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    sg = ctypes.c_int()
    la = ctypes.c_double()
    st = _load().oracle_det(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), k, c,
                            ctypes.byref(sg), ctypes.byref(la))
    if st != OK:
        raise MemoryError("oracle_det")
    return sg.value, la.value


def scan_limit(beta_hs, c0, dc, n_c) -> int:
    return _load().oracle_scan_limit(beta_hs, c0, dc, n_c)


def scan(h, alpha, beta, rho, lam, c0, dc, n_c) -> tuple[int, float, int]:
    """Algorithm 1 for one wavelength: (status, C_t, index)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    ct = ctypes.c_double()
    idx = ctypes.c_int()
    st = _load().oracle_scan(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam, c0,
                             dc, n_c, ctypes.byref(ct), ctypes.byref(idx))
    return st, ct.value, idx.value


def negative_eigenvalues(h, alpha, beta, rho, k, c) -> int:
    """Number of negative eigenvalues of the assembled K(k, c) (numpy's
    symmetric eigensolver on the oracle's dense matrix)."""
    return int((np.linalg.eigvalsh(assemble(h, alpha, beta, rho, k, c)) < 0.0).sum())


def clamped_modes(k, c, h, alpha, beta, rho, max_sublayers=400) -> int:
    """Number of modes below c of one layer with both faces clamped (the J0
    of Wittrick-Williams for that element), by brute force: the layer cut
    into m equal sublayers, each under its pole-free bound beta sqrt(1 +
    (pi / (k h/m))^2) (so none of them has a clamped mode below c), assembled
    over the m - 1 interior nodes; by Wittrick-Williams the count is the
    number of negative eigenvalues of that dense matrix (numpy's symmetric
    eigensolver). -1 when more than max_sublayers would be needed."""
    m = 2
    while beta * np.sqrt(1.0 + (np.pi * m / (k * h)) ** 2) <= c:
        m += 1
        if m > max_sublayers:
            return -1
    Ke = layer_stiffness(k, c, h / m, alpha, beta, rho)
    n = 2 * (m - 1)
    K = np.zeros((n, n))
    for i in range(m):
        for p in range(4):
            for q in range(4):
                a, b = i + p // 2, i + q // 2
                if 1 <= a <= m - 1 and 1 <= b <= m - 1:
                    K[2 * (a - 1) + p % 2, 2 * (b - 1) + q % 2] += Ke[p, q]
    return int((np.linalg.eigvalsh(K) < 0.0).sum())


def scan_changes(h, alpha, beta, rho, lam, c0, dc, n_c, max_changes):
    """Algorithm 1 continued (higher modes): the first max_changes sign
    changes of det K along the grid, each with the change in the number of
    negative eigenvalues of K across it (Wittrick-Williams: +1 where a mode of
    the layered structure is crossed, -1 at a pole, a mode of a clamped
    layer). Returns (status, idx[max_changes], delta[max_changes]) with -1 /
    0 padding; status OK when max_changes were found, else NO_ROOT."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    idx = np.full(max_changes, -1, dtype=np.int32)
    nf = ctypes.c_int()
    st = _load().oracle_scan_changes(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam,
                                     c0, dc, n_c, max_changes, _ptr(idx), ctypes.byref(nf))
    if st not in (OK, NO_ROOT):
        raise ValueError(f"oracle_scan_changes failed ({st})")
    k = 2.0 * np.pi / lam
    delta = np.zeros(max_changes, dtype=np.int32)
    for m in range(nf.value):
        n = int(idx[m])
        delta[m] = (negative_eigenvalues(h, alpha, beta, rho, k, grid_velocity(c0, dc, n))
                    - negative_eigenvalues(h, alpha, beta, rho, k, grid_velocity(c0, dc, n - 1)))
    return st, idx, delta


def dispersion(models, c0, dc, n_c, n_threads: int = 0):
    """Algorithm 1 over a ragged batch. ``models`` is a dict with n_layers,
    h, alpha, beta, rho, n_lambda, lambda (concatenated as in the C ABI).
    Returns (ct, idx, status) arrays of length sum(n_lambda)."""
    nl = _i32(models["n_layers"])
    nw = _i32(models["n_lambda"])
    h, a, b, r = (_f64(models[k]) for k in ("h", "alpha", "beta", "rho"))
    lam = _f64(models["lambda"])
    L = lam.size
    ct = np.empty(L)
    idx = np.empty(L, dtype=np.int32)
    st = np.empty(L, dtype=np.int32)
    err = _load().oracle_dispersion(nl.size, _ptr(nl), _ptr(h), _ptr(a), _ptr(b), _ptr(r),
                                    _ptr(nw), _ptr(lam), c0, dc, n_c, _ptr(ct), _ptr(idx),
                                    _ptr(st), n_threads)
    if err != OK:
        raise MemoryError("oracle_dispersion")
    return ct, idx, st


def halfspace_stiffness_complex(k, c, alpha, beta, rho) -> np.ndarray:
    """2x2 complex half-space stiffness for any c > 0 (principal roots r, s)."""
    out = np.empty(4, dtype=np.complex128)
    _load().oracle_halfspace_stiffness_complex(k, c, alpha, beta, rho, _ptr(out))
    return out.reshape(2, 2)


def assemble_complex(h, alpha, beta, rho, k, c) -> np.ndarray:
    """Dense complex global stiffness (real layers, complex half-space)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    n = 2 * (h.size + 1)
    K = np.empty((n, n), dtype=np.complex128)
    _load().oracle_assemble_complex(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), k, c,
                                    _ptr(K))
    return K


def lu_det_complex(A) -> tuple[complex, float]:
    """(phase, ln|det|) of a dense complex matrix, det = phase * exp(ln|det|)."""
    A = np.array(A, dtype=np.complex128, copy=True, order="C")
    ph = np.zeros(1, dtype=np.complex128)
    la = ctypes.c_double()
    _load().oracle_lu_det_complex(A.shape[0], _ptr(A), _ptr(ph), ctypes.byref(la))
    return complex(ph[0]), la.value


def det_leaky(h, alpha, beta, rho, k, c) -> tuple[int, float]:
    """(sign of Re det K, ln|det K|) for any c > 0 (leaky continuation)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    sg = ctypes.c_int()
    la = ctypes.c_double()
    st = _load().oracle_det_leaky(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), k, c,
                                  ctypes.byref(sg), ctypes.byref(la))
    if st != OK:
        raise ValueError(f"oracle_det_leaky failed ({st})")
    return sg.value, la.value


def scan_leaky(h, alpha, beta, rho, lam, c0, dc, n_c) -> tuple[int, float, int]:
    """Algorithm 1 over the whole grid with the sign of Re det K:
    (status, C_t, index)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    ct = ctypes.c_double()
    idx = ctypes.c_int()
    st = _load().oracle_scan_leaky(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam,
                                   c0, dc, n_c, ctypes.byref(ct), ctypes.byref(idx))
    return st, ct.value, idx.value


def det_sign_banded(h, alpha, beta, rho, k, c) -> int:
    """Sign of det K by the banded (2x2 block) elimination of the CPU
    baseline."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    sg = ctypes.c_int()
    st = _load().oracle_det_sign_banded(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), k,
                                        c, ctypes.byref(sg))
    if st != OK:
        raise ValueError(f"oracle_det_sign_banded failed ({st})")
    return sg.value


def scan_banded(h, alpha, beta, rho, lam, c0, dc, n_c) -> tuple[int, float, int]:
    """Algorithm 1 with the banded determinant sign: (status, C_t, index)."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    ct = ctypes.c_double()
    idx = ctypes.c_int()
    st = _load().oracle_scan_banded(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam,
                                    c0, dc, n_c, ctypes.byref(ct), ctypes.byref(idx))
    return st, ct.value, idx.value


def dispersion_banded(models, c0, dc, n_c, n_threads: int = 0):
    """The CPU banded baseline over a ragged batch (layout of dispersion)."""
    nl = _i32(models["n_layers"])
    nw = _i32(models["n_lambda"])
    h, a, b, r = (_f64(models[k]) for k in ("h", "alpha", "beta", "rho"))
    lam = _f64(models["lambda"])
    L = lam.size
    ct = np.empty(L)
    idx = np.empty(L, dtype=np.int32)
    st = np.empty(L, dtype=np.int32)
    err = _load().oracle_dispersion_banded(nl.size, _ptr(nl), _ptr(h), _ptr(a), _ptr(b), _ptr(r),
                                           _ptr(nw), _ptr(lam), c0, dc, n_c, _ptr(ct), _ptr(idx),
                                           _ptr(st), n_threads)
    if err != OK:
        raise MemoryError("oracle_dispersion_banded")
    return ct, idx, st


def refine(h, alpha, beta, rho, lam, c_lo, c_hi, rel_tol=1e-13) -> float:
    """Bisection on sgn det K inside [c_lo, c_hi]."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    root = ctypes.c_double()
    st = _load().oracle_refine(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam,
                               c_lo, c_hi, rel_tol, ctypes.byref(root))
    return root.value if st == OK else float("nan")


def root(h, alpha, beta, rho, lam, c0, dc, n_c, idx, rel_tol=1e-13) -> float:
    """Refined continuous root inside [V[idx-1], V[idx]]."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    out = ctypes.c_double()
    st = _load().oracle_root(h.size, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam, c0,
                             dc, n_c, idx, rel_tol, ctypes.byref(out))
    return out.value if st == OK else float("nan")


def root_grad_fd(h, alpha, beta, rho, lam, c0, dc, n_c, idx, rel_step=1e-4, rel_tol=1e-13):
    """Central-difference gradient of the refined root with respect to
    beta_1..beta_{N+1} (Poisson ratio held) and h_1..h_N."""
    h, alpha, beta, rho = _f64(h), _f64(alpha), _f64(beta), _f64(rho)
    N = h.size
    gb = np.empty(N + 1)
    gh = np.empty(max(N, 1))
    st = _load().oracle_root_grad_fd(N, _ptr(h), _ptr(alpha), _ptr(beta), _ptr(rho), lam,
                                     c0, dc, n_c, idx, rel_step, rel_tol, _ptr(gb), _ptr(gh))
    if st != OK:
        raise ValueError("oracle_root_grad_fd: invalid input")
    return gb, gh[:N]


def misfit_paper(ct, ce) -> float:
    """Algorithm 2: mean relative error."""
    ct, ce = _f64(ct), _f64(ce)
    return _load().oracle_misfit_paper(ct.size, _ptr(ct), _ptr(ce))


def misfit_lsq(ct, ce, sigma) -> float:
    """1/(2 sigma^2) * sum (C - C_e)^2."""
    ct, ce = _f64(ct), _f64(ce)
    return _load().oracle_misfit_lsq(ct.size, _ptr(ct), _ptr(ce), sigma)
