"""Plain FP64 CPU oracle for the symmetric eigenvalue path (arXiv 1604.03703).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` leg of ``bench.py`` may import this
package; the product path (``paper_1604_03703_gb300``) never does.  The
arithmetic lives in ``oracle.c`` (plain C, FP64, no fused multiply-add); this
module only builds it and marshals numpy arrays.  See ``oracle.c`` for the
paper passage each function follows.

Parity status: every function here is pinned by tests in
``tests/test_oracle_pins.py`` against closed forms, brute-force Jacobi,
LDL^T inertia counts, invariants of orthogonal similarity and the band
structure the paper's algorithms ensure.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False):
    """The same oracle.c compiled with OpenMP (independent loops on all
    cores, same arithmetic per output) for the all-cores CPU baseline;
    None if the compiler has no OpenMP runtime."""
    if not force and os.path.exists(_LIB_OMP) and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC):
        return _LIB_OMP
    tmp = _LIB_OMP + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.check_call(cmd, stderr=subprocess.DEVNULL)
    except (subprocess.CalledProcessError, OSError):
        return None
    os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def load_omp():
    """Handle of the OpenMP build (orc_tridiagonalize, orc_bisect_range), or None."""
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            path = build_omp()
            if path is None:
                return None
            lib = ctypes.CDLL(path)
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_tridiagonalize.restype = None
            lib.orc_tridiagonalize.argtypes = [i, _dp, i, _dp, _dp, i]
            lib.orc_bisect_range.restype = i
            lib.orc_bisect_range.argtypes = [i, _dp, _dp, d, i, i, i, _dp]
            _lib_omp = lib
    return _lib_omp


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_house.restype = d
            lib.orc_house.argtypes = [i, _dp, i, _dp]
            lib.orc_tridiagonalize.restype = None
            lib.orc_tridiagonalize.argtypes = [i, _dp, i, _dp, _dp, i]
            lib.orc_pivmin.restype = d
            lib.orc_pivmin.argtypes = [i, _dp]
            lib.orc_sturm_count.restype = i
            lib.orc_sturm_count.argtypes = [i, _dp, _dp, d, d]
            lib.orc_sturm_count_minors.restype = i
            lib.orc_sturm_count_minors.argtypes = [i, _dp, _dp, d]
            lib.orc_gershgorin.restype = d
            lib.orc_gershgorin.argtypes = [i, _dp, _dp, d, _dp, _dp]
            lib.orc_bisect.restype = i
            lib.orc_bisect.argtypes = [i, _dp, _dp, d, i, _dp]
            lib.orc_bisect_range.restype = i
            lib.orc_bisect_range.argtypes = [i, _dp, _dp, d, i, i, i, _dp]
            lib.orc_bisect_ldlt.restype = i
            lib.orc_bisect_ldlt.argtypes = [i, _dp, _dp, d, i, i, ctypes.POINTER(ctypes.c_int), _dp]
            lib.orc_eigvalsh.restype = i
            lib.orc_eigvalsh.argtypes = [i, _dp, i, d, _dp]
            lib.orc_jacobi.restype = i
            lib.orc_jacobi.argtypes = [i, _dp, i, _dp]
            lib.orc_inertia.restype = i
            lib.orc_inertia.argtypes = [i, _dp, i, d]
            lib.orc_band_inertia.restype = i
            lib.orc_band_inertia.argtypes = [i, _dp, i, i, d]
            lib.orc_panel_qr.restype = i
            lib.orc_panel_qr.argtypes = [i, i, _dp, i, _dp, i, _dp, i]
            lib.orc_sign_margin_reset.restype = None
            lib.orc_sign_margin_reset.argtypes = []
            lib.orc_sign_margin_get.restype = d
            lib.orc_sign_margin_get.argtypes = []
            lib.orc_full_to_band.restype = None
            lib.orc_full_to_band.argtypes = [i, _dp, i, i]
            lib.orc_band_to_band.restype = None
            lib.orc_band_to_band.argtypes = [i, _dp, i, i, i, i, ctypes.c_long]
            lib.orc_band_to_band_wavefront.restype = None
            lib.orc_band_to_band_wavefront.argtypes = [i, _dp, i, i, i, i, i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _fortran(a) -> np.ndarray:
    """Column-major FP64 copy (the oracle's storage order)."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


# ---------------------------------------------------------------- reflectors
def house(x):
    """Householder reflector of x: returns (v, tau, beta) with v[0] = 1 and
    (I - tau v v^T) x = beta e_1; "always reflect" sign rule (Lemma 3.4)."""
    x = np.array(x, dtype=np.float64, copy=True)
    beta = ctypes.c_double()
    tau = _load().orc_house(x.size, _ptr(x), 1, ctypes.byref(beta))
    v = x.copy()
    v[0] = 1.0
    return v, tau, beta.value


# ------------------------------------------------------- tridiagonal / Sturm
def tridiagonalize(A, nsteps: int = -1):
    """Unblocked Householder tridiagonalisation (Algorithm 4.1 with b = 1).
    Reads the lower triangle of A; returns (d, e)."""
    M = _fortran(A)
    n = M.shape[0]
    d = np.zeros(max(n, 1))
    e = np.zeros(max(n, 1))
    _load().orc_tridiagonalize(n, _ptr(M), n, _ptr(d), _ptr(e), nsteps)
    return d[:n], e[: max(n - 1, 0)]


def tridiagonalize_inplace(M: np.ndarray, d: np.ndarray, e: np.ndarray, nsteps: int, omp: bool = False) -> None:
    """In-place form used to time a bounded sample of the reduction (omp:
    the OpenMP build, same results)."""
    assert M.flags.f_contiguous and M.dtype == np.float64
    lib = load_omp() if omp else _load()
    lib.orc_tridiagonalize(M.shape[0], _ptr(M), M.shape[0], _ptr(d), _ptr(e), nsteps)


def pivmin(e) -> float:
    e = np.ascontiguousarray(e, dtype=np.float64)
    return _load().orc_pivmin(e.size + 1, _ptr(e) if e.size else _ptr(np.zeros(1)))


def sturm_count(d, e, x: float) -> int:
    """Number of eigenvalues of T(d, e) below x (negative LDL^T pivots)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    n = d.size
    e2 = np.zeros(max(n, 1))
    e2[: n - 1] = e * e
    pm = pivmin(e)
    return _load().orc_sturm_count(n, _ptr(d), _ptr(e2), float(x), pm)


def sturm_count_minors(d, e, x: float) -> int:
    """Number of eigenvalues of T(d, e) below x: sign changes of the leading
    principal minors of T - xI on the exactly rescaled matrix (the count
    the bisection uses)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(np.append(np.asarray(e, dtype=np.float64), 0.0))
    return _load().orc_sturm_count_minors(d.size, _ptr(d), _ptr(e), float(x))


def gershgorin(d, e):
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(np.append(e, 0.0), dtype=np.float64)
    gl, gu = ctypes.c_double(), ctypes.c_double()
    tn = _load().orc_gershgorin(d.size, _ptr(d), _ptr(e), pivmin(e[:-1]), ctypes.byref(gl), ctypes.byref(gu))
    return gl.value, gu.value, tn


def bisect(d, e, rtol: float = 1e-14, maxit: int = 200, return_noconv: bool = False):
    """All eigenvalues of the tridiagonal T(d, e), ascending, by bisection."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.size
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = np.asarray(e, dtype=np.float64)[: n - 1]
    out = np.zeros(max(n, 1))
    nc = _load().orc_bisect(n, _ptr(d), _ptr(ee), float(rtol), int(maxit), _ptr(out))
    return (out[:n], nc) if return_noconv else out[:n]


def bisect_range(d, e, k0: int, k1: int, rtol: float = 1e-14, maxit: int = 200, omp: bool = False):
    """Eigenvalues k0 <= k < k1 (ascending indices) of T(d, e) by bisection
    (omp: the OpenMP build, same results)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.size
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = np.asarray(e, dtype=np.float64)[: n - 1]
    out = np.zeros(max(k1 - k0, 1))
    lib = load_omp() if omp else _load()
    lib.orc_bisect_range(n, _ptr(d), _ptr(ee), float(rtol), int(maxit), int(k0), int(k1), _ptr(out))
    return out[: k1 - k0]


def bisect_ldlt(d, e, rtol: float = 1e-14, idx=None, maxit: int = 200, return_noconv: bool = False):
    """Eigenvalues of T(d, e) with indices ``idx`` (0-based ascending order;
    all n when None) by plain bisection on the LDL^T pivot count with the
    pivmin guard from the unscaled Gershgorin interval -- the textbook
    definition, independent of ``bisect``'s minors count and rescaling."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    n = d.size
    ee = np.zeros(max(n, 1))
    ee[: n - 1] = np.asarray(e, dtype=np.float64)[: n - 1]
    ix = np.arange(n, dtype=np.intc) if idx is None else np.ascontiguousarray(idx, dtype=np.intc)
    out = np.zeros(max(ix.size, 1))
    nc = _load().orc_bisect_ldlt(n, _ptr(d), _ptr(ee), float(rtol), int(maxit), int(ix.size),
                                 ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(out))
    return (out[: ix.size], nc) if return_noconv else out[: ix.size]


def eigvalsh(A, rtol: float = 1e-14):
    """Eigenvalues of symmetric A (lower triangle read), ascending."""
    M = _fortran(A)
    n = M.shape[0]
    out = np.zeros(max(n, 1))
    _load().orc_eigvalsh(n, _ptr(M), n, float(rtol), _ptr(out))
    return out[:n]


# ------------------------------------------------------------- cross-checks
def jacobi(A):
    """Cyclic Jacobi eigenvalues (ascending), lower triangle read."""
    M = _fortran(A)
    n = M.shape[0]
    out = np.zeros(max(n, 1))
    _load().orc_jacobi(n, _ptr(M), n, _ptr(out))
    return out[:n]


def inertia(A, x: float) -> int:
    """Number of eigenvalues of A below x via long-double LDL^T of A - xI."""
    M = _fortran(A)
    return _load().orc_inertia(M.shape[0], _ptr(M), M.shape[0], float(x))


def band_inertia(AB, b: int, x: float) -> int:
    """Number of eigenvalues below x of the symmetric band matrix held in
    packed lower storage AB (ldab x n, AB[d, j] = B[j + d, j]), by banded
    LDL^T of B - xI (Sylvester), O(n b^2)."""
    AB = np.asfortranarray(np.asarray(AB, dtype=np.float64))
    ldab, n = AB.shape
    return _load().orc_band_inertia(n, _ptr(AB), ldab, int(b), float(x))


def inertia_lapack(A, x: float) -> int:
    """Number of eigenvalues of the symmetric A (lower triangle read) below
    x by Sylvester's law of inertia, with LAPACK's Bunch-Kaufman LDL^T
    (scipy.linalg.ldl) as the factorisation step: the count of negative
    eigenvalues of its block-diagonal D (1x1 and 2x2 blocks).  For dense
    matrices too large for the long-double factorisation above."""
    import scipy.linalg

    M = np.array(A, dtype=np.float64, order="F", copy=True)
    M[np.diag_indices_from(M)] -= x
    _, Dm, _ = scipy.linalg.ldl(M, lower=True, overwrite_a=True, check_finite=False)
    neg, i, n = 0, 0, Dm.shape[0]
    while i < n:
        if i + 1 < n and Dm[i + 1, i] != 0.0:
            a, c, bb = Dm[i, i], Dm[i + 1, i + 1], Dm[i + 1, i]
            det = a * c - bb * bb
            neg += 1 if det < 0 else (2 if a + c < 0 else 0)
            i += 2
        else:
            neg += Dm[i, i] < 0
            i += 1
    return int(neg)


# ------------------------------------------------------------- stage oracles
def panel_qr(P):
    """Householder QR of the m x nc panel: returns (R, U, T, r) with
    P = (I - U T U^T)[:, :] @ [R; 0] and r = min(nc, m-1) reflectors."""
    P = _fortran(P)
    m, nc = P.shape
    r_max = max(min(nc, m - 1), 1)
    U = np.zeros((m, r_max), order="F")
    T = np.zeros((r_max, r_max), order="F")
    r = _load().orc_panel_qr(m, nc, _ptr(P), m, _ptr(U), m, _ptr(T), r_max)
    return P, U[:, :r], T[:r, :r], r


def full_to_band(A, b: int, return_margin: bool = False):
    """Algorithm 4.1 (right-looking): returns the full symmetric band matrix
    (and, with return_margin, the smallest |alpha|/||x|| of its reflectors:
    the band is unique entry by entry when that is far above rounding)."""
    M = _fortran(A)
    M = np.tril(M) + np.tril(M, -1).T  # full symmetric storage from the lower triangle
    M = np.asfortranarray(M)
    lib = _load()
    lib.orc_sign_margin_reset()
    lib.orc_full_to_band(M.shape[0], _ptr(M), M.shape[0], int(b))
    return (M, lib.orc_sign_margin_get()) if return_margin else M


def band_to_band(B, b: int, h: int, nc_paper: bool = False, max_chases: int = -1):
    """Algorithm 4.2 (b -> h) on dense storage: returns the full symmetric
    result (after ``max_chases`` chases when that is >= 0)."""
    M = _fortran(B)
    M = np.tril(M) + np.tril(M, -1).T
    M = np.asfortranarray(M)
    _load().orc_band_to_band(M.shape[0], _ptr(M), M.shape[0], int(b), int(h), 1 if nc_paper else 0, int(max_chases))
    return M


def band_to_band_wavefront(B, b: int, h: int, wave: int, tie_desc: bool = False):
    """Algorithm 4.2's chases run in wavefront order t = wave*i + j (ties in
    increasing or decreasing i); equals band_to_band bit for bit iff the
    pipelined schedule is legal."""
    M = _fortran(B)
    M = np.tril(M) + np.tril(M, -1).T
    M = np.asfortranarray(M)
    _load().orc_band_to_band_wavefront(M.shape[0], _ptr(M), M.shape[0], int(b), int(h), int(wave), 1 if tie_desc else 0)
    return M


def band_schedule(b0: int):
    """Halving schedule b0 -> b0/2 -> ... -> 1 (Algorithm 4.3 with k = 2);
    an odd b stops the halving with one final b -> 1 step."""
    s = [b0]
    while s[-1] > 1:
        b = s[-1]
        s.append(b // 2 if b % 2 == 0 else 1)
    return s


def eigvalsh_via_stages(A, b0: int, rtol: float = 1e-14):
    """Algorithm 4.3 on one processor: full-to-band, band halvings, bisection."""
    M = full_to_band(A, b0)
    sched = band_schedule(b0)
    for b, h in zip(sched[:-1], sched[1:]):
        M = band_to_band(M, b, h)
    d = np.diag(M).copy()
    e = np.diag(M, -1).copy()
    return bisect(d, e, rtol)
