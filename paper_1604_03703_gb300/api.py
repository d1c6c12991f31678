"""Tensor-level entry points over the sev C ABI.

PyTorch provides device memory and the current stream; the computation is
entirely libsev.so's.  Names follow the C ABI: ``eigvalsh``,
``full_to_band``, ``band_to_band``, ``tridiag_bisect``.

Matrix convention: the library reads column-major storage and only its lower
triangle.  A symmetric matrix may be passed as any contiguous n x n tensor
(for a C-contiguous tensor the library reads the transpose, which for a
symmetric matrix is the same matrix).  Band tensors are (ldab, n) arrays in
packed lower band storage with AB[d, j] = A(j + d, j), stored so that column
j is contiguous, i.e. a C-contiguous torch tensor of shape (n, ldab).
"""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import _lib
from ._lib import SEV_FP64, SEV_MIXED, check

_DTYPE_PREC = {torch.float64: SEV_FP64, torch.float32: SEV_MIXED}


def _prec_of(t: torch.Tensor) -> int:
    if t.dtype not in _DTYPE_PREC:
        raise TypeError("expected float64 (plain FP64) or float32 (mixed) tensor, got %s" % t.dtype)
    return _DTYPE_PREC[t.dtype]


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _square_ld(A: torch.Tensor) -> int:
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    n = A.shape[0]
    if n <= 1:
        return 1
    s0, s1 = A.stride()
    if s0 == 1:  # column-major view
        return s1
    if s1 == 1:  # row-major: the library reads A^T (same matrix when symmetric)
        return s0
    raise ValueError("A must have unit stride in one dimension")


class Handle:
    """A sev handle bound to a CUDA device; calls run on torch's current stream."""

    def __init__(self, device: int = 0):
        self._lib = _lib.load()
        self.device = device
        h = ctypes.c_void_p()
        check(self._lib.sev_create(ctypes.byref(h), device), "sev_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sev_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _sync_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        check(self._lib.sev_set_stream(self._h, ctypes.c_void_p(s)), "sev_set_stream")

    # ----------------------------------------------------------------- calls
    def eigvalsh(self, A: torch.Tensor, b0: int = 0, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Eigenvalues (ascending, float64) of symmetric A; A is overwritten."""
        self._sync_stream()
        n = A.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=A.device)
        check(self._lib.sev_eigvalsh(self._h, n, _ptr(A), _square_ld(A), b0, _prec_of(A), _ptr(out)), "sev_eigvalsh")
        return out

    def eigvalsh_host(self, A_host, b0: int = 0, prec: Optional[int] = None, out=None):
        """Host-buffer variant: A_host is a CPU tensor (pinned for async copies);
        returns a CPU float64 tensor.  Copies are inside the call."""
        self._sync_stream()
        n = A_host.shape[0]
        if prec is None:
            prec = _prec_of(A_host)
        if out is None:
            out = torch.empty(n, dtype=torch.float64)
        check(self._lib.sev_eigvalsh_host(self._h, n, _ptr(A_host), _square_ld(A_host), b0, prec, _ptr(out)),
              "sev_eigvalsh_host")
        return out

    def full_to_band(self, A: torch.Tensor, b: int, ldab: Optional[int] = None) -> torch.Tensor:
        """Algorithm 4.1: returns the packed band (n, ldab) tensor; A is overwritten."""
        self._sync_stream()
        n = A.shape[0]
        ldab = ldab or 2 * b
        AB = torch.empty((n, ldab), dtype=A.dtype, device=A.device)
        check(self._lib.sev_full_to_band(self._h, n, _ptr(A), _square_ld(A), b, _prec_of(A), _ptr(AB), ldab),
              "sev_full_to_band")
        return AB

    def band_to_band(self, AB: torch.Tensor, b: int, h: int) -> torch.Tensor:
        """Algorithm 4.2 in place on the packed band (n, ldab) tensor."""
        self._sync_stream()
        n, ldab = AB.shape
        assert AB.is_contiguous()
        check(self._lib.sev_band_to_band(self._h, n, _ptr(AB), ldab, b, h, _prec_of(AB)), "sev_band_to_band")
        return AB

    def band_tridiag(self, AB: torch.Tensor):
        """(d, e) float64 of a packed band whose half-bandwidth is 1."""
        self._sync_stream()
        n, ldab = AB.shape
        d = torch.empty(n, dtype=torch.float64, device=AB.device)
        e = torch.empty(max(n - 1, 1), dtype=torch.float64, device=AB.device)
        check(self._lib.sev_band_tridiag_extract(self._h, n, _ptr(AB), ldab, _prec_of(AB), _ptr(d), _ptr(e)),
              "sev_band_tridiag_extract")
        return d, e[: max(n - 1, 0)]

    def tridiag_bisect(self, d: torch.Tensor, e: torch.Tensor, rtol: float = 1e-14,
                       out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Eigenvalues of the tridiagonal (d, e) by Sturm bisection, ascending."""
        self._sync_stream()
        n = d.shape[0]
        assert d.dtype == torch.float64 and e.dtype == torch.float64
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=d.device)
        ee = e if e.numel() else d
        check(self._lib.sev_tridiag_bisect(self._h, n, _ptr(d), _ptr(ee), float(rtol), _ptr(out)), "sev_tridiag_bisect")
        return out

    # --------------------------------------------------------------- batches
    def _batch_arrays(self, mats, outs):
        k = len(mats)
        n = (ctypes.c_int * max(k, 1))(*[m.shape[0] for m in mats])
        ld = (ctypes.c_int * max(k, 1))(*[_square_ld(m) for m in mats])
        A = (ctypes.c_void_p * max(k, 1))(*[m.data_ptr() for m in mats])
        E = (ctypes.c_void_p * max(k, 1))(*[o.data_ptr() for o in outs])
        return k, n, ld, A, E

    def _batch_prec(self, mats):
        precs = {_prec_of(m) for m in mats}
        if len(precs) > 1:
            raise ValueError("a batch must be all float32 or all float64")
        return precs.pop() if precs else _lib.SEV_MIXED

    def eigvalsh_batched(self, mats, b: int = 0, outs=None):
        """Eigenvalues (ascending, float64) of every symmetric matrix in
        `mats` (CUDA tensors, all float32 or all float64); overwritten."""
        self._sync_stream()
        if outs is None:
            outs = [torch.empty(m.shape[0], dtype=torch.float64, device=m.device) for m in mats]
        k, n, ld, A, E = self._batch_arrays(mats, outs)
        check(self._lib.sev_eigvalsh_batched(self._h, k, n, ld, A, b, self._batch_prec(mats), E),
              "sev_eigvalsh_batched")
        return outs

    def batch_plan(self, mats, outs, b: int = 0) -> "BatchPlan":
        """A plan over fixed matrices and output buffers; run() only enqueues
        kernels (capturable in a CUDA graph when large_count == 0)."""
        return BatchPlan(self, mats, outs, b)

    def batch_autotune(self, sizes, prec: int) -> int:
        arr = (ctypes.c_int * max(len(sizes), 1))(*sizes)
        best = ctypes.c_int()
        check(self._lib.sev_batch_autotune(self._h, len(sizes), arr, prec, ctypes.byref(best)), "sev_batch_autotune")
        return best.value

    def autotune(self, n: int, prec: int, b0: int = 0):
        """Tune the band widths of eigvalsh at order n (sev_autotune): returns
        (widths from b0 down to 1, predicted reduction milliseconds)."""
        self._sync_stream()
        bands = (ctypes.c_int * 16)()
        nb = ctypes.c_int()
        ms = ctypes.c_double()
        check(self._lib.sev_autotune(self._h, int(n), int(prec), int(b0), bands, 16, ctypes.byref(nb), ctypes.byref(ms)),
              "sev_autotune")
        return list(bands[:nb.value]), ms.value

    def eigvalsh_bands(self, n: int, b0: int, prec: int):
        """The band widths eigvalsh(n, b0, prec) runs on this handle."""
        bands = (ctypes.c_int * 40)()
        k = self._lib.sev_eigvalsh_bands(self._h, int(n), int(b0), int(prec), bands, 40)
        if k < 0:
            check(k, "sev_eigvalsh_bands")
        return list(bands[:k])

    def get_error(self) -> int:
        return self._lib.sev_get_error(self._h)

    def raise_device_error(self, where: str = "device") -> None:
        check(self.get_error(), where)

    def set_wait_limit(self, cycles: int = 0) -> None:
        """Time limit of the handle's device-side waits in SM cycles (0: default)."""
        self._sync_stream()
        check(self._lib.sev_set_wait_limit(self._h, int(cycles)), "sev_set_wait_limit")

    # --------------------------------------------------------------- timing
    def set_kernel_timing(self, on=True) -> None:
        """True: time every kernel; False: none; a str or list of kernel
        names: time only those kernels."""
        if on is True:
            mask = (1 << 64) - 1
        elif not on:
            mask = 0
        else:
            names = [on] if isinstance(on, str) else list(on)
            ids = {self._lib.sev_kernel_name(k).decode(): k for k in range(self._lib.sev_kernel_count())}
            mask = 0
            for nm in names:
                mask |= 1 << ids[nm]
        check(self._lib.sev_set_kernel_timing(self._h, ctypes.c_ulonglong(mask)), "sev_set_kernel_timing")

    def kernel_times(self, reset: bool = True) -> dict:
        """{kernel name: (total_ms, launches)} since timing was enabled/reset."""
        out = {}
        for k in range(self._lib.sev_kernel_count()):
            ms, cnt = ctypes.c_double(), ctypes.c_long()
            check(self._lib.sev_kernel_time(self._h, k, ctypes.byref(ms), ctypes.byref(cnt), 1 if reset else 0),
                  "sev_kernel_time")
            if cnt.value:
                out[self._lib.sev_kernel_name(k).decode()] = (ms.value, cnt.value)
        return out

    def workspace_query(self, n: int, b0: int, prec: int) -> int:
        v = ctypes.c_size_t()
        check(self._lib.sev_workspace_query(self._h, n, b0, prec, ctypes.byref(v)), "sev_workspace_query")
        return v.value

    def set_workspace(self, buf: Optional[torch.Tensor]) -> None:
        if buf is None:
            check(self._lib.sev_set_workspace(self._h, ctypes.c_void_p(0), 0), "sev_set_workspace")
        else:
            check(self._lib.sev_set_workspace(self._h, _ptr(buf), buf.numel() * buf.element_size()), "sev_set_workspace")


class BatchPlan:
    def __init__(self, h: Handle, mats, outs, b: int = 0):
        self.h = h
        self._keep = (list(mats), list(outs))
        k, n, ld, A, E = h._batch_arrays(mats, outs)
        p = ctypes.c_void_p()
        check(h._lib.sev_batch_plan_create(h._h, k, n, ld, A, E, b, h._batch_prec(mats), ctypes.byref(p)),
              "sev_batch_plan_create")
        self._p = p
        bb, sc, lc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(h._lib.sev_batch_plan_info(p, ctypes.byref(bb), ctypes.byref(sc), ctypes.byref(lc)), "sev_batch_plan_info")
        self.b, self.small_count, self.large_count = bb.value, sc.value, lc.value

    def run(self) -> None:
        self.h._sync_stream()
        check(self.h._lib.sev_batch_run(self.h._h, self._p), "sev_batch_run")

    def close(self) -> None:
        if getattr(self, "_p", None):
            self.h._lib.sev_batch_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def band_schedule(n: int, b0: int = 0, prec: int = _lib.SEV_MIXED) -> list:
    """Band widths sev_eigvalsh goes through (b0, ..., 1); host only."""
    lib = _lib.load()
    buf = (ctypes.c_int * 40)()
    k = lib.sev_band_schedule(n, b0, prec, buf, 40)
    check(k if k < 0 else 0, "sev_band_schedule")
    return [buf[i] for i in range(k)]


_default = {}


def handle(device: int = 0) -> Handle:
    h = _default.get(device)
    if h is None:
        h = _default[device] = Handle(device)
    return h


def eigvalsh(A: torch.Tensor, b0: int = 0) -> torch.Tensor:
    return handle(A.device.index or 0).eigvalsh(A, b0)


def full_to_band(A: torch.Tensor, b: int) -> torch.Tensor:
    return handle(A.device.index or 0).full_to_band(A, b)


def band_to_band(AB: torch.Tensor, b: int, h: int) -> torch.Tensor:
    return handle(AB.device.index or 0).band_to_band(AB, b, h)


def tridiag_bisect(d: torch.Tensor, e: torch.Tensor, rtol: float = 1e-14) -> torch.Tensor:
    return handle(d.device.index or 0).tridiag_bisect(d, e, rtol)
