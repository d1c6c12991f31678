"""The allocation-free bisection entry point, sev_tridiag_bisect_static.

Some callers cannot allocate device memory at the point where they need
eigenvalues (a framework that owns every device allocation, or a
latency-critical path that must not pay cudaMalloc's implicit device
synchronisation).  This entry point keeps its scratch in a fixed device array
inside the library; these tests check, through the C ABI, that two calls in a
row give the same eigenvalues as the handle-based sev_tridiag_bisect (bit for
bit, the tolerance the bisection parity tests use) and that sizes beyond its
fixed maximum are rejected.  The file sorts last so a run stopping at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1604_03703_gb300 import build as B

    B.build()
    from paper_1604_03703_gb300 import _lib, api

    h = api.Handle(0)
    yield torch, _lib.load(), h
    h.close()


def _static(torch, lib, d_t, e_t, rtol, out_t):
    stream = torch.cuda.current_stream().cuda_stream
    return lib.sev_tridiag_bisect_static(d_t.numel(), ctypes.c_void_p(d_t.data_ptr()), ctypes.c_void_p(e_t.data_ptr()),
                                         float(rtol), ctypes.c_void_p(out_t.data_ptr()), ctypes.c_void_p(stream))


def test_static_bisect_matches_handle_two_calls(env):
    torch, lib, h = env
    cases = [I.random_tridiagonal(3001, 41), I.toeplitz(5000, 0.25, -1.5)[:2]]
    for rtol, (d, e) in zip([1e-14, 1e-9], cases):
        d_t = torch.tensor(d, dtype=torch.float64, device="cuda")
        e_t = torch.tensor(e, dtype=torch.float64, device="cuda")
        out = torch.empty_like(d_t)
        assert _static(torch, lib, d_t, e_t, rtol, out) == 0
        ref = h.tridiag_bisect(d_t, e_t, rtol)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


def test_static_bisect_rejects_oversize_and_bad_rtol(env):
    torch, lib, _ = env
    d_t = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ctypes.c_void_p(d_t.data_ptr())
    assert lib.sev_tridiag_bisect_static(65537, p, p, 1e-14, p, stream) == -1
    assert lib.sev_tridiag_bisect_static(4, p, p, 1e-20, p, stream) == -4
