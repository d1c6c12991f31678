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


def _cases():
    d_cl = np.repeat(np.array([-1.0, 0.0, 2.0]), 40)
    e_cl = np.where(np.arange(119) % 7 == 0, 1e-12, 0.0)
    return [
        ("random n=3001", *I.random_tridiagonal(3001, 41), 1e-14),
        ("toeplitz n=5000", *I.toeplitz(5000, 0.25, -1.5)[:2], 1e-9),
        ("n=1", np.array([0.75]), np.zeros(0), 1e-14),
        ("n=2", np.array([1.0, 3.0]), np.array([2.0]), 1e-14),
        ("T=0", np.zeros(64), np.zeros(63), 1e-14),
        ("clusters", d_cl, e_cl, 1e-14),
        # the largest order: the parameters and status word sit right after
        # the n + 1 squared off-diagonals at the end of the fixed array
        ("random n=65536", *I.random_tridiagonal(65536, 42), 1e-9),
    ]


@pytest.mark.parametrize("case", range(7))
def test_static_bisect_matches_handle_two_calls(env, case):
    """Two calls in a row on the same fixed array: each equals the handle's
    sev_tridiag_bisect bit for bit."""
    torch, lib, h = env
    name, d, e, rtol = _cases()[case]
    d_t = torch.tensor(d, dtype=torch.float64, device="cuda")
    e_t = torch.tensor(e if e.size else np.zeros(1), dtype=torch.float64, device="cuda")
    ref = h.tridiag_bisect(d_t, e_t[: max(d.size - 1, 0)], rtol).cpu().numpy()
    for call in range(2):
        out = torch.full_like(d_t, np.nan)
        assert _static(torch, lib, d_t, e_t, rtol, out) == 0, (name, call)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), ref, err_msg="%s call %d" % (name, call))


def test_static_bisect_argument_checks(env):
    """Every argument error is refused on the host before anything is
    launched; n = 0 is a no-op and n = 65536, the fixed maximum, is accepted."""
    torch, lib, _ = env
    d_t = torch.zeros(65536, dtype=torch.float64, device="cuda")
    out = torch.full_like(d_t, np.nan)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = ctypes.c_void_p(d_t.data_ptr())
    o = ctypes.c_void_p(out.data_ptr())
    null = ctypes.c_void_p(0)
    assert lib.sev_tridiag_bisect_static(65537, p, p, 1e-14, o, stream) == -1
    assert lib.sev_tridiag_bisect_static(-1, p, p, 1e-14, o, stream) == -1
    assert lib.sev_tridiag_bisect_static(4, null, p, 1e-14, o, stream) == -2
    assert lib.sev_tridiag_bisect_static(4, p, null, 1e-14, o, stream) == -3
    assert lib.sev_tridiag_bisect_static(4, p, p, 1e-20, o, stream) == -4
    assert lib.sev_tridiag_bisect_static(4, p, p, 1.0, o, stream) == -4
    assert lib.sev_tridiag_bisect_static(4, p, p, 1e-14, null, stream) == -5
    assert lib.sev_tridiag_bisect_static(0, null, null, 1e-14, null, stream) == 0
    assert lib.sev_tridiag_bisect_static(1, p, null, 1e-14, o, stream) == 0  # n = 1 reads no e
    assert lib.sev_tridiag_bisect_static(65536, p, p, 1e-14, o, stream) == 0  # T = 0 at the maximum order
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)
