"""Batched eigenvalues (many independent matrices, one persistent launch)
against the oracle, matrix by matrix; the graph-captured plan against the
direct call; the autotuner's choice."""
import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


@pytest.fixture(scope="module")
def H(torch_cuda):
    from paper_1604_03703_gb300 import build as B

    B.build()
    from paper_1604_03703_gb300 import api

    h = api.Handle(0)
    yield h
    h.close()


def make(torch, mats, dtype):
    """Device copies (column-major views of the symmetric host matrices)."""
    return [torch.from_numpy(np.ascontiguousarray(A)).to(dtype).cuda() for A in mats]


def check_vs_oracle(orc, mats_host, got, tol):
    for A, lam in zip(mats_host, got):
        ref = orc.eigvalsh(A, 1e-14)
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.all(np.diff(lam) >= 0)
        assert np.abs(lam - ref).max() <= tol * scale, (A.shape[0], np.abs(lam - ref).max() / scale)


EDGE = [1, 2, 3, 5, 9, 17, 33, 64, 100]


@pytest.mark.parametrize("b", [4, 8, 16, 32])
def test_batched_mixed_vs_oracle(H, torch_cuda, orc, b):
    torch = torch_cuda
    sizes = list(EDGE) + [int(m) for m in I.batch_sizes(20, 32, 512, 9500 + b)]
    host = [I.semicircle(m, 9600 + k) for k, m in enumerate(sizes)]
    dev = make(torch, host, torch.float32)
    host32 = [t.double().cpu().numpy() for t in dev]  # the exact matrices the GPU gets
    got = [t.cpu().numpy() for t in H.eigvalsh_batched(dev, b)]
    H.raise_device_error("batched mixed")
    check_vs_oracle(orc, host32, got, 1e-4)


@pytest.mark.parametrize("b", [4, 8, 16])
def test_batched_fp64_vs_oracle(H, torch_cuda, orc, b):
    torch = torch_cuda
    sizes = list(EDGE) + [int(m) for m in I.batch_sizes(12, 32, 512, 9700 + b)]
    host = [I.semicircle(m, 9800 + k) for k, m in enumerate(sizes)]
    got = [t.cpu().numpy() for t in H.eigvalsh_batched(make(torch, host, torch.float64), b)]
    H.raise_device_error("batched fp64")
    check_vs_oracle(orc, host, got, 1e-11)


def test_batched_prescribed_spectrum_and_large_route(H, torch_cuda, orc):
    """Q D Q^T matrices with known D, including orders above the batched
    kernel's limit (they run the single-matrix path inside the same call)."""
    torch = torch_cuda
    sizes = [300, 1100, 40, 1300, 512]
    Ds = [np.linspace(-1, 1, m) for m in sizes]
    host = [I.qdq(D, 9900 + k) for k, D in enumerate(Ds)]
    dev = make(torch, host, torch.float64)
    plan_outs = [torch.empty(m, dtype=torch.float64, device="cuda") for m in sizes]
    plan = H.batch_plan(dev, plan_outs, 8)
    assert plan.large_count == 2 and plan.small_count == 3
    plan.run()
    torch.cuda.synchronize()
    H.raise_device_error("batched plan")
    for D, lam in zip(Ds, plan_outs):
        assert np.abs(lam.cpu().numpy() - D).max() <= 1e-11
    plan.close()


def test_batched_graph_capture_replays_bitwise(H, torch_cuda):
    torch = torch_cuda
    sizes = [int(m) for m in I.batch_sizes(40, 32, 400, 10000)]
    host = [I.semicircle(m, 10100 + k) for k, m in enumerate(sizes)]
    orig = make(torch, host, torch.float32)
    work = [t.clone() for t in orig]
    outs = [torch.empty(m, dtype=torch.float64, device="cuda") for m in sizes]
    plan = H.batch_plan(work, outs, 16)
    assert plan.large_count == 0
    direct = [t.cpu().numpy() for t in H.eigvalsh_batched([t.clone() for t in orig], 16)]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # warm-up outside capture
        plan.run()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    for w, o in zip(work, orig):
        w.copy_(o)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        plan.run()
    for _ in range(2):
        for w, o in zip(work, orig):
            w.copy_(o)
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        H.raise_device_error("graph replay")
        for a, b in zip(outs, direct):
            np.testing.assert_array_equal(a.cpu().numpy(), b)
    plan.close()


def test_batch_autotune_choice_is_used(H, torch_cuda):
    from paper_1604_03703_gb300 import _lib

    sizes = [int(m) for m in I.batch_sizes(64, 32, 512, 10200)]
    best = H.batch_autotune(sizes, _lib.SEV_MIXED)
    assert best in (4, 8, 16, 32)
    torch = torch_cuda
    mats = make(torch, [I.semicircle(m, 10300 + k) for k, m in enumerate(sizes[:4])], torch.float32)
    outs = [torch.empty(t.shape[0], dtype=torch.float64, device="cuda") for t in mats]
    plan = H.batch_plan(mats, outs, 0)
    assert plan.b == best
    plan.close()


def test_batched_4096_small_workload(H, torch_cuda, orc):
    """The 4096-matrix workload in the benchmark's launch: sampled matrices
    against the oracle, every matrix's trace against its eigenvalue sum."""
    torch = torch_cuda
    host = I.batch_small()
    dev = make(torch, host, torch.float32)
    host32 = [t.double().cpu().numpy() for t in dev]
    got = [t.cpu().numpy() for t in H.eigvalsh_batched(dev, 0)]
    H.raise_device_error("batched 4096")
    idx = np.linspace(0, len(host) - 1, 12).astype(int)
    check_vs_oracle(orc, [host32[i] for i in idx], [got[i] for i in idx], 1e-4)
    for A, lam in zip(host32, got):
        nrm = np.abs(lam).max()
        assert abs(lam.sum() - np.trace(A)) <= A.shape[0] * 1e-5 * nrm
