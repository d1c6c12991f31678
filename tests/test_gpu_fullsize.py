"""Parity at full size, in the launch configuration the benchmark times.

At n = 16384 (and 8192) the oracle cannot tridiagonalise the matrix, so the
CUDA path is checked on outputs the oracle computes one by one (sampled
eigenvalue indices of the bisection, bitwise) and on properties that hold at
any size: eigenvalues against the prescribed spectrum of Q D Q^T,
eigenvalue counts of the reduced tridiagonal against Sylvester inertia of
the input (banded or dense LDL^T), trace and Frobenius norm, exact zeros
outside the band."""
import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)


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


def clean_shifts(count_fn, xs, delta, want=4):
    """Shifts x whose window [x - delta, x + delta] holds no eigenvalue of
    the reference matrix (equal counts at both ends); returns (x, count)."""
    out = []
    for x in xs:
        lo, hi = count_fn(x - delta), count_fn(x + delta)
        if lo == hi:
            out.append((x, lo))
        if len(out) == want:
            break
    assert len(out) >= 2, "no eigenvalue-free window found"
    return out


# ----------------------------------------------------------------- bisection
@pytest.mark.parametrize("rtol", [1e-9, 1e-14])
@pytest.mark.parametrize("kind", ["random", "clustered"])
def test_bisect_n16384_sampled_vs_oracles(H, torch_cuda, orc, rtol, kind):
    torch = torch_cuda
    n = 16384
    if kind == "random":
        d, e = I.random_tridiagonal(n, 9100)
    else:  # the benchmark's clustered spectrum on the diagonal, weakly coupled
        d = np.sort(I.workload_clustered_d(n))
        e = 1e-3 * I.random_tridiagonal(n, 9101)[1]
    got = H.tridiag_bisect(torch.from_numpy(d).cuda(), torch.from_numpy(e).cuda(), rtol).cpu().numpy()
    assert np.all(np.diff(got) >= 0)
    ks = np.unique(np.concatenate([np.arange(0, 8), np.arange(n - 8, n), np.linspace(0, n - 1, 48).astype(int)]))
    for k in ks:
        assert got[k] == orc.bisect_range(d, e, int(k), int(k) + 1, rtol)[0], k
    # the textbook LDL^T bisection (independent count, unscaled interval) at the same indices
    ref = orc.bisect_ldlt(d, e, rtol, ks)
    tn = orc.gershgorin(d, e)[2]
    assert np.all(np.abs(got[ks] - ref) <= np.maximum(rtol * np.abs(ref), rtol * tn) + 8 * EPS64 * tn)


# --------------------------------------------------------------- band stages
@pytest.mark.parametrize(
    "dtype_name,b0,mids",
    [("float32", 128, None), ("float64", 64, None), ("float32", 128, [32])],
    ids=["fp32-schedule", "fp64-schedule", "fp32-128-32-1"],
)
def test_band_stages_n16384_inertia(H, torch_cuda, orc, dtype_name, b0, mids):
    """Band stages at n = 16384 on a random band matrix: the library's own
    schedule (mids None: 128 -> 32 -> 16 -> 1 mixed, 64 -> 16 -> 1 FP64, the
    calls eigvalsh makes) and 128 -> 32 -> 1 (the b -> 1 kernel at b = 32).
    The tridiagonal's Sturm counts equal the inertia of the input band at
    shifts away from its eigenvalues."""
    torch = torch_cuda
    from paper_1604_03703_gb300 import api, _lib as L

    dtype = getattr(torch, dtype_name)
    n, ldab = 16384, 2 * b0
    if mids is None:
        prec = L.SEV_MIXED if dtype_name == "float32" else L.SEV_FP64
        widths = api.band_schedule(n, b0, prec)
    else:
        widths = [b0] + list(mids) + [1]
    assert widths[0] == b0 and widths[-1] == 1
    AB = I.random_band_packed(n, b0, ldab, 9200 + b0)
    AB_t = torch.from_numpy(np.ascontiguousarray(AB.T)).to(dtype).cuda()
    AB = AB_t.double().cpu().numpy().T.copy()  # the exact input the GPU sees
    for b, h in zip(widths[:-1], widths[1:]):
        H.band_to_band(AB_t, b, h)
    d_t, e_t = H.band_tridiag(AB_t)
    torch.cuda.synchronize()
    H.raise_device_error("band stages")
    assert torch.count_nonzero(AB_t[:, 2:]).item() == 0
    d, e = d_t.cpu().numpy(), e_t.cpu().numpy()
    # trace and Frobenius norm
    fro_in = float(AB[0] @ AB[0] + 2.0 * np.sum(AB[1:] ** 2))
    fro_out = float(d @ d + 2.0 * e @ e)
    eps = EPS32 if dtype_name == "float32" else EPS64
    nrm = float(np.abs(AB).sum(axis=0).max() * 2)  # >= ||B||_2
    assert abs(d.sum() - AB[0].sum()) <= 20 * n * eps * nrm
    assert abs(fro_out - fro_in) <= 20 * n * eps * fro_in
    # eigenvalue counts at clean shifts
    radius = 2.0 * np.sqrt(2 * b0 + 1)  # edge of the band matrix's spectrum
    delta = (3e-5 if dtype_name == "float32" else 1e-9) * radius
    rng = np.random.default_rng(9300 + b0)
    xs = rng.uniform(-0.8, 0.8, 16) * radius
    # (the banded LDL^T runs in long double: software quad precision on some
    # hosts, seconds per shift at b = 128, so the extra route checks 2 shifts)
    shifts = clean_shifts(lambda t: orc.band_inertia(AB, b0, t), xs, delta, want=4 if mids is None else 2)
    for x, want in shifts:
        assert orc.sturm_count(d, e, x) == want


# ---------------------------------------------------------------- eigvalsh
@pytest.fixture(scope="module")
def bench_matrix(torch_cuda):
    D = np.sort(I.workload_clustered_d(16384))
    A64 = I.qdq_torch(D, I.SEED_BASE + 2, "cuda")
    return A64, D


def test_eigvalsh_n16384_mixed_vs_prescribed(H, torch_cuda, bench_matrix):
    """The benchmark's workload and call (FP32, b0 = 128): every eigenvalue
    within the stated 1e-4 ||A||_2 of the prescribed spectrum."""
    A64, D = bench_matrix
    A = A64.float()
    lam = H.eigvalsh(A, 128).cpu().numpy()
    H.raise_device_error("eigvalsh mixed")
    assert np.all(np.diff(lam) >= 0)
    err = np.abs(lam - D).max() / np.abs(D).max()
    assert err <= 1e-4, err


def test_eigvalsh_n16384_fp64_vs_prescribed(H, torch_cuda, bench_matrix):
    """FP64 form of the same matrix (b0 = 64): within 1e-11 ||A||_2."""
    A64, D = bench_matrix
    A = A64.clone()
    lam = H.eigvalsh(A, 64).cpu().numpy()
    H.raise_device_error("eigvalsh fp64")
    err = np.abs(lam - D).max() / np.abs(D).max()
    assert err <= 1e-11, err


@pytest.mark.parametrize("dtype_name", ["float64", "float32"])
def test_eigvalsh_n8192_semicircle_inertia(H, torch_cuda, orc, dtype_name):
    """n = 8192 semicircle matrix, b0 = 64, FP64 and mixed: eigenvalue counts
    against the inertia of A - xI (LAPACK LDL^T) at clean shifts, trace and
    Frobenius norm against the input."""
    torch = torch_cuda
    A = I.workload_semicircle(8192)
    At = torch.from_numpy(A).to(getattr(torch, dtype_name)).cuda()
    Ain = At.double().cpu().numpy()
    lam = H.eigvalsh(At, 64).cpu().numpy()
    H.raise_device_error("eigvalsh semicircle")
    nrm = float(np.abs(lam).max())
    tol = 1e-4 if dtype_name == "float32" else 1e-11
    n = A.shape[0]
    assert abs(lam.sum() - np.trace(Ain)) <= n * tol * nrm
    assert abs(lam @ lam - np.sum(Ain * Ain)) <= 2 * n * tol * nrm * nrm
    delta = (1e-5 if dtype_name == "float32" else 1e-10) * nrm
    xs = np.random.default_rng(9400).uniform(-1.5, 1.5, 8)
    for x, want in clean_shifts(lambda t: orc.inertia_lapack(Ain, t), xs, delta, want=3):
        assert int((lam < x).sum()) == want
