"""Seeded synthetic inputs for the symmetric eigenvalue path.

This module is shared by the oracle tests and the CUDA path; it holds none
of the method's arithmetic (no reduction, no QR of a panel, no Sturm count):
only random draws and the construction of test matrices with prescribed
spectra.  Seeds are ``SEED_BASE + workload index (+ matrix index)``.

Workload recipes (the paper has no experiments or datasets; these are the
synthetic stand-ins, stated with their sizes):

* ``qdq``: A = Q diag(D) Q^T, Q the Q factor (signs fixed by diag R > 0) of a
  seeded N(0,1) n x n matrix, symmetrised as (A + A^T)/2.  Eigenvalues are D
  up to the rounding of the construction.
* ``semicircle``: lower triangle (with diagonal) iid N(0,1), mirrored, scaled
  by 1/sqrt(n); spectrum close to the semicircle on [-2, 2].
* ``clustered_d``: 1024 magnitudes 10^(-6 + 6m/1023) with random signs, each
  repeated 16 times as s*g + r*1e-10 (r = 0..15): 16-fold clusters with gap
  1e-10 (n = 16384).
* ``toeplitz``: tridiagonal (d = a, e = b) with eigenvalues a + 2b cos(k pi/(n+1)).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1604037030


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def haar_q(n: int, seed: int) -> np.ndarray:
    """Orthogonal Q from the QR of a seeded N(0,1) matrix (diag R made > 0)."""
    G = rng(seed).standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def qdq(D, seed: int) -> np.ndarray:
    """A = Q diag(D) Q^T in FP64 (C-contiguous, symmetric)."""
    D = np.asarray(D, dtype=np.float64)
    Q = haar_q(D.size, seed)
    A = (Q * D) @ Q.T
    return 0.5 * (A + A.T)


def semicircle(n: int, seed: int) -> np.ndarray:
    """Symmetric N(0,1)/sqrt(n) matrix (lower triangle drawn, mirrored)."""
    G = rng(seed).standard_normal((n, n))
    L = np.tril(G)
    A = L + np.tril(L, -1).T
    return A / np.sqrt(n)


def linspace_d(n: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return np.linspace(lo, hi, n)


def clustered_d(n: int, seed: int, cluster: int = 16, gap: float = 1e-10) -> np.ndarray:
    """Geometric magnitudes over [1e-6, 1] with random signs, each repeated
    ``cluster`` times with spacing ``gap``; returned sorted ascending."""
    m = n // cluster
    g = 10.0 ** (-6.0 + 6.0 * np.arange(m) / max(m - 1, 1))
    s = np.where(rng(seed).random(m) < 0.5, -1.0, 1.0)
    D = (s * g)[:, None] + gap * np.arange(cluster)[None, :]
    D = D.reshape(-1)
    if D.size < n:
        D = np.concatenate([D, np.zeros(n - D.size)])
    return np.sort(D)


def toeplitz(n: int, a: float, b: float):
    """Tridiagonal Toeplitz (d, e) and its closed-form eigenvalues (ascending)."""
    d = np.full(n, float(a))
    e = np.full(max(n - 1, 0), float(b))
    k = np.arange(1, n + 1)
    lam = np.sort(a + 2.0 * b * np.cos(k * np.pi / (n + 1)))
    return d, e, lam


def random_tridiagonal(n: int, seed: int):
    r = rng(seed)
    return r.standard_normal(n), r.standard_normal(max(n - 1, 0))


def random_band(n: int, b: int, seed: int) -> np.ndarray:
    """Dense symmetric matrix with half-bandwidth b, N(0,1) entries in band."""
    G = rng(seed).standard_normal((n, n))
    i, j = np.indices((n, n))
    L = np.where((i >= j) & (i - j <= b), G, 0.0)
    return L + np.tril(L, -1).T


def random_band_packed(n: int, b: int, ldab: int, seed: int) -> np.ndarray:
    """Packed lower band (ldab x n, AB[d, j] = B[j + d, j]) of a symmetric
    matrix with half-bandwidth b and N(0,1) entries in the band; rows d > b
    and the entries past the matrix's end are zero."""
    AB = rng(seed).standard_normal((ldab, n))
    AB[b + 1:, :] = 0.0
    for dd in range(1, min(b, n - 1) + 1):
        AB[dd, n - dd:] = 0.0
    AB[min(b, n - 1) + 1: b + 1, :] = 0.0
    return AB


def dense_to_band(A: np.ndarray, ldab: int) -> np.ndarray:
    """Packed lower band storage: AB[d, j] = A[j + d, j] for 0 <= d < ldab
    (column-major, i.e. AB is ldab x n with column j contiguous)."""
    n = A.shape[0]
    AB = np.zeros((ldab, n), dtype=A.dtype)
    for dd in range(min(ldab, n)):
        AB[dd, : n - dd] = np.diagonal(A, -dd)
    return AB


def band_to_dense(AB: np.ndarray) -> np.ndarray:
    """Full symmetric matrix from packed lower band storage."""
    ldab, n = AB.shape
    A = np.zeros((n, n), dtype=AB.dtype)
    for dd in range(min(ldab, n)):
        idx = np.arange(n - dd)
        A[idx + dd, idx] = AB[dd, : n - dd]
        A[idx, idx + dd] = AB[dd, : n - dd]
    return A


# --------------------------------------------------------------- workloads
def workload_qdq512():
    """n = 512, D = linspace(-1, 1), b0 = 32 (plain FP64 parity case)."""
    n = 512
    D = linspace_d(n)
    return qdq(D, SEED_BASE + 0), D


def workload_semicircle(n: int = 8192):
    """Semicircle N(0,1)/sqrt(n) matrix (b0 = 64 in the FP64 vs mixed case)."""
    return semicircle(n, SEED_BASE + 1)


def workload_clustered_d(n: int = 16384) -> np.ndarray:
    return clustered_d(n, SEED_BASE + 2)


def qdq_torch(D, seed: int, device, dtype=None):
    """A = Q diag(D) Q^T generated with torch on ``device`` in FP64 (for the
    n = 16384 workload, whose host QR would take minutes).  Same recipe as
    ``qdq``; the random stream is torch's, seeded with ``seed``."""
    import ctypes
    import os

    import torch

    if torch.device(device).type == "cuda":
        # Load torch's CUDA linear-algebra library by full path first: under a
        # profiler's injected environment its lazy dlopen by bare name can miss.
        lib = os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg.so")
        if os.path.exists(lib):
            ctypes.CDLL(lib, mode=ctypes.RTLD_GLOBAL)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    n = len(D)
    G = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    del G
    s = torch.sign(torch.diagonal(R))
    s[s == 0] = 1.0
    del R
    Q.mul_(s[None, :])
    Dt = torch.as_tensor(np.asarray(D, dtype=np.float64), device=device)
    A = (Q * Dt[None, :]) @ Q.T
    del Q
    A = 0.5 * (A + A.T)
    if dtype is not None:
        A = A.to(dtype)
    return A


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Matrix orders drawn uniformly from lo..hi inclusive."""
    return rng(seed).integers(lo, hi + 1, size=count)


def batch_small(count: int = 4096, seed: int = SEED_BASE + 3):
    """The many-small-matrices workload: orders uniform in 32..512, each a
    symmetric N(0,1)/sqrt(n) matrix (seed + 1 + index)."""
    sizes = batch_sizes(count, 32, 512, seed)
    return [semicircle(int(m), seed + 1 + k) for k, m in enumerate(sizes)]


def batch_scf(count: int = 64, seed: int = SEED_BASE + 4):
    """The SCF-like sequence: orders uniform in 1024..6144; per distinct
    order one A0 = Q diag(D) Q^T with D uniform in [-10, 10]; matrix k is
    A0(n_k) + 1e-3 E_k with E_k a symmetric N(0,1)/sqrt(n) matrix."""
    sizes = batch_sizes(count, 1024, 6144, seed)
    base = {}
    out = []
    for k, m in enumerate(sizes):
        m = int(m)
        if m not in base:
            D = rng(seed + 100000 + m).uniform(-10.0, 10.0, m)
            base[m] = qdq(D, seed + 200000 + m)
        out.append(base[m] + 1e-3 * semicircle(m, seed + 1 + k))
    return out


def batch_scf_torch(count: int = 64, seed: int = SEED_BASE + 4, device="cuda", dtype=None):
    """batch_scf generated with torch on the GPU (the host QRs of orders up
    to 6144 take minutes): orders from batch_sizes(count, 1024, 6144, seed);
    per distinct order A0 = qdq_torch(D) with D uniform in [-10, 10] (numpy
    stream seed + 100000 + n, Q from seed + 200000 + n); matrix k adds
    1e-3 E_k, E_k symmetric N(0,1)/sqrt(n) from torch's stream seed + 1 + k."""
    import torch

    sizes = batch_sizes(count, 1024, 6144, seed)
    base = {}
    out = []
    for k, m in enumerate(sizes):
        m = int(m)
        if m not in base:
            D = rng(seed + 100000 + m).uniform(-10.0, 10.0, m)
            base[m] = qdq_torch(D, seed + 200000 + m, device)
        g = torch.Generator(device=device)
        g.manual_seed(seed + 1 + k)
        G = torch.randn(m, m, generator=g, device=device, dtype=torch.float64)
        E = torch.tril(G)
        E = (E + torch.tril(E, -1).T) / np.sqrt(m)
        A = base[m] + 1e-3 * E
        out.append(A if dtype is None else A.to(dtype))
    return out
