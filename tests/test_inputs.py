"""CPU checks of the seeded input generators against the recipes they state
(sizes, value distributions, structure, determinism).  The generators hold
none of the method's arithmetic; these tests use numpy's LAPACK only to
confirm the prescribed spectra of the constructions."""
import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I


def test_clustered_d_recipe():
    D = I.workload_clustered_d(16384)
    assert D.shape == (16384,) and np.all(np.diff(D) >= 0)
    # 1024 clusters of 16: within a cluster consecutive values differ by 1e-10
    mags = np.abs(D)
    assert mags.min() >= 1e-6 - 16e-10 and mags.max() <= 1.0 + 16e-10
    gaps = np.diff(D)
    small = gaps[gaps < 1e-9]
    assert small.size == 1024 * 15 and np.sum(gaps >= 1e-9) == 1023
    np.testing.assert_allclose(small, 1e-10, rtol=1e-4, atol=0)
    # random signs: both present, roughly balanced
    neg = np.sum(D < 0) // 16
    assert 400 < neg < 624
    # geometric magnitudes: log10 of the cluster leads evenly spaced over [-6, 0]
    lead = np.sort(np.abs(D))[::16]  # smallest magnitude of each cluster: g or g - 15e-10
    np.testing.assert_allclose(lead, 10.0 ** (-6.0 + 6.0 * np.arange(1024) / 1023), rtol=2e-3)


def test_qdq_has_prescribed_spectrum_and_is_symmetric():
    D = I.linspace_d(200)
    A = I.qdq(D, 11)
    assert np.array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    assert np.abs(lam - np.sort(D)).max() <= 200 * np.finfo(float).eps * 10
    Q = I.haar_q(50, 12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(50), atol=1e-13)


def test_qdq_torch_cpu_matches_recipe():
    torch = pytest.importorskip("torch")
    D = np.linspace(-2.0, 3.0, 96)
    A = I.qdq_torch(D, 7, "cpu")
    assert A.dtype == torch.float64 and torch.equal(A, A.T)
    lam = np.linalg.eigvalsh(A.numpy())
    assert np.abs(lam - D).max() <= 1e-12
    A2 = I.qdq_torch(D, 7, "cpu")
    assert torch.equal(A, A2)  # seeded
    assert I.qdq_torch(D, 7, "cpu", torch.float32).dtype == torch.float32


def test_semicircle_scale_and_symmetry():
    A = I.semicircle(600, 5)
    assert np.array_equal(A, A.T)
    lam = np.linalg.eigvalsh(A)
    assert 1.8 < lam.max() < 2.2 and -2.2 < lam.min() < -1.8
    # entries N(0, 1/n)
    assert abs(np.std(A[np.tril_indices(600)]) * np.sqrt(600) - 1.0) < 0.02
    assert np.array_equal(A, I.semicircle(600, 5))
    assert not np.array_equal(A, I.semicircle(600, 6))


def test_toeplitz_closed_form_generator():
    d, e, lam = I.toeplitz(40, 0.5, -0.25)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    np.testing.assert_allclose(np.linalg.eigvalsh(T), lam, atol=1e-14)


@pytest.mark.parametrize("n,b,ldab", [(37, 4, 8), (10, 12, 24), (64, 16, 32), (5, 1, 2)])
def test_band_packing(n, b, ldab):
    AB = I.random_band_packed(n, b, ldab, 3)
    assert AB.shape == (ldab, n)
    assert not AB[b + 1:].any()
    for dd in range(ldab):
        assert not AB[dd, max(n - dd, 0):].any()  # past the matrix's end
    A = I.band_to_dense(AB)
    assert np.array_equal(A, A.T)
    i, j = np.indices(A.shape)
    assert not A[np.abs(i - j) > b].any()
    assert np.array_equal(I.dense_to_band(A, ldab), AB)
    B = I.random_band(n, b, 4)
    assert not B[np.abs(i - j) > b].any() and np.array_equal(B, B.T)
    assert np.array_equal(I.band_to_dense(I.dense_to_band(B, ldab)), B)


def test_batch_recipes():
    sizes = I.batch_sizes(4096, 32, 512, I.SEED_BASE + 3)
    assert sizes.min() >= 32 and sizes.max() <= 512 and sizes.min() < 40 and sizes.max() > 505
    assert np.array_equal(sizes, I.batch_sizes(4096, 32, 512, I.SEED_BASE + 3))
    mats = I.batch_small(16)
    assert [m.shape[0] for m in mats] == list(I.batch_sizes(16, 32, 512, I.SEED_BASE + 3))
    assert all(np.array_equal(m, m.T) for m in mats)
    scf = I.batch_sizes(64, 1024, 6144, I.SEED_BASE + 4)
    assert scf.min() >= 1024 and scf.max() <= 6144
