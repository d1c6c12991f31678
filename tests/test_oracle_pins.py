"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle itself (closed forms, brute-force Jacobi,
long-double inertia counts, library routines on special cases, invariants of
orthogonal similarity, and the band structure Algorithms 4.1/4.2 ensure)."""
import os

import numpy as np
import pytest

from paper_1604_03703_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def band_excess(M, b):
    i, j = np.indices(M.shape)
    sel = np.abs(i - j) > b
    return float(np.abs(M[sel]).max()) if sel.any() else 0.0


def max_fill(M):
    i, j = np.nonzero(M)
    return int(np.abs(i - j).max()) if i.size else 0


# ------------------------------------------------------------ golden files
def test_golden_householder(orc):
    rows = [l.split() for l in open(os.path.join(GOLD, "householder_3_4.txt")) if l.strip() and l[0] != "#"]
    for r in rows:
        x0, x1, beta, tau, v0, v1 = map(float, r)
        v, t, bb = orc.house([x0, x1])
        assert bb == pytest.approx(beta, abs=1e-15)
        assert t == pytest.approx(tau, abs=1e-15)
        assert v[0] == v0 and v[1] == pytest.approx(v1, abs=1e-15)


def test_golden_tridiagonal(orc):
    for line in open(os.path.join(GOLD, "tridiag_closed_forms.txt")):
        if not line.strip() or line[0] == "#":
            continue
        f = [s.strip() for s in line.split("|")]
        n = int(f[0])
        d = np.array(f[1].split(), dtype=float)
        e = np.array(f[2].split(), dtype=float) if f[2] else np.zeros(0)
        lam = np.array(f[3].split(), dtype=float)
        got = orc.bisect(d, e, 1e-15)
        assert got.shape == (n,)
        np.testing.assert_allclose(got, lam, atol=4e-15 * max(1, np.abs(lam).max()))


# ------------------------------------------------------------- reflectors
@pytest.mark.parametrize("m", [1, 2, 3, 17, 64])
def test_house_maps_to_beta_e1(orc, m):
    x = I.rng(5 + m).standard_normal(m) * 1e3
    v, tau, beta = orc.house(x)
    H = np.eye(m) - tau * np.outer(v, v)
    y = H @ x
    assert abs(y[0] - beta) <= 1e-12 * np.linalg.norm(x)
    assert np.abs(y[1:]).max(initial=0.0) <= 1e-12 * np.linalg.norm(x)
    np.testing.assert_allclose(H @ H.T, np.eye(m), atol=1e-14)
    assert abs(abs(beta) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)
    assert beta * x[0] <= 0  # beta = -sgn(alpha) ||x||
    assert 1.0 <= tau <= 2.0


def test_house_no_overflow(orc):
    x = np.array([1e300, 3e300, -2e300])
    v, tau, beta = orc.house(x)
    assert np.isfinite(beta) and abs(abs(beta) - np.linalg.norm(x / 1e300) * 1e300) < 1e286
    x = np.array([1e-300, 3e-300])
    v, tau, beta = orc.house(x)
    assert abs(abs(beta) - np.sqrt(10.0) * 1e-300) < 1e-314


# ---------------------------------------------------------- Sturm/bisection
@pytest.mark.parametrize("n,a,b", [(1, 0.3, 0.0), (2, 1.0, 2.0), (10, 2.0, -1.0), (100, 0.0, 1.0), (513, -3.0, 0.25)])
def test_bisect_toeplitz_closed_form(orc, n, a, b):
    d, e, lam = I.toeplitz(n, a, b)
    got = orc.bisect(d, e, 1e-14)
    tn = abs(a) + 2 * abs(b)
    np.testing.assert_allclose(got, lam, atol=max(4e-14 * tn, 1e-300), rtol=0)


def test_sturm_count_monotone_and_ends(orc):
    d, e = I.random_tridiagonal(200, 11)
    gl, gu, tn = orc.gershgorin(d, e)
    assert orc.sturm_count(d, e, gl) == 0
    assert orc.sturm_count(d, e, gu) == 200
    xs = np.linspace(gl, gu, 997)
    c = [orc.sturm_count(d, e, x) for x in xs]
    assert all(c1 <= c2 for c1, c2 in zip(c, c[1:]))
    lam = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))  # library routine
    for x in xs[::37]:
        if np.min(np.abs(lam - x)) > 1e-9:
            assert orc.sturm_count(d, e, x) == int((lam < x).sum())


def test_bisect_diagonal_and_split(orc):
    d = np.array([3.0, -1.0, 2.0, 2.0, 0.0])
    got = orc.bisect(d, np.zeros(4), 1e-15)
    np.testing.assert_allclose(got, np.sort(d), atol=1e-15)
    # e with a zero splits T into blocks: eigenvalues are the union
    d1, e1, l1 = I.toeplitz(4, 1.0, 0.5)
    d2, e2, l2 = I.toeplitz(3, -2.0, 1.0)
    got = orc.bisect(np.concatenate([d1, d2]), np.concatenate([e1, [0.0], e2]), 1e-15)
    np.testing.assert_allclose(got, np.sort(np.concatenate([l1, l2])), atol=2e-14)


def test_bisect_tolerance_respected(orc):
    d, e = I.random_tridiagonal(64, 3)
    lam = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))
    tn = orc.gershgorin(d, e)[2]
    for rtol in [1e-6, 1e-10, 1e-14]:
        got = orc.bisect(d, e, rtol)
        assert np.abs(got - lam).max() <= rtol * tn + 1e-13 * tn


# ------------------------------------- textbook LDL^T bisection (O3 form)
def test_bisect_ldlt_golden(orc):
    for line in open(os.path.join(GOLD, "tridiag_closed_forms.txt")):
        if not line.strip() or line[0] == "#":
            continue
        f = [s.strip() for s in line.split("|")]
        n = int(f[0])
        d = np.array(f[1].split(), dtype=float)
        e = np.array(f[2].split(), dtype=float) if f[2] else np.zeros(0)
        lam = np.array(f[3].split(), dtype=float)
        got = orc.bisect_ldlt(d, e, 1e-15)
        assert got.shape == (n,)
        np.testing.assert_allclose(got, lam, atol=4e-15 * max(1, np.abs(lam).max()))


@pytest.mark.parametrize("n,a,b", [(1, 0.3, 0.0), (2, 1.0, 2.0), (10, 2.0, -1.0), (100, 0.0, 1.0), (513, -3.0, 0.25)])
def test_bisect_ldlt_toeplitz_closed_form(orc, n, a, b):
    d, e, lam = I.toeplitz(n, a, b)
    got = orc.bisect_ldlt(d, e, 1e-14)
    tn = abs(a) + 2 * abs(b)
    np.testing.assert_allclose(got, lam, atol=max(4e-14 * tn, 1e-300), rtol=0)


def test_bisect_ldlt_diagonal_split_and_signs(orc):
    d = np.array([3.0, -1.0, 2.0, 2.0, 0.0])
    np.testing.assert_allclose(orc.bisect_ldlt(d, np.zeros(4), 1e-15), np.sort(d), atol=1e-15)
    d1, e1, l1 = I.toeplitz(4, 1.0, 0.5)
    d2, e2, l2 = I.toeplitz(3, -2.0, 1.0)
    got = orc.bisect_ldlt(np.concatenate([d1, d2]), np.concatenate([e1, [0.0], e2]), 1e-15)
    np.testing.assert_allclose(got, np.sort(np.concatenate([l1, l2])), atol=2e-14)
    # the spectrum depends on e only through e^2: flipping signs changes nothing
    d, e = I.random_tridiagonal(80, 12)
    s = np.where(I.rng(13).random(79) < 0.5, -1.0, 1.0)
    np.testing.assert_array_equal(orc.bisect_ldlt(d, e * s, 1e-14), orc.bisect_ldlt(d, e, 1e-14))


def test_bisect_ldlt_vs_library_and_subset(orc):
    d, e = I.random_tridiagonal(300, 14)
    lam = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))  # library routine
    tn = orc.gershgorin(d, e)[2]
    for rtol in [1e-6, 1e-10, 1e-14]:
        got = orc.bisect_ldlt(d, e, rtol)
        assert np.all(np.diff(got) >= 0)
        assert np.abs(got - lam).max() <= rtol * tn + 1e-13 * tn
    idx = np.array([299, 0, 150, 7])
    np.testing.assert_array_equal(orc.bisect_ldlt(d, e, 1e-14, idx), orc.bisect_ldlt(d, e, 1e-14)[idx])


def test_bisect_ldlt_clusters(orc):
    # 16-fold clusters of gap 1e-10 around well separated centres, as in the
    # clustered workload: every member resolved to the bisection tolerance
    lam = np.concatenate([c + 1e-10 * np.arange(16) for c in (-0.75, -1e-3, 0.5)])
    A = I.qdq(lam, 15)
    d, e = orc.tridiagonalize(A)
    got = orc.bisect_ldlt(d, e, 1e-14)
    assert np.abs(got - np.sort(lam)).max() <= 1e-13


# ----------------------------------------------------- cross-check routines
def test_jacobi_closed_forms(orc):
    A = np.array([[1.0, 2.0], [2.0, 3.0]])
    np.testing.assert_allclose(orc.jacobi(A), [2 - np.sqrt(5), 2 + np.sqrt(5)], atol=1e-15)
    d, e, lam = I.toeplitz(12, 0.5, -0.7)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    np.testing.assert_allclose(orc.jacobi(T), lam, atol=1e-14)


def test_inertia_closed_form(orc):
    d, e, lam = I.toeplitz(30, 1.0, 1.0)
    Q = I.haar_q(30, 4)
    A = Q @ (np.diag(d) + np.diag(e, 1) + np.diag(e, -1)) @ Q.T
    A = 0.5 * (A + A.T)
    for k in range(29):
        x = 0.5 * (lam[k] + lam[k + 1])
        assert orc.inertia(A, x) == k + 1
    assert orc.inertia(A, lam[0] - 1) == 0 and orc.inertia(A, lam[-1] + 1) == 30


# ------------------------------------------------------ tridiagonalisation
@pytest.mark.parametrize("n", [1, 2, 3, 5, 16])
def test_eigvalsh_vs_jacobi(orc, n):
    A = I.semicircle(n, 100 + n)
    np.testing.assert_allclose(orc.eigvalsh(A), orc.jacobi(A), atol=1e-13)


def test_eigvalsh_qdq_prescribed_spectrum(orc):
    n = 200
    D = np.sort(I.rng(7).uniform(-10, 10, n))
    A = I.qdq(D, 8)
    got = orc.eigvalsh(A)
    assert np.abs(got - D).max() <= 50 * np.sqrt(n) * EPS * 10


def test_eigvalsh_inertia_pinned(orc):
    n = 48
    A = I.semicircle(n, 21)
    lam = orc.eigvalsh(A)
    for k in range(n - 1):
        x = 0.5 * (lam[k] + lam[k + 1])
        assert orc.inertia(A, x) == k + 1


def test_tridiagonalize_invariants(orc):
    n = 64
    A = I.semicircle(n, 5)
    d, e = orc.tridiagonalize(A)
    assert abs(d.sum() - np.trace(A)) < 1e-13
    fro = np.sqrt((d ** 2).sum() + 2 * (e ** 2).sum())
    assert abs(fro - np.linalg.norm(A)) < 1e-13
    # lower triangle only is read: garbage in the strict upper triangle is ignored
    B = np.tril(A) + np.triu(np.full((n, n), np.nan), 1)
    d2, e2 = orc.tridiagonalize(B)
    np.testing.assert_array_equal(d, d2)
    np.testing.assert_array_equal(e, e2)


def test_tridiagonalize_of_tridiagonal_is_signed_identity(orc):
    d, e = I.random_tridiagonal(20, 9)
    T = np.diag(d) + np.diag(e, -1)
    d2, e2 = orc.tridiagonalize(T)
    np.testing.assert_allclose(d2, d, atol=1e-15)
    np.testing.assert_allclose(np.abs(e2), np.abs(e), atol=1e-15)


# ---------------------------------------------------------------- panel QR
@pytest.mark.parametrize("m,nc", [(40, 8), (9, 8), (8, 8), (5, 8), (64, 1), (2, 3)])
def test_panel_qr_factorisation_and_wy_identity(orc, m, nc):
    P0 = I.rng(m * 31 + nc).standard_normal((m, nc))
    R, U, T, r = orc.panel_qr(P0)
    assert r == min(nc, m - 1)
    assert np.all(np.tril(R, -1) == 0.0)
    Q = np.eye(m) - U @ T @ U.T
    np.testing.assert_allclose(Q.T @ Q, np.eye(m), atol=1e-14)
    np.testing.assert_allclose(Q @ R, P0, atol=1e-13)
    assert np.allclose(np.triu(U[:r, :r]), np.eye(r))  # unit lower trapezoidal
    assert np.all(np.tril(T, -1) == 0.0)
    # Cor. 3.7: U^T U = T^-1 + T^-T
    if r:
        Ti = np.linalg.inv(T)
        np.testing.assert_allclose(U.T @ U, Ti + Ti.T, atol=1e-12)
    # compact WY equals the explicit product of the reflectors H_0 ... H_{r-1}
    H = np.eye(m)
    for k in range(r):
        v = U[:, k]
        H = H @ (np.eye(m) - T[k, k] * np.outer(v, v))
    np.testing.assert_allclose(H, Q, atol=1e-14)
    # R agrees with LAPACK's QR up to the sign of each row (uniqueness)
    if m >= nc and r == nc:
        R_lapack = np.linalg.qr(P0, mode="r")
        np.testing.assert_allclose(np.abs(R[:nc]), np.abs(R_lapack), atol=1e-13)


# ------------------------------------------------------------ full-to-band
@pytest.mark.parametrize("n,b", [(40, 1), (40, 3), (40, 8), (41, 8), (37, 36), (64, 16), (33, 32), (5, 8)])
def test_full_to_band_structure_and_spectrum(orc, n, b):
    A = I.semicircle(n, 1000 + 7 * n + b)
    lam = np.linalg.eigvalsh(A)  # library routine on the input
    B = orc.full_to_band(A, b)
    assert band_excess(B, b) == 0.0
    np.testing.assert_array_equal(B, B.T)
    np.testing.assert_allclose(np.linalg.eigvalsh(B), lam, atol=1e-13)
    assert abs(np.trace(B) - np.trace(A)) < 1e-13
    assert abs(np.linalg.norm(B) - np.linalg.norm(A)) < 1e-13


def test_full_to_band_b1_matches_tridiagonalize(orc):
    A = I.semicircle(50, 77)
    B = orc.full_to_band(A, 1)
    d, e = orc.tridiagonalize(A)
    np.testing.assert_allclose(np.diag(B), d, atol=1e-14)
    np.testing.assert_allclose(np.diag(B, -1), e, atol=1e-14)


def test_full_to_band_first_panel_is_qr(orc):
    n, b = 30, 6
    A = I.semicircle(n, 3)
    B = orc.full_to_band(A, b)
    R_lapack = np.linalg.qr(A[b:, :b], mode="r")
    np.testing.assert_allclose(np.abs(B[b:2 * b, :b]), np.abs(R_lapack), atol=1e-14)
    np.testing.assert_array_equal(B[:b, :b], A[:b, :b])


def test_full_to_band_jacobi_small(orc):
    A = I.semicircle(12, 9)
    B = orc.full_to_band(A, 3)
    np.testing.assert_allclose(orc.jacobi(B), orc.jacobi(A), atol=1e-13)


# ------------------------------------------------------------ band-to-band
@pytest.mark.parametrize("n,b,h", [(40, 2, 1), (40, 4, 2), (41, 8, 4), (64, 16, 8), (37, 6, 3), (40, 6, 2), (40, 8, 2), (33, 5, 1), (20, 16, 8), (9, 8, 4), (3, 2, 1)])
def test_band_to_band_structure_and_spectrum(orc, n, b, h):
    A = I.random_band(n, b, 2000 + n + 13 * b + h)
    lam = np.linalg.eigvalsh(A)
    C = orc.band_to_band(A, b, h)
    assert band_excess(C, h) == 0.0
    # the two update lines add U V^T and V U^T in separate passes, so the
    # result is symmetric to rounding, not bitwise
    np.testing.assert_allclose(C, C.T, atol=4 * EPS * np.linalg.norm(A))
    np.testing.assert_allclose(np.linalg.eigvalsh(C), lam, atol=1e-13)
    assert abs(np.trace(C) - np.trace(A)) < 1e-13
    assert abs(np.linalg.norm(C) - np.linalg.norm(A)) < 1e-13


@pytest.mark.parametrize("n,b,h", [(40, 4, 2), (53, 8, 4), (40, 6, 2), (30, 2, 1)])
def test_band_to_band_printed_nc_gives_same_bits(orc, n, b, h):
    """Reading A6: the printed update range h+3b and the tight one agree
    exactly, because every extra entry the printed range covers is zero."""
    A = I.random_band(n, b, 3000 + n + b)
    np.testing.assert_array_equal(orc.band_to_band(A, b, h), orc.band_to_band(A, b, h, nc_paper=True))


@pytest.mark.parametrize("n,b,h", [(48, 8, 4), (45, 6, 3), (40, 4, 1), (30, 2, 1)])
def test_band_to_band_fill_stays_below_2b(orc, n, b, h):
    """Reading A9: between chases no entry lies 2b or more off the diagonal,
    so packed storage with 2b diagonals holds every intermediate state."""
    A = I.random_band(n, b, 4000 + n)
    worst = 0
    for k in range(0, 400, 3):
        worst = max(worst, max_fill(orc.band_to_band(A, b, h, max_chases=k)))
    assert worst <= 2 * b - 1
    assert worst > b  # bulges do appear


def test_band_to_band_jacobi_small(orc):
    A = I.random_band(14, 4, 17)
    C = orc.band_to_band(A, 4, 2)
    np.testing.assert_allclose(orc.jacobi(C), orc.jacobi(A), atol=1e-13)


def test_band_to_band_of_narrower_band_keeps_spectrum(orc):
    # an input that is already of band h still goes through valid similarities
    A = I.random_band(30, 2, 5)
    C = orc.band_to_band(A, 4, 2)
    np.testing.assert_allclose(np.linalg.eigvalsh(C), np.linalg.eigvalsh(A), atol=1e-13)
    assert band_excess(C, 2) == 0.0


# --------------------------------------------------------------- pipeline
def test_stage_pipeline_matches_direct(orc):
    A, D = I.qdq(np.linspace(-1, 1, 96), 12), np.linspace(-1, 1, 96)
    via = orc.eigvalsh_via_stages(A, 16)
    direct = orc.eigvalsh(A)
    np.testing.assert_allclose(via, direct, atol=2e-14)
    np.testing.assert_allclose(via, D, atol=1e-13)


def test_band_schedule(orc):
    assert orc.band_schedule(32) == [32, 16, 8, 4, 2, 1]
    assert orc.band_schedule(6) == [6, 3, 1]
    assert orc.band_schedule(1) == [1]


@pytest.mark.parametrize("n,b,h", [(64, 8, 4), (61, 6, 3), (50, 8, 2), (45, 8, 1), (70, 16, 8), (30, 2, 1)])
def test_band_to_band_wavefront_legality(orc, n, b, h):
    """Chase (i, j) conflicts with (i-1, j+2): the pipeline t = 2i + j that
    the Fig. 2 caption pictures depends on the order inside a time step,
    while t = 3i + j (chase (i, j) waits for (i-1, j+2)) reproduces the
    sequential order of Algorithm 4.2 bit for bit in either tie order."""
    A = I.random_band(n, b, 5000 + n + b)
    seq = orc.band_to_band(A, b, h)
    for tie in (False, True):
        np.testing.assert_array_equal(orc.band_to_band_wavefront(A, b, h, 3, tie), seq)
    two = [np.array_equal(orc.band_to_band_wavefront(A, b, h, 2, tie), seq) for tie in (False, True)]
    assert not all(two)


def test_bisect_range_matches_full(orc):
    d, e = I.random_tridiagonal(90, 12)
    full = orc.bisect(d, e, 1e-14)
    np.testing.assert_array_equal(orc.bisect_range(d, e, 10, 33, 1e-14), full[10:33])


@pytest.mark.parametrize("n,b", [(40, 5), (64, 1), (33, 8), (7, 6)])
def test_band_inertia_counts(orc, n, b):
    """Sylvester: negative LDL^T pivots of B - xI count the eigenvalues below
    x; pinned to the eigenvalues of the dense matrix (LAPACK) at shifts in
    the middle of spectral gaps, and to the tridiagonal Sturm count at b = 1."""
    AB = I.random_band_packed(n, b, 2 * b + 2, 7100 + n + b)
    B = I.band_to_dense(AB)
    lam = np.linalg.eigvalsh(B)
    xs = [lam[0] - 1.0, lam[-1] + 1.0] + [0.5 * (lam[k] + lam[k + 1]) for k in range(0, n - 1, max(1, n // 7))]
    for x in xs:
        want = int((lam < x).sum())
        assert orc.band_inertia(AB, b, x) == want
        assert orc.inertia(B, x) == want
        if b == 1:
            assert orc.sturm_count(AB[0], AB[1, : n - 1], x) == want


def test_band_inertia_diagonal_closed_form(orc):
    d = np.array([3.0, -1.0, 2.0, -5.0, 0.5])
    AB = np.zeros((3, 5))
    AB[0] = d
    for x in (-6.0, -2.0, 0.0, 1.0, 2.5, 4.0):
        assert orc.band_inertia(AB, 2, x) == int((d < x).sum())


def test_inertia_lapack_counts(orc):
    """LAPACK Bunch-Kaufman LDL^T as the factorisation step: pinned to
    eigenvalue counts, including 2x2 pivots (a zero-diagonal matrix)."""
    A = I.semicircle(60, 77)
    lam = np.linalg.eigvalsh(A)
    for x in [lam[0] - 1.0, 0.5 * (lam[9] + lam[10]), 0.5 * (lam[40] + lam[41]), lam[-1] + 1.0]:
        assert orc.inertia_lapack(A, x) == int((lam < x).sum())
    K = np.kron(np.eye(5), np.array([[0.0, 1.0], [1.0, 0.0]]))  # eigenvalues +-1, forces 2x2 pivots
    assert orc.inertia_lapack(K, 0.0) == 5
    assert orc.inertia_lapack(K, -2.0) == 0
    assert orc.inertia_lapack(K, 2.0) == 10


@pytest.mark.parametrize("n", [1, 2, 3, 10, 257])
def test_sturm_minors_equals_pivot_count(orc, n):
    """The minors count (Sturm's theorem) and the LDL^T pivot count agree
    with the eigenvalue count of the dense matrix at shifts inside gaps."""
    d, e = I.random_tridiagonal(n, 11000 + n)
    T = np.diag(d) + (np.diag(e, -1) + np.diag(e, 1) if n > 1 else 0.0)
    lam = np.linalg.eigvalsh(T)
    xs = [lam[0] - 1.0, lam[-1] + 1.0] + [0.5 * (lam[k] + lam[k + 1]) for k in range(n - 1)][:: max(1, n // 9)]
    for x in xs:
        want = int((lam < x).sum())
        assert orc.sturm_count_minors(d, e, x) == want
        assert orc.sturm_count(d, e, x) == want


def test_sturm_minors_extreme_scales_and_zero(orc):
    d, e = I.random_tridiagonal(400, 11100)
    xs = [-3.0, -0.7, 0.0, 0.4, 2.9]
    base = [orc.sturm_count_minors(d, e, x) for x in xs]
    for k in (-600, -300, 300, 600):  # exact power-of-two scalings: no overflow, same counts
        s = 2.0 ** k
        assert [orc.sturm_count_minors(d * s, e * s, x * s) for x in xs] == base
    z = np.zeros(50)
    # x exactly at an eigenvalue: a zero minor counts as a sign change, as a
    # zero pivot counts as negative under the pivmin rule
    assert orc.sturm_count_minors(z, z[:49], 0.0) == orc.sturm_count(z, z[:49], 0.0) == 50
    assert orc.sturm_count_minors(z, z[:49], 1.0) == 50
    assert orc.sturm_count_minors(z, z[:49], -1.0) == 0
    np.testing.assert_array_equal(orc.bisect(z, z[:49], 1e-14), z)  # T = 0: every eigenvalue exactly 0


def test_bisect_power_of_two_scale_invariance(orc):
    """The bisection runs on the exactly rescaled matrix, so scaling T by
    2^k scales every computed eigenvalue by exactly 2^k."""
    d, e = I.random_tridiagonal(150, 11200)
    ref = orc.bisect(d, e, 1e-14)
    for k in (-400, -7, 5, 400):
        s = 2.0 ** k
        np.testing.assert_array_equal(orc.bisect(d * s, e * s, 1e-14), ref * s)
