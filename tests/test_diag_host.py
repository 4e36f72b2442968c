"""CPU checks of the host-side spectral diagnostics of the C ABI (no GPU).

ok_hessenberg_eigenvalues (implicit double-shift QR) against closed forms:
polynomial roots through a companion matrix, roots of unity of the cyclic
shift (a matrix on which unshifted and plain Francis shifts stall), a rotation,
Jordan and triangular matrices; against LAPACK (numpy) on random Hessenberg
matrices, including extreme scaling, grading and tiny subdiagonals.
ok_givens_unrotate against the Givens reduction the Arnoldi kernel applies
(restated here from its definition: rows (i, i+1) map (a, b) to
(c a + s b, -s a + c b), the new rotation zeroes the subdiagonal).
"""
import numpy as np
import pytest

import paper_1603_04570_gb300 as ok

scipy_opt = pytest.importorskip("scipy.optimize")


def match(a, b):
    """Largest distance of an optimal one-to-one pairing of two eigenvalue sets."""
    assert len(a) == len(b)
    if len(a) == 0:
        return 0.0
    C = np.abs(np.asarray(a)[:, None] - np.asarray(b)[None, :])
    r, c = scipy_opt.linear_sum_assignment(C)
    return C[r, c].max()


def hessenberg(rng, k, scale=1.0):
    return np.triu(rng.standard_normal((k, k)), -1) * scale


def test_polynomial_roots_from_the_companion_matrix():
    roots = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, -0.5])
    c = np.poly(roots)
    k = len(roots)
    C = np.zeros((k, k))
    C[0, :] = -c[1:]
    C[np.arange(1, k), np.arange(k - 1)] = 1.0
    lam = ok.ok_hessenberg_eigenvalues(C)
    assert np.abs(lam.imag).max() == 0.0
    assert np.abs(np.sort(lam.real) - np.sort(roots)).max() < 1e-9


@pytest.mark.parametrize("k", [2, 3, 4, 5, 8, 17, 63])
def test_cyclic_shift_gives_the_roots_of_unity(k):
    P = np.zeros((k, k))
    P[np.arange(1, k), np.arange(k - 1)] = 1.0
    P[0, k - 1] = 1.0
    assert match(ok.ok_hessenberg_eigenvalues(P), np.exp(2j * np.pi * np.arange(k) / k)) < 1e-13


def test_small_closed_forms():
    lam = ok.ok_hessenberg_eigenvalues(np.array([[0.0, -1.0], [1.0, 0.0]]))
    assert match(lam, np.array([1j, -1j])) == 0.0
    lam = ok.ok_hessenberg_eigenvalues(np.array([[2.0, 3.0], [1.0, 4.0]]))     # (l-1)(l-5)
    assert match(lam, np.array([1.0, 5.0])) < 1e-15
    assert ok.ok_hessenberg_eigenvalues(np.array([[7.5]]))[0] == 7.5
    assert ok.ok_hessenberg_eigenvalues(np.zeros((0, 0))).size == 0
    assert np.all(ok.ok_hessenberg_eigenvalues(np.zeros((4, 4))) == 0)
    J = np.eye(5) + np.diag(np.ones(4), 1)                                     # one Jordan block
    assert np.abs(ok.ok_hessenberg_eigenvalues(J) - 1.0).max() < 1e-12


def test_triangular_and_reducible_matrices():
    rng = np.random.default_rng(3)
    T = np.triu(rng.standard_normal((30, 30)))
    assert match(ok.ok_hessenberg_eigenvalues(T), np.diag(T).astype(complex)) == 0.0
    H = hessenberg(rng, 30)
    H[10, 9] = H[20, 19] = 0.0                                                  # three blocks
    assert match(ok.ok_hessenberg_eigenvalues(H), np.linalg.eigvals(H)) < 1e-12 * np.abs(H).max()


def test_symmetric_tridiagonal_against_eigvalsh():
    rng = np.random.default_rng(4)
    d, e = rng.standard_normal(50), rng.standard_normal(49)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = ok.ok_hessenberg_eigenvalues(T)
    assert np.abs(lam.imag).max() == 0.0
    assert match(lam, np.linalg.eigvalsh(T).astype(complex)) < 1e-12


def test_random_hessenberg_against_lapack():
    rng = np.random.default_rng(0)
    for k in list(range(1, 64)) + [64, 100]:
        H = hessenberg(rng, k)
        assert match(ok.ok_hessenberg_eigenvalues(H), np.linalg.eigvals(H)) < 1e-10 * np.abs(H).max(), k


@pytest.mark.parametrize("scale", [1e-150, 1e-30, 1e30, 1e100])
def test_scaling_is_exact(scale):
    rng = np.random.default_rng(1)
    H = hessenberg(rng, 20)
    lam = ok.ok_hessenberg_eigenvalues(H)
    assert match(ok.ok_hessenberg_eigenvalues(H * scale) / scale, lam) < 1e-13 * np.abs(lam).max()


def test_graded_and_nearly_reducible_matrices():
    rng = np.random.default_rng(2)
    G = hessenberg(rng, 30) * np.logspace(0, -12, 30)[None, :]
    assert match(ok.ok_hessenberg_eigenvalues(G), np.linalg.eigvals(G)) < 1e-12
    S = hessenberg(rng, 30)
    S[np.arange(1, 30), np.arange(29)] *= 1e-14
    assert match(ok.ok_hessenberg_eigenvalues(S), np.linalg.eigvals(S)) < 1e-12


def test_entries_below_the_subdiagonal_are_ignored():
    A = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [np.nan, 0.0, 3.0]])
    assert match(ok.ok_hessenberg_eigenvalues(A), np.array([1.0, 2.0, 3.0])) == 0.0


@pytest.mark.parametrize("bad", [np.array([[np.nan]]), np.array([[1.0, np.inf], [1.0, 2.0]])])
def test_nonfinite_hessenberg_is_rejected(bad):
    with pytest.raises(ok.OkError) as e:
        ok.ok_hessenberg_eigenvalues(bad)
    assert e.value.status == ok.OK_ERR_NONFINITE


def test_invalid_sizes_are_rejected():
    lib = ok.load()
    buf = np.zeros(16)
    p = buf.ctypes.data
    assert lib.ok_hessenberg_eigenvalues(-1, p, 4, p, p) == ok.OK_ERR_INVALID_ARG
    assert lib.ok_hessenberg_eigenvalues(3, p, 2, p, p) == ok.OK_ERR_INVALID_ARG       # ldh < k
    assert lib.ok_hessenberg_eigenvalues(2, None, 2, p, p) == ok.OK_ERR_INVALID_ARG
    assert lib.ok_hessenberg_eigenvalues(4097, p, 4097, p, p) == ok.OK_ERR_INVALID_ARG    # k cap
    assert lib.ok_hessenberg_eigenvalues(1_500_000_000, p, 1_500_000_000, p, p) == ok.OK_ERR_INVALID_ARG
    assert lib.ok_givens_unrotate(3, p, 3, p, p) == ok.OK_ERR_INVALID_ARG              # ldh < k + 1
    assert lib.ok_givens_unrotate(-1, p, 4, p, p) == ok.OK_ERR_INVALID_ARG
    assert lib.ok_givens_unrotate(0, None, 1, None, None) == ok.OK_SUCCESS


def givens_reduce(Hbar):
    """R and the rotations of the least-squares update, column by column."""
    k = Hbar.shape[1]
    R = Hbar.copy()
    cs, sn = np.zeros(k), np.zeros(k)
    for j in range(k):
        for i in range(j):
            a, b = R[i, j], R[i + 1, j]
            R[i, j], R[i + 1, j] = cs[i] * a + sn[i] * b, -sn[i] * a + cs[i] * b
        a, b = R[j, j], R[j + 1, j]
        r = np.hypot(a, b)
        cs[j], sn[j] = (a / r, b / r) if r > 0 else (1.0, 0.0)
        R[j, j], R[j + 1, j] = r, 0.0
    return R, cs, sn


@pytest.mark.parametrize("k", [1, 2, 7, 40, 63])
def test_givens_restoration_inverts_the_reduction(k):
    rng = np.random.default_rng(k)
    Hbar = np.triu(rng.standard_normal((k + 1, k)), -1)
    Hbar[np.arange(1, k + 1), np.arange(k)] = np.abs(Hbar[np.arange(1, k + 1), np.arange(k)])
    R, cs, sn = givens_reduce(Hbar)
    assert np.abs(np.tril(R, -1)).max() == 0.0
    back = ok.ok_givens_unrotate(R, cs, sn)
    assert np.abs(back - Hbar).max() < 1e-14 * np.abs(Hbar).max() * k
    # a breakdown column (zero subdiagonal) and a zero column survive the round trip
    Hbar[k, k - 1] = 0.0
    Hbar[:, 0] = 0.0
    R, cs, sn = givens_reduce(Hbar)
    assert np.abs(ok.ok_givens_unrotate(R, cs, sn) - Hbar).max() < 1e-14 * max(np.abs(Hbar).max(), 1) * k


def test_leading_columns_are_the_shorter_arnoldi_matrix():
    """Restoring only the first m columns of a reduction gives Hbar_m."""
    rng = np.random.default_rng(9)
    Hbar = np.triu(rng.standard_normal((21, 20)), -1)
    R, cs, sn = givens_reduce(Hbar)
    m = 8
    back = ok.ok_givens_unrotate(R[:m + 1, :m], cs[:m], sn[:m])
    assert np.abs(back - Hbar[:m + 1, :m]).max() < 1e-14 * np.abs(Hbar).max() * m
