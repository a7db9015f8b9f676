"""The cosine transform of walls in y and of the cosine z solve, as the
kernels compute it (no GPU): one complex FFT of length n per column with
Makhoul's row order and pairwise twiddles, against scipy's DCT-II and its
inverse.  Each step below mirrors one step of the device stage; the check
is against the library routine, so a wrong row order, twiddle sign, pairing
or scale fails here."""
import numpy as np
import pytest

sfft = pytest.importorskip("scipy.fft")


def dct_row(r, n):
    """Global row that shared row r receives (forward) or returns to (inverse)."""
    return 2 * r if r < n // 2 else 2 * (n - 1 - r) + 1


def forward(x):
    """X_m = sum_j x_j cos(pi m (2j + 1) / (2n)) for the columns of x."""
    n = x.shape[0]
    w = np.exp(-1j * np.pi * np.arange(n) / (2 * n))
    v = np.array([x[dct_row(r, n)] for r in range(n)])      # rows enter reordered
    Z = np.fft.fft(v, axis=0)                                # DIR = -1, unnormalised
    X = np.empty_like(Z)
    for r in range(n):                                        # the store: X_r from Z_r and Z_{n-r}
        a = Z[r] * w[r]
        b = Z[0 if r == 0 else n - r] * np.conj(w[r])
        X[r] = 0.5 * (a + b)
    return X


def inverse(Y):
    """x with forward(x) = Y, times n (the caller's 1/(nx ny) scaling is
    the periodic inverse's too)."""
    n = Y.shape[0]
    w = np.exp(-1j * np.pi * np.arange(n) / (2 * n))
    V = Y.astype(np.complex128).copy()
    for m in range(1, n // 2 + 1):                            # in place, pair (m, n - m)
        a, b = V[m].copy(), V[n - m].copy()
        d, e = a - 1j * b, a + 1j * b
        V[m] = d * np.conj(w[m])
        if m != n - m:
            V[n - m] = e * w[m]
    v = np.fft.ifft(V, axis=0) * n                            # DIR = +1, unnormalised
    x = np.empty_like(v)
    for r in range(n):                                        # rows leave reordered
        x[dct_row(r, n)] = v[r]
    return x


@pytest.mark.parametrize("n", [2, 4, 6, 10, 12, 30, 48, 512])
def test_forward_is_the_dct_ii(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n, 5)) + 1j * rng.standard_normal((n, 5))
    ref = 0.5 * (sfft.dct(x.real, type=2, axis=0) + 1j * sfft.dct(x.imag, type=2, axis=0))
    assert np.max(np.abs(forward(x) - ref)) < 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("n", [2, 4, 6, 10, 12, 30, 48, 512])
def test_inverse_undoes_forward_up_to_n(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    assert np.max(np.abs(inverse(forward(x)) / n - x)) < 1e-12 * np.max(np.abs(x))


def test_rows_form_a_permutation():
    for n in (2, 6, 30, 512):
        assert sorted(dct_row(r, n) for r in range(n)) == list(range(n))


def test_cosine_modes_diagonalise_the_neumann_difference():
    """The divide of the z solve: cos(pi m (k + 1/2)/n) has eigenvalue
    -(4/h^2) sin^2(pi m/(2n)) under the second difference with no flux
    through the ends."""
    n, h = 12, 0.3
    L = np.zeros((n, n))
    for k in range(n):
        if k > 0:
            L[k, k - 1] += 1; L[k, k] -= 1
        if k < n - 1:
            L[k, k + 1] += 1; L[k, k] -= 1
    L /= h * h
    for m in range(n):
        c = np.cos(np.pi * m * (np.arange(n) + 0.5) / n)
        lam = -4.0 / h ** 2 * np.sin(np.pi * m / (2 * n)) ** 2
        assert np.max(np.abs(L @ c - lam * c)) < 1e-11 * max(1.0, abs(lam))
