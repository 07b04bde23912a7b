"""GPU parity of sigma_generator_degrees (deg det and codeg det of a
sigma-basis generator, the two numbers block Wiedemann's rank is read from,
Sec. 3.3) against the oracle's determinant by evaluation and interpolation
(oracle/sigma.py): random polynomial matrices with rows multiplied by powers
of x (nonzero codegrees, rows of different degrees), the choice of the n rows
of least (delta, index) among m, valuations that need the truncation order
raised, and the singular cases.  The block-Wiedemann pipelines in
test_gpu_sigma.py check the rank it gives on GPU-made generators."""
import numpy as np
import pytest

from oracle import sigma

pytestmark = pytest.mark.gpu


def _random_generator(seed, n, e, p, shifts):
    """An n x n polynomial matrix (coefficient-major, e + 1 + max shift
    coefficients) whose row r is a random row of degree <= e times x^shifts[r]."""
    rng = np.random.default_rng(seed)
    top = e + 1 + max(shifts)
    U = np.zeros((top, n, n), dtype=np.int64)
    for r in range(n):
        U[shifts[r]:shifts[r] + e + 1, r, :] = rng.integers(0, p, (e + 1, n))
    return U


def _oracle_degrees(U, p):
    dp = sigma.det_poly(sigma.trim(U.astype(object)), p)
    assert any(dp), "singular test matrix"
    return sigma.degree_and_codegree(dp)


@pytest.mark.parametrize("seed,n,e,shifts", [
    (1, 1, 3, [2]),
    (2, 3, 2, [0, 1, 3]),
    (3, 5, 1, [0, 0, 2, 1, 0]),
    (4, 4, 3, [5, 0, 0, 2]),
    (5, 16, 1, [0] * 8 + [1] * 8),
    (6, 3, 2, [20, 21, 22]),            # codeg 63: the truncation order doubles past 32
])
def test_degrees_against_the_oracle(lib, seed, n, e, shifts):
    p = 65521
    U = _random_generator(seed, n, e, p, shifts)
    want = _oracle_degrees(U, p)
    got = lib.sigma_generator_degrees(p, U.astype(np.uint32), [0] * n, n)
    assert got == want


def test_generator_rows_are_the_least_delta(lib):
    # m = 6 rows, n = 3: the generator is rows 4, 1, 5 (delta 0, 1, 1; ties by
    # index), and the other rows (larger delta) are junk that must not count
    p, n, m = 1_000_003, 3, 6
    rng = np.random.default_rng(9)
    G = _random_generator(10, n, 2, p, [1, 0, 2])
    P = rng.integers(0, p, (G.shape[0], m, m)).astype(np.int64)
    for i, r in enumerate((4, 1, 5)):
        P[:, r, :n] = G[:, i, :]
    delta = [3, 1, 2, 4, 0, 1]
    want = _oracle_degrees(G, p)
    assert lib.sigma_generator_degrees(p, P.astype(np.uint32), delta, n) == want


def test_singular_generators_are_refused(lib):
    p, n = 65521, 3
    U = _random_generator(11, n, 2, p, [0, 0, 0])
    Z = U.copy()
    Z[:, 1, :] = 0                       # a zero row
    with pytest.raises(lib.FFSPMVError) as e:
        lib.sigma_generator_degrees(p, Z.astype(np.uint32), [0] * n, n)
    assert e.value.status == 5
    E = U.copy()
    E[:, 2, :] = E[:, 0, :]              # two equal rows: det = 0, no pivot below the limit
    with pytest.raises(lib.FFSPMVError) as e:
        lib.sigma_generator_degrees(p, E.astype(np.uint32), [0] * n, n, max_precision=64)
    assert e.value.status == 5
