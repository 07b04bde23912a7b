"""The arithmetic the x-panel kernel relies on for m > 2^16, restated with
Python integers and checked on the CPU: the Montgomery reduction of v' x
with v' = v 2^32 mod m gives v x mod m below 2m (odd m < 2^31), Newton's
iteration gives -1/m mod 2^32, and a row's pair of u32 sums (low 16 bits of
every added value, and the rest) stays below 2^31 for up to 2^15 terms below
2^32, however the terms are grouped into added values.  The kernel itself is
checked against the oracle in test_gpu_spmv.py."""
import numpy as np
import pytest

MASK32 = (1 << 32) - 1


def neg_inv32(m):
    y = m
    for _ in range(4):
        y = (y * (2 - m * y)) & MASK32
    return (-y) & MASK32


def mont_red(v, x, m, mneg):
    lo, hi = (v * x) & MASK32, (v * x) >> 32
    u = (lo * mneg) & MASK32
    return hi + ((u * m) >> 32) + (1 if lo else 0)


ODD_MODULI = [65537, 65539, 1_000_003, 2**31 - 1, 2**31 - 3, 2**30 + 1, 3 * 5 * 7 * 11 * 13 * 17 * 19 * 23 + 2]


@pytest.mark.parametrize("m", ODD_MODULI)
def test_newton_inverse(m):
    assert m % 2 == 1
    assert (m * neg_inv32(m)) & MASK32 == MASK32          # m (-1/m) = -1 mod 2^32


@pytest.mark.parametrize("m", ODD_MODULI)
def test_montgomery_term_is_the_product_below_2m(m):
    rng = np.random.default_rng(m % 9973)
    mneg = neg_inv32(m)
    vs = [int(t) for t in rng.integers(0, m, 4000)] + [0, 1, m - 1]
    xs = [int(t) for t in rng.integers(0, 2**32, 4000)] + [0, 1, m - 1]  # x < 2^32 is all the bound needs
    for v, x in zip(vs, xs):
        vp = (v << 32) % m                                  # the layout's stored value
        t = mont_red(vp, x, m, mneg)
        assert t % m == (v * x) % m
        assert t < 2 * m < 2**32
    # the extremes: largest v' and x
    for vp in (m - 1, m - 2):
        for x in (MASK32, m - 1):
            assert mont_red(vp, x, m, mneg) < 2 * m


def test_split_row_sums_stay_below_2_31():
    # 2^15 terms at the largest value below 2^32, added one by one, in pairs,
    # in runs of eight (a pack's segmented sum) and as two cluster partial sums
    rng = np.random.default_rng(5)
    L = 1 << 15
    for terms in ([MASK32] * L, [int(t) for t in rng.integers(2**31, 2**32, L)]):
        for group in (1, 2, 8, 1000, L // 2):
            lo = hi = 0
            for k in range(0, L, group):
                c = sum(terms[k:k + group])
                lo += c & 0xFFFF
                hi += c >> 16
                assert lo < 2**31 and hi < 2**31
            assert lo + (hi << 16) == sum(terms)
