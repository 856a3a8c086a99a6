"""The integer the split-precision kernels peel into BF16 slices, T = rint(v 2^k) with ties to even
(Ozaki, Ogita, Oishi and Rump's error-free splitting), computed from the bits of v by the library's own
routine (run on the host through df_rint_pow2) against numpy's exact scaling and rounding. CPU only."""
import numpy as np
import pytest

from paper_1707_03771_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding


def _ref(v, k):
    return np.rint(np.ldexp(v, k)).astype(np.int64)


def test_random_values_at_row_exponents(lib):
    """Values of every magnitude with the exponent of their row (|v 2^-e| < 1), for 3, 5 and 7 slices."""
    rng = np.random.default_rng(11)
    v = rng.standard_normal(200_000) * np.exp2(rng.integers(-60, 60, 200_000))
    _, ev = np.frexp(v)
    e = ev + rng.integers(0, 45, v.size)            # the row's exponent is at least the value's
    for S in (3, 5, 7):
        k = (7 * S - e).astype(np.int32)
        assert np.array_equal(lib.rint_pow2(v, k), _ref(v, k))


def test_exact_ties_round_to_even(lib):
    rng = np.random.default_rng(12)
    j = rng.integers(-2**40, 2**40, 50_000)
    k = rng.integers(-30, 60, j.size).astype(np.int32)
    v = np.ldexp((2 * j + 1).astype(np.float64), -(k + 1))   # v 2^k = j + 1/2 exactly
    got = lib.rint_pow2(v, k)
    assert np.array_equal(got, _ref(v, k))
    assert np.all(got % 2 == 0)
    near = np.nextafter(v, np.inf)                            # just above the tie: rounds up
    assert np.array_equal(lib.rint_pow2(near, k), _ref(near, k))


def test_edges(lib):
    """Zero, signed zero, subnormals (the FP64 route), results of 2^52 and more, and the last shifts
    (d = 53: 1/2 and 3/4; d = 54: below 1/2)."""
    sub = np.ldexp(np.arange(1, 200, dtype=np.float64), -1074)
    v = np.concatenate([[0.0, -0.0, 1.0, 1.5, -1.5, 1.0, 1.99, 1.5, -1.5, 3.0],
                        sub, -sub, [2.0**-1022, np.nextafter(2.0**-1022, 0)]])
    k = np.concatenate([[40, 40, -1, -1, -1, -2, -2, 60, 60, 51],
                        np.full(sub.size, 1070), np.full(sub.size, 1072), [1030, 1080]]).astype(np.int32)
    assert np.array_equal(lib.rint_pow2(v, k), _ref(v, k))


def test_rejects_bad_arguments(lib):
    L = lib.load()
    assert L.df_rint_pow2(None, None, -1, None) == lib.DF_E_ARG
    assert L.df_rint_pow2(None, None, 3, None) == lib.DF_E_ARG
    assert L.df_rint_pow2(None, None, 0, None) == lib.DF_OK
