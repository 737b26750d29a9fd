"""The lattice embed's shortcut for m_i = rint(x_i / (d+1)) (step 3 of the
lattice conventions, Appendix A) gives the division's m_i and delta_i.

The kernel takes k = rint(x RN(1/(d+1))) and rem = RN(x - (d+1) k), keeps
them when |rem| <= 0.499 (d+1) and otherwise divides (the bound holds for
|k| < 2^40; larger values fail the kernel's 1e12 range check).  This
emulates that rule in FP64 numpy (IEEE round-to-nearest, the kernel's
operation order, no fused operations) on random values, values near +-1e12
(d+1), exact multiples, exact half-way points and their FP64 neighbours, and
the grid-like coordinates that pixel positions produce, and compares with
rint(x / (d+1)) and x - (d+1) rint(x / (d+1)).
"""
import numpy as np
import pytest


def _shortcut(x, d1):
    inv = 1.0 / d1
    q = np.rint(x * inv)
    rem = x - d1 * q
    keep = np.abs(rem) <= 0.499 * d1
    qd = np.rint(x / d1)
    return np.where(keep, q, qd), np.where(keep, rem, x - d1 * qd), keep


@pytest.mark.parametrize("d1", [2, 3, 4, 6, 7, 9])
def test_shortcut_equals_division(d1):
    rng = np.random.default_rng(d1)
    k = rng.integers(-10 ** 6, 10 ** 6, 200_000).astype(np.float64)
    big = rng.integers(-2 ** 40, 2 ** 40, 200_000).astype(np.float64)
    half, bighalf = (k + 0.5) * d1, (big + 0.5) * d1
    g = np.arange(-3000, 3000, dtype=np.float64)
    x = np.concatenate([
        rng.uniform(-1e3, 1e3, 400_000), rng.uniform(-1e12, 1e12, 200_000) * d1, rng.normal(0, 1, 200_000),
        rng.uniform(-2 ** 40, 2 ** 40, 200_000) * d1,
        half, np.nextafter(half, np.inf), np.nextafter(half, -np.inf), k * d1, np.nextafter(k * d1, np.inf),
        bighalf, np.nextafter(bighalf, np.inf), np.nextafter(bighalf, -np.inf),
        *[g / 3.0 * i for i in range(1, 7)], g / 80.0 * 7, g / 13.0 * 5,
    ])
    q, rem, keep = _shortcut(x, float(d1))
    qd = np.rint(x / d1)
    np.testing.assert_array_equal(q, qd)
    np.testing.assert_array_equal(rem, x - d1 * qd)
    # the shortcut decides almost everywhere away from half-way points
    assert keep[:400_000].mean() > 0.99


def test_rank_keys_order_like_doubles():
    # the ranks compare deltas as order-preserving 64-bit integers (-0 as +0)
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 3, 5000), [0.0, -0.0, 1e-300, -1e-300, 2.5, -2.5]])
    bits = (v + 0.0).view(np.int64)
    key = np.where(bits < 0, bits ^ np.int64(0x7FFFFFFFFFFFFFFF), bits)
    i, j = rng.integers(0, v.size, (2, 200_000))
    np.testing.assert_array_equal(key[i] > key[j], v[i] > v[j])
    np.testing.assert_array_equal(key[i] == key[j], v[i] == v[j])
