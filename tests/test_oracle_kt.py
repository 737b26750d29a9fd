"""Pins of the oracle's Kleinberg-Tardos rounding of an LP point (end of
Section 5: the rounding behind the LP's factor-2 guarantee for Potts)."""
import numpy as np

from oracle import lp
from paper_1608_06192_gb300 import synthetic as S


def test_hand_worked_phases():
    # four pixels, three labels, four phases worked by hand:
    #   (label 0, 0.5):  pixel 0 (0.6 > 0.5) -> 0
    #   (label 2, 0.7):  nobody (0.6, 0.0, 0.5 are not above 0.7)
    #   (label 1, 0.25): pixel 2 (1.0) -> 1; pixel 3 has exactly 0.25: not above
    #   (label 2, 0.05): pixels 1 (0.6) and 3 (0.5) -> 2
    y = np.array([[0.6, 0.3, 0.1],
                  [0.2, 0.2, 0.6],
                  [0.0, 1.0, 0.0],
                  [0.25, 0.25, 0.5]], dtype=np.float32)
    labs = np.array([0, 2, 1, 2], dtype=np.int32)
    thr = np.array([0.5, 0.7, 0.25, 0.05], dtype=np.float32)
    np.testing.assert_array_equal(lp.kt_round(y, labs[:3], thr[:3]), [0, -1, 1, -1])
    np.testing.assert_array_equal(lp.kt_round(y, labs, thr), [0, 2, 1, 2])


def test_a_labelling_rounds_to_itself():
    rng = np.random.default_rng(0)
    lab = rng.integers(0, 7, size=500)
    y = np.eye(7, dtype=np.float32)[lab]
    pl, pt = S.kt_phases(7, 400, seed=1)
    np.testing.assert_array_equal(lp.kt_round(y, pl, pt), lab)


def test_continuing_a_run_equals_one_run_over_all_phases():
    y = S.dirichlet_labels(300, 5, seed=2)
    pl, pt = S.kt_phases(5, 120, seed=3)
    first = lp.kt_round(y, pl[:8], pt[:8])
    assert (first < 0).any() and (first >= 0).any()
    np.testing.assert_array_equal(lp.kt_round(y, pl[8:], pt[8:], labels=first), lp.kt_round(y, pl, pt))


def _runs(y, runs, phases, seed):
    L = y.shape[1]
    rng = np.random.default_rng(seed)
    out = np.empty((runs, y.shape[0]), dtype=np.int32)
    for r in range(runs):
        pl = rng.integers(0, L, size=phases).astype(np.int32)
        pt = rng.random(phases, dtype=np.float32)
        out[r] = lp.kt_round(y, pl, pt)
    assert (out >= 0).all()
    return out


def test_marginals_and_pairwise_separation_by_simulation():
    # P(x_a = i) = y_a(i), and P(x_a != x_b) is the exact separation
    # probability, at most 2d / (1 + d) <= 2d with d = |y_a - y_b|_1 / 2 (the
    # factor 2 for Potts).  3000 independent roundings; 0.05 is above five
    # standard deviations.
    y = np.array([[0.7, 0.2, 0.1],
                  [0.1, 0.1, 0.8],
                  [0.5, 0.5, 0.0],
                  [0.65, 0.25, 0.1]], dtype=np.float32)
    x = _runs(y, 3000, 60, seed=4)
    for i in range(3):
        np.testing.assert_allclose((x == i).mean(axis=0), y[:, i], atol=0.05)
    for a in range(4):
        for b in range(a + 1, 4):
            p = lp.kt_separation_probability(y[a], y[b])
            d = 0.5 * np.abs(y[a] - y[b]).sum()
            assert p <= 2 * d / (1 + d) + 1e-12
            assert abs((x[:, a] != x[:, b]).mean() - p) <= 0.05


def test_separation_probability_special_cases():
    # equal rows are never separated; disjoint one-hot rows always are; two
    # labels with y_a = (1, 0), y_b = (t, 1 - t): b gets label 0 w.p. t
    e = np.array([0.2, 0.3, 0.5])
    assert lp.kt_separation_probability(e, e) == 0.0
    assert lp.kt_separation_probability([1.0, 0.0], [0.0, 1.0]) == 1.0
    for t in (0.0, 0.3, 0.9):
        assert abs(lp.kt_separation_probability([1.0, 0.0], [t, 1.0 - t]) - (1.0 - t)) <= 1e-15
