"""Pins of the oracle's LP relaxation (Eq. 18-20, Appendix D-E, Algorithm 3)."""
import itertools
import json
import os

import networkx as nx
import numpy as np
import pytest
from scipy.optimize import linprog, minimize

from oracle import crf, lp
from oracle import permutohedral as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _problem(seed, n, L):
    rng = np.random.default_rng(seed)
    f = rng.normal(scale=1.2, size=(n, 3))
    k = crf.BruteGaussian([f], [1.5])
    return k, rng.normal(size=(n, L)), rng


def test_six_point_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "lp_dc_six_points.json")))
    K = np.array(g["K"])
    rank = lp.label_rank(np.array(g["y"]))
    np.testing.assert_array_equal(rank, np.arange(6))
    U = lp.upper_sums_dc(rank, lp.brute_partitioned(K))
    np.testing.assert_allclose(U, g["upper_sums"], rtol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 7, 16, 40])
def test_divide_and_conquer_equals_pairwise_subgradient(n):
    k, phi, rng = _problem(n, n, 3)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    y = rng.dirichlet(np.ones(3), size=n)
    y[: n // 3, 0] = y[0, 0]                      # ties are broken by pixel index
    c = Kd.sum(axis=1)
    G_dc = lp.subgradient_dc(phi, y, c, lp.brute_partitioned(Kd))
    G_pairs = lp.subgradient_pairs(phi, Kd, y)
    np.testing.assert_allclose(G_dc, G_pairs, rtol=1e-12, atol=1e-12)


def test_lp_objective_euler_identity_and_integer_points():
    n, L = 25, 4
    k, phi, rng = _problem(5, n, L)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    c = Kd.sum(axis=1)
    for _ in range(3):
        y = rng.dirichlet(np.ones(L), size=n)
        G = lp.subgradient_dc(phi, y, c, lp.brute_partitioned(Kd))
        np.testing.assert_allclose(lp.s_lp_from_g(y, G), crf.s_lp_pairs(phi, Kd, y), rtol=1e-12)
    x = rng.integers(0, L, n)
    y = np.eye(L)[x]
    G = lp.subgradient_dc(phi, y, c, lp.brute_partitioned(Kd))
    np.testing.assert_allclose(lp.s_lp_from_g(y, G), crf.energy_pairs(phi, Kd, 1 - np.eye(L), x), rtol=1e-12)


def test_subgradient_inequality():
    # G(y) is a subgradient of the convex S_LP: S(z) >= S(y) + <G(y), z - y>
    n, L = 15, 3
    k, phi, rng = _problem(6, n, L)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    c = Kd.sum(axis=1)
    y = rng.dirichlet(np.ones(L), size=n)
    G = lp.subgradient_dc(phi, y, c, lp.brute_partitioned(Kd))
    for _ in range(20):
        z = rng.dirichlet(np.ones(L), size=n)
        assert crf.s_lp_pairs(phi, Kd, z) >= crf.s_lp_pairs(phi, Kd, y) + np.sum(G * (z - y)) - 1e-10


def _two_label_instance(seed=7, n=8):
    rng = np.random.default_rng(seed)
    f = rng.normal(scale=1.0, size=(n, 2))
    Kd = crf.BruteGaussian([f], [1.0]).dense()
    np.fill_diagonal(Kd, 0.0)
    phi = rng.normal(scale=1.0, size=(n, 2))
    return Kd, phi


def _lp_optimum(Kd, phi):
    n, L = phi.shape
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    nv = n * L + len(pairs) * L
    cvec = np.zeros(nv)
    cvec[: n * L] = phi.reshape(-1)
    A_ub, b_ub = [], []
    for p, (a, b) in enumerate(pairs):
        for i in range(L):
            zi = n * L + p * L + i
            cvec[zi] = Kd[a, b]           # ordered pairs / 2 = unordered pairs
            for sgn in (1, -1):
                row = np.zeros(nv)
                row[a * L + i], row[b * L + i], row[zi] = sgn, -sgn, -1
                A_ub.append(row)
                b_ub.append(0.0)
    A_eq = np.zeros((n, nv))
    for a in range(n):
        A_eq[a, a * L:(a + 1) * L] = 1
    res = linprog(cvec, A_ub=np.array(A_ub), b_ub=b_ub, A_eq=A_eq, b_eq=np.ones(n), bounds=(0, None),
                  method="highs")
    assert res.status == 0
    return res.fun


def test_two_label_lp_is_tight_min_cut():
    Kd, phi = _two_label_instance()
    n = len(phi)
    brute = min(crf.energy_pairs(phi, Kd, 1 - np.eye(2), np.array(x)) for x in itertools.product((0, 1), repeat=n))
    G = nx.DiGraph()
    const = 0.0
    for a in range(n):
        m = min(phi[a])
        const += m
        G.add_edge("s", a, capacity=phi[a, 1] - m)
        G.add_edge(a, "t", capacity=phi[a, 0] - m)
        for b in range(n):
            if b != a:
                G.add_edge(a, b, capacity=2.0 * Kd[a, b])
    cut, _ = nx.minimum_cut(G, "s", "t")
    np.testing.assert_allclose(cut + const, brute, rtol=1e-9)
    np.testing.assert_allclose(_lp_optimum(Kd, phi), brute, rtol=1e-7)


def test_projected_subgradient_approaches_lp_optimum():
    Kd, phi = _two_label_instance(8, 8)
    c = Kd.sum(axis=1)
    opt = _lp_optimum(Kd, phi)
    y0 = np.full((8, 2), 0.5)
    y, e = lp.lp_solve(phi, y0, c, lp.brute_partitioned(Kd), steps=2000, beta0=0.3)
    assert e.min() <= opt + 1e-3 * abs(opt)
    assert e.min() >= opt - 1e-9


def test_simplex_projection():
    rng = np.random.default_rng(9)
    V = rng.normal(scale=2.0, size=(50, 5))
    Y = lp.project_simplex(V)
    assert Y.min() >= 0
    np.testing.assert_allclose(Y.sum(1), 1.0, atol=1e-12)
    # KKT: y = max(v - tau, 0) with one tau per row
    for v, y in zip(V, Y):
        pos = y > 0
        tau = (v[pos] - y[pos]).mean()
        np.testing.assert_allclose(v[pos] - y[pos], tau, atol=1e-12)
        assert np.all(v[~pos] <= tau + 1e-12)
    # against a generic constrained solver
    for v in V[:5]:
        r = minimize(lambda z: np.sum((z - v) ** 2), np.full(5, 0.2), method="SLSQP", bounds=[(0, None)] * 5,
                     constraints=[{"type": "eq", "fun": lambda z: z.sum() - 1}], options={"ftol": 1e-14})
        np.testing.assert_allclose(lp.project_simplex(v[None])[0], r.x, atol=1e-6)
    # points of the simplex are fixed, uniform shifts do not matter
    z = rng.dirichlet(np.ones(5), size=4)
    np.testing.assert_allclose(lp.project_simplex(z), z, atol=1e-12)
    np.testing.assert_allclose(lp.project_simplex(z + 3.0), z, atol=1e-12)


def test_lattice_divide_and_conquer_top_level_is_full_filter():
    # with two points left and right of the top split only, the level-0 term is
    # the full lattice filter of the right half's indicator, read on the left half
    rng = np.random.default_rng(3)
    f = rng.normal(size=(8, 2)).astype(np.float32)
    lat = P.Permutohedral(f)
    rank = np.arange(8)
    seen = []
    def spy(v, part):
        seen.append((v.copy(), part.copy()))
        return lat.filter_partitioned(v, part)
    U = lp.upper_sums_dc(rank, spy)
    assert len(seen) == 3
    v0, p0 = seen[0]
    np.testing.assert_array_equal(v0, (rank >= 4).astype(float))
    np.testing.assert_array_equal(p0, 0)
    full = lat.filter((rank >= 4).astype(float))
    lvl1 = lat.filter_partitioned(seen[1][0], seen[1][1])
    lvl2 = lat.filter_partitioned(seen[2][0], seen[2][1])
    expect = np.where(rank < 4, full, 0) + np.where(seen[1][0] == 0, lvl1, 0) + np.where(seen[2][0] == 0, lvl2, 0)
    np.testing.assert_allclose(U, expect, rtol=1e-12)


# ---------------------------------------------------------------------------
# r-HST metrics (Appendix F)

def _tree(L=6):
    """A 2-level tree over 6 labels: root -> {0,1,2}, {3,4,5} -> leaves.

    Subtrees below the root with the length of the edge above them (edges halve
    downwards, an r-HST with r = 2): two groups (length 2) and six leaves (1).
    """
    members = np.zeros((8, L))
    members[0, :3] = 1
    members[1, 3:] = 1
    for i in range(6):
        members[2 + i, i] = 1
    c_t = np.array([2.0, 2.0] + [1.0] * 6)
    return members, c_t


def _tree_distance(i, j):
    # path length between leaves: 0, 2 (siblings: 1 + 1) or 6 (1 + 2 + 2 + 1)
    if i == j:
        return 0.0
    return 2.0 if (i < 3) == (j < 3) else 6.0


def test_potts_is_the_tree_of_single_labels():
    n, L = 20, 4
    k, phi, rng = _problem(11, n, L)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    y = rng.dirichlet(np.ones(L), size=n)
    c = Kd.sum(axis=1)
    G_tree = lp.subgradient_tree_dc(phi, y, c, lp.brute_partitioned(Kd), np.eye(L), np.ones(L))
    np.testing.assert_allclose(G_tree, lp.subgradient_dc(phi, y, c, lp.brute_partitioned(Kd)), rtol=1e-13,
                               atol=1e-13)


@pytest.mark.parametrize("n", [2, 9, 30])
def test_tree_divide_and_conquer_equals_pairs(n):
    members, c_t = _tree()
    k, phi, rng = _problem(12 + n, n, 6)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    y = rng.dirichlet(np.ones(6), size=n)
    y[: n // 2] = y[0]                                   # ties in every subtree column
    G_dc = lp.subgradient_tree_dc(phi, y, Kd.sum(axis=1), lp.brute_partitioned(Kd), members, c_t)
    np.testing.assert_allclose(G_dc, lp.subgradient_tree_pairs(phi, Kd, y, members, c_t), rtol=1e-12,
                               atol=1e-12)


def test_tree_lp_objective_euler_identity_subgradient_and_integer_points():
    members, c_t = _tree()
    n = 16
    k, phi, rng = _problem(13, n, 6)
    Kd = k.dense()
    np.fill_diagonal(Kd, 0.0)
    c = Kd.sum(axis=1)
    y = rng.dirichlet(np.ones(6), size=n)
    G = lp.subgradient_tree_dc(phi, y, c, lp.brute_partitioned(Kd), members, c_t)
    S = lp.s_lp_tree_pairs(phi, Kd, y, members, c_t)
    np.testing.assert_allclose(lp.s_lp_from_g(y, G), S, rtol=1e-12)
    for _ in range(10):                                  # convexity: G is a subgradient
        z = rng.dirichlet(np.ones(6), size=n)
        assert lp.s_lp_tree_pairs(phi, Kd, z, members, c_t) >= S + np.sum(G * (z - y)) - 1e-10
    # at a labelling the LP is the tree-metric energy sum_a phi + sum_{a != b} K_ab d(x_a, x_b) / 2
    x = rng.integers(0, 6, n)
    Y = np.eye(6)[x]
    E = np.sum(phi[np.arange(n), x]) + sum(Kd[a, b] * _tree_distance(x[a], x[b]) / 2.0
                                           for a in range(n) for b in range(n) if a != b)
    np.testing.assert_allclose(lp.s_lp_tree_pairs(phi, Kd, Y, members, c_t), E, rtol=1e-12)


@pytest.mark.parametrize("L", [2, 5, 21, 64])
def test_synthetic_hst_tree_is_a_tree(L):
    # the benchmark's tree: subtrees nest or are disjoint, every label is a
    # leaf, and the path length between labels (the sum of c_T over the
    # subtrees holding exactly one of them) is a metric; at L = 21 it is 2
    # between siblings of a group, 6 across groups of a half and 14 across
    # halves (edges of length 1, 2 and 4)
    from paper_1608_06192_gb300 import synthetic as S
    members, c_t = S.hst_tree(L)
    sets = [frozenset(np.nonzero(m)[0]) for m in members]
    for a in sets:
        for b in sets:
            assert a <= b or b <= a or not (a & b)
    assert all(frozenset([i]) in sets for i in range(L))
    D = np.array([[sum(c for t, c in zip(sets, c_t) if (i in t) != (j in t)) for j in range(L)] for i in range(L)])
    assert np.all(D == D.T) and np.all(np.diag(D) == 0) and np.all(D + np.eye(L) > 0)
    for i in range(L):
        for j in range(L):
            for k in range(L):
                assert D[i, k] <= D[i, j] + D[j, k]
    if L == 21:
        assert D[0, 1] == 2 and D[0, 4] == 6 and D[0, 20] == 14 and D[10, 13] == 2 and D[10, 14] == 6
