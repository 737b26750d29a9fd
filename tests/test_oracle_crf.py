"""Pins of the oracle's exact CRF definitions (Eq. 1, 3-4, 6-8, 10-11)."""
import json
import os

import numpy as np

from oracle import crf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_kernel_three_points_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "kernel_three_points.json")))
    k = crf.BruteGaussian([np.array(g["features"])], [1.0])
    np.testing.assert_allclose(k.dense(), np.array(g["K"]), rtol=1e-14)
    np.testing.assert_allclose(k.apply(np.array(g["v"])[:, None])[:, 0], g["Kv"], rtol=1e-13)


def test_features_of_appendix_g():
    rgb = np.array([[[10.0, 20.0, 30.0], [40.0, 50.0, 60.0]]], dtype=np.float32)   # H=1, W=2
    fb, fs = crf.features(rgb, 80.0, 13.0, 3.0)
    np.testing.assert_allclose(fb[1], [1 / 80, 0, 40 / 13, 50 / 13, 60 / 13], rtol=1e-15)
    np.testing.assert_allclose(fs[1], [1 / 3, 0], rtol=1e-15)
    # the kernel exp(-|p|^2/(2 theta^2) - |I|^2/(2 theta_b^2)) of Appendix G with sigma = 2 theta^2
    kb = crf.BruteGaussian([fb], [1.0]).dense()[0, 1]
    expect = np.exp(-1.0 / (2 * 80.0 ** 2) - 3 * 30.0 ** 2 / (2 * 13.0 ** 2))
    np.testing.assert_allclose(kb, expect, rtol=1e-13)
    np.testing.assert_array_equal(crf.to_fp32_features(fb), (fb.astype(np.float32)))


def _small(seed=0, n=12, L=3):
    rng = np.random.default_rng(seed)
    f1 = rng.normal(size=(n, 2))
    f2 = rng.normal(size=(n, 3))
    k = crf.BruteGaussian([f1, f2], [2.0, 0.5])
    phi = rng.normal(size=(n, L))
    return k, phi, rng


def test_psi_matches_kronecker_product():
    k, phi, rng = _small()
    n, L = phi.shape
    mu = rng.uniform(0, 1, (L, L))
    c = crf.DenseCRF(phi, k, mu)
    Kd = k.dense()
    psi = np.kron(mu, Kd - k.sum_w * np.eye(n))        # label-major vector y[(i, a)]
    y = rng.uniform(size=(n, L))
    lhs = c.psi(y)
    rhs = (psi @ y.T.reshape(-1)).reshape(L, n).T
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_d_is_row_sum_of_absolute_pairwise():
    k, phi, rng = _small(1)
    n, L = phi.shape
    mu = rng.normal(size=(L, L))
    c = crf.DenseCRF(phi, k, mu)
    Kd = k.dense()
    d = np.zeros((n, L))
    for a in range(n):
        for i in range(L):
            d[a, i] = sum(abs(mu[i, j] * Kd[a, b]) for b in range(n) if b != a for j in range(L))
    np.testing.assert_allclose(c.d, d, rtol=1e-12)


def test_energies_agree_at_integer_points():
    k, phi, rng = _small(2, n=10, L=4)
    c = crf.DenseCRF(phi, k)
    for _ in range(5):
        x = rng.integers(0, 4, 10)
        e_pairs = crf.energy_pairs(phi, k.dense(), c.mu, x)
        y = np.zeros((10, 4))
        y[np.arange(10), x] = 1.0
        np.testing.assert_allclose(c.energy(x), e_pairs, rtol=1e-12)
        np.testing.assert_allclose(c.s_qp(y), e_pairs, rtol=1e-12)
        # y^T D y = d^T y at binary y, so the convexified objective is tight there
        np.testing.assert_allclose(c.s_cvx(y), e_pairs, rtol=1e-12)
        np.testing.assert_allclose(crf.s_lp_pairs(phi, k.dense(), y), e_pairs, rtol=1e-12)


def test_convexified_objective_is_convex_and_lower_bounds_qp():
    # Psi + D is diagonally dominant, hence PSD; and S_cvx <= S_QP on M since
    # S_cvx - S_QP = sum d (y^2 - y) <= 0 for y in [0, 1]
    k, phi, rng = _small(3, n=8, L=3)
    mu = rng.normal(size=(3, 3))
    c = crf.DenseCRF(phi, k, (mu + mu.T) / 2)
    n, L = phi.shape
    M = np.zeros((n * L, n * L))
    for j in range(n * L):
        e = np.zeros(n * L)
        e[j] = 1
        M[:, j] = c.psi_plus_D(e.reshape(n, L)).reshape(-1)
    assert np.linalg.eigvalsh((M + M.T) / 2).min() > -1e-10
    for _ in range(5):
        y = rng.dirichlet(np.ones(L), size=n)
        assert c.s_cvx(y) <= c.s_qp(y) + 1e-12
