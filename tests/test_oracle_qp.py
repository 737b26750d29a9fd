"""Pins of the oracle's Frank-Wolfe and CCCP (Algorithm 1-2, Appendix B)."""
import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import crf, qp
from oracle import permutohedral as P
from paper_1608_06192_gb300 import synthetic as S


def _brute_problem(seed=0, n=16, L=3, w=(3.0, 1.0)):
    rng = np.random.default_rng(seed)
    f1 = rng.normal(scale=1.5, size=(n, 2))
    f2 = rng.normal(scale=1.5, size=(n, 3))
    k = crf.BruteGaussian([f1, f2], list(w))
    phi = rng.normal(scale=2.0, size=(n, L))
    y0 = rng.dirichlet(np.ones(L), size=n)
    return crf.DenseCRF(phi, k), y0


def test_step_size_is_exact_line_minimiser():
    c, y0 = _brute_problem(1)
    lin = c.phi - c.d
    P_y = c.psi_plus_D(y0)
    g = lin + 2 * P_y
    s = np.zeros_like(y0)
    s[np.arange(len(y0)), np.argmin(g, 1)] = 1
    _, _, rec = qp.frank_wolfe(c, y0, 1)
    alpha = rec[0, 2]
    grid = np.linspace(0, 1, 20001)
    vals = [c.s_cvx(y0 + a * (s - y0)) for a in grid]
    assert abs(grid[int(np.argmin(vals))] - alpha) < 1e-4
    # A and B are the quadratic and linear coefficients of S_cvx along s - y
    for a in (0.3, 0.9):
        pred = c.s_cvx(y0) + rec[0, 4] * a + rec[0, 3] * a * a
        np.testing.assert_allclose(c.s_cvx(y0 + a * (s - y0)), pred, rtol=1e-11)


def test_step_size_cases():
    assert qp.step_size(2.0, -1.0) == 0.25
    assert qp.step_size(1.0, -5.0) == 1.0
    assert qp.step_size(1.0, 3.0) == 0.0
    assert qp.step_size(0.0, -1.0) == 1.0
    assert qp.step_size(-1.0, 0.5) == 1.0 if -1.0 + 0.5 < 0 else 0.0
    assert qp.step_size(0.0, 0.0) == 0.0


def test_gap_nonnegative_energy_monotone_and_reuse_exact():
    c, y0 = _brute_problem(2)
    y, P_y, rec = qp.frank_wolfe(c, y0, 60)
    assert np.all(rec[:, 1] >= -1e-10)
    assert np.all(np.diff(rec[:, 0]) <= 1e-10)
    np.testing.assert_allclose(P_y, c.psi_plus_D(y), rtol=1e-9, atol=1e-9)
    # the conditional gradient is a vertex minimising <s, g> over M (Eq. 14):
    # no feasible point has a lower linear value
    g = c.phi - c.d + 2 * P_y
    s_val = g.min(axis=1).sum()
    rng = np.random.default_rng(0)
    for _ in range(20):
        z = rng.dirichlet(np.ones(c.L), size=c.n)
        assert np.sum(g * z) >= s_val - 1e-12


def test_frank_wolfe_reaches_convex_optimum():
    c, y0 = _brute_problem(3, n=10, L=3)
    y, _, rec = qp.frank_wolfe(c, y0, 3000)
    n, L = c.n, c.L
    cons = [{"type": "eq", "fun": (lambda v, a=a: v.reshape(n, L)[a].sum() - 1.0)} for a in range(n)]
    res = minimize(lambda v: c.s_cvx(v.reshape(n, L)), y0.reshape(-1), method="SLSQP",
                   bounds=[(0, 1)] * (n * L), constraints=cons, options={"maxiter": 500, "ftol": 1e-12})
    assert res.success
    best = res.fun
    # the Frank-Wolfe gap bounds the suboptimality: S(y^t) - gap_t <= S* <= S(y^t)
    tol = 1e-7 * abs(best)
    assert np.all(rec[:, 0] - rec[:, 1] <= best + tol)
    assert best <= c.s_cvx(y) + tol
    assert c.s_cvx(y) - best <= 2e-3 * abs(best)


def test_fw_on_lattice_operator_is_monotone():
    p = S.qp_small()
    fb, fs = crf.features(p.rgb, *p.thetas)
    k = P.LatticeGaussian([crf.to_fp32_features(fb), crf.to_fp32_features(fs)], p.weights)
    c = crf.DenseCRF(p.unaries, k)
    _, _, rec = qp.frank_wolfe(c, p.y0, 20)
    assert np.all(np.diff(rec[:, 0]) <= 1e-9 * np.abs(rec[:-1, 0]).max())
    assert np.all(rec[:, 1] >= -1e-9 * np.abs(rec[:, 0]).max())


@pytest.mark.parametrize("kind", ["brute", "lattice"])
def test_cccp_monotone(kind):
    if kind == "brute":
        c, y0 = _brute_problem(4, n=20, L=4)
    else:
        p = S.qp_small()
        fb, fs = crf.features(p.rgb, *p.thetas)
        k = P.LatticeGaussian([crf.to_fp32_features(fb), crf.to_fp32_features(fs)], p.weights)
        c, y0 = crf.DenseCRF(p.unaries, k), p.y0
    y, e = qp.cccp_dc_gen(c, y0, outer=6, inner=15)
    assert np.all(np.diff(e) <= 1e-9 * np.abs(e).max())
    np.testing.assert_allclose(e[-1], c.s_qp(y), rtol=1e-9)


def test_replayed_decisions_follow_the_definitions():
    # Replaying decisions (another run's s^t) must reproduce the free run when
    # they are the run's own argmins, and otherwise follow Algorithm 1 and
    # Appendix B along the given vertices: energy S_cvx(y^t) (Eq. 10), gap
    # <g, y^t - s^t>, A and B the coefficients of S_cvx(y^t + a (s^t - y^t)),
    # y^{t+1} = y^t + alpha (s^t - y^t).
    c, y0 = _brute_problem(5, n=18, L=4)
    own = []
    y1, _, rec1 = qp.frank_wolfe(c, y0, 7, on_step=lambda t, g, s: own.append(np.array(s)))
    y2, _, rec2 = qp.frank_wolfe(c, y0, 7, decisions=own)
    np.testing.assert_array_equal(y1, y2)
    np.testing.assert_array_equal(rec1, rec2)
    assert all(np.array_equal(s, np.argmin(c.phi - c.d + 2 * c.psi_plus_D(y), 1)) for s, y in
               zip(own[:1], [y0]))
    rng = np.random.default_rng(3)
    dec = rng.integers(0, c.L, size=(7, c.n))
    grads = []
    y3, _, rec3 = qp.frank_wolfe(c, y0, 7, decisions=dec, on_step=lambda t, g, s: grads.append(g.copy()))
    y = np.array(y0, dtype=np.float64)
    rows = np.arange(c.n)
    for t in range(7):
        s = np.zeros_like(y)
        s[rows, dec[t]] = 1.0
        np.testing.assert_allclose(rec3[t, 0], c.s_cvx(y), rtol=1e-12)
        g = c.phi - c.d + 2 * c.psi_plus_D(y)
        np.testing.assert_allclose(grads[t], g, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(rec3[t, 1], np.sum(g * (y - s)), rtol=1e-10, atol=1e-10)
        for a in (0.25, 0.8):
            pred = c.s_cvx(y) + rec3[t, 4] * a + rec3[t, 3] * a * a
            np.testing.assert_allclose(c.s_cvx(y + a * (s - y)), pred, rtol=1e-11)
        assert rec3[t, 2] == qp.step_size(rec3[t, 3], rec3[t, 4])
        y = y + rec3[t, 2] * (s - y)
    np.testing.assert_allclose(y3, y, rtol=1e-12, atol=1e-14)


def test_cccp_replayed_decisions_reproduce_the_run():
    # CCCP (Algorithm 2) with every inner Frank-Wolfe run replaying given
    # vertices: its own decisions give back the free run exactly
    c, y0 = _brute_problem(6, n=20, L=4)
    own = []
    y1, e1 = qp.cccp_dc_gen(c, y0, 3, 5, on_step=lambda t, g, s: own.append(np.array(s)))
    assert len(own) == 15
    y2, e2 = qp.cccp_dc_gen(c, y0, 3, 5, decisions=own)
    np.testing.assert_array_equal(y1, y2)
    np.testing.assert_array_equal(e1, e2)
