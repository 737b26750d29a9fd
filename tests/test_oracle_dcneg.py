"""Pins of the oracle's CCCP for negative semi-definite compatibilities (Section 5.2, Appendix C)."""
import numpy as np
from scipy.optimize import minimize

from oracle import crf, qp
from oracle.lp import project_simplex


def _slsqp_simplex(f, L, x0=None):
    x0 = np.full(L, 1.0 / L) if x0 is None else x0
    r = minimize(f, x0, method="SLSQP", bounds=[(0, None)] * L,
                 constraints=[{"type": "eq", "fun": lambda z: z.sum() - 1}], options={"ftol": 1e-15, "maxiter": 500})
    return r.x


def _tangent_nsd_mu(L, seed):
    # mu = 1 1^T - G with G positive definite: z^T mu z = -z^T G z < 0 for sum z = 0
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(L, L))
    return np.ones((L, L)) - (R @ R.T / L + np.eye(L))


def _problem(seed, n=14, L=4, mu=None, weights=(1.5, 0.7)):
    rng = np.random.default_rng(seed)
    k = crf.BruteGaussian([rng.normal(scale=1.2, size=(n, 3)), rng.normal(size=(n, 2))], list(weights))
    return crf.DenseCRF(rng.normal(scale=2.0, size=(n, L)), k, mu, clamp=False), rng


def test_potts_pixel_problem_is_a_projection():
    # min lin^T y - sum_w y^T mu y on the simplex, mu Potts: Proj(-lin / (2 sum_w))
    rng = np.random.default_rng(0)
    L, sw = 5, 1.7
    mu = 1.0 - np.eye(L)
    for _ in range(6):
        lin = rng.normal(scale=3.0, size=L)
        y = project_simplex((-lin / (2 * sw))[None])[0]
        ref = _slsqp_simplex(lambda z: lin @ z - sw * z @ mu @ z, L)
        np.testing.assert_allclose(y, ref, atol=1e-6)


def test_pixel_frank_wolfe_reaches_the_pixel_minimiser():
    # the general-mu path (per-pixel Frank-Wolfe, exact step) converges to the
    # minimiser: the projection for Potts, SLSQP for another tangent-NSD mu
    rng = np.random.default_rng(1)
    L, sw = 4, 1.3
    lin = rng.normal(scale=2.0, size=(6, L))
    y0 = np.full((6, L), 1.0 / L)
    potts = 1.0 - np.eye(L)
    y_fw = qp.dc_neg_pixel_fw(lin, y0, potts, sw, 3000)
    np.testing.assert_allclose(y_fw, project_simplex(-lin / (2 * sw)), atol=2e-3)
    mu = _tangent_nsd_mu(L, 2)
    y_fw = qp.dc_neg_pixel_fw(lin, y0, mu, sw, 3000)
    for a in range(6):
        f = lambda z: lin[a] @ z - sw * z @ mu @ z
        ref = _slsqp_simplex(f, L)
        # Frank-Wolfe converges as O(1/t) when the minimiser lies on a face
        assert f(ref) - 1e-9 <= f(y_fw[a]) <= f(ref) + 1e-3


def test_energy_record_is_s_qp():
    c, rng = _problem(3)
    y = rng.dirichlet(np.ones(c.L), size=c.n)
    _, e = qp.cccp_dc_neg(c, y, 0)
    np.testing.assert_allclose(e[0], c.s_qp(y), rtol=1e-12)


def test_linearisation_majorises_s_qp():
    # S_QP(y) <= convex(y) + concave(y^t) + <grad concave(y^t), y - y^t> on M,
    # with equality at y^t: the CCCP surrogate of Section 5.2
    for mu in (None, _tangent_nsd_mu(4, 5)):
        c, rng = _problem(4, mu=mu)
        sw = c.kernel.sum_w
        yt = rng.dirichlet(np.ones(c.L), size=c.n)
        Kd = c.kernel.dense()

        def convex(y):
            return np.sum(c.phi * y) - sw * np.sum(y * (y @ c.mu.T))

        def concave(y):
            return np.sum(y * (Kd @ y @ c.mu.T))

        grad = (Kd @ yt + Kd.T @ yt) @ c.mu.T
        for _ in range(10):
            y = rng.dirichlet(np.ones(c.L), size=c.n)
            surrogate = convex(y) + concave(yt) + np.sum(grad * (y - yt))
            assert c.s_qp(y) <= surrogate + 1e-9
        np.testing.assert_allclose(convex(yt) + concave(yt), c.s_qp(yt), rtol=1e-12)


def test_cccp_decreases_s_qp_monotonically():
    for mu, inner in ((None, 0), (_tangent_nsd_mu(4, 7), 50)):
        c, rng = _problem(6, n=20, mu=mu, weights=(0.4, 0.2))
        y0 = rng.dirichlet(np.ones(c.L), size=c.n)
        y, e = qp.cccp_dc_neg(c, y0, 6, inner)
        assert np.all(np.diff(e) <= 1e-9 * np.abs(e).max())
        assert e[-1] < e[0]
        np.testing.assert_allclose(y.sum(1), 1.0, atol=1e-12)
        assert y.min() >= -1e-12


def test_concave_part_is_concave_on_the_simplex_directions():
    # (mu (x) K) restricted to zero-sum rows is negative semi-definite
    c, rng = _problem(8, n=9, L=3)
    Kd = c.kernel.dense()
    for _ in range(20):
        D = rng.normal(size=(c.n, c.L))
        D -= D.mean(axis=1, keepdims=True)
        assert np.sum(D * (Kd @ D @ c.mu.T)) <= 1e-10
