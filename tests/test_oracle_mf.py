"""Pins of the oracle's mean-field baseline and rounding (Section 1, Section 6.2)."""
import numpy as np
from scipy.optimize import minimize

from oracle import crf, mf


def _problem(seed, n=6, L=3, weights=(0.3, 0.2)):
    rng = np.random.default_rng(seed)
    k = crf.BruteGaussian([rng.normal(scale=1.0, size=(n, 3)), rng.normal(size=(n, 2))], list(weights))
    return crf.DenseCRF(rng.normal(scale=1.0, size=(n, L)), k, clamp=False), rng


def test_without_pairwise_terms_one_update_is_the_unary_softmax():
    c, rng = _problem(0, weights=(0.0, 0.0))
    q0 = rng.dirichlet(np.ones(c.L), size=c.n)
    Q, _ = mf.mean_field(c, q0, 1)
    E = np.exp(-c.phi)
    np.testing.assert_allclose(Q, E / E.sum(1, keepdims=True), rtol=1e-14)


def test_fixed_point_is_a_stationary_point_of_the_mean_field_free_energy():
    # F(Q) = sum Q log Q + E_Q[E] = sum Q log Q + phi^T Q + Q^T Psi Q (Eq. 1
    # sums ordered pairs): a fixed point of the parallel update minimises F
    # here (weak coupling, so the iteration converges), checked against a
    # generic solver
    c, rng = _problem(1)
    Q, _ = mf.mean_field(c, mf.softmax_rows(-c.phi), 400)
    n, L = c.phi.shape

    def free(z):
        q = np.clip(z.reshape(n, L), 1e-300, None)
        return float(np.sum(q * np.log(q)) + np.sum(c.phi * q) + np.sum(q * c.psi(q)))

    cons = [{"type": "eq", "fun": (lambda z, a=a: z.reshape(n, L)[a].sum() - 1)} for a in range(n)]
    r = minimize(free, np.full(n * L, 1.0 / L), method="SLSQP", bounds=[(1e-12, 1)] * (n * L), constraints=cons,
                 options={"ftol": 1e-15, "maxiter": 1000})
    np.testing.assert_allclose(Q, r.x.reshape(n, L), atol=2e-5)
    # and it is a fixed point of the update
    np.testing.assert_allclose(mf.softmax_rows(-c.phi - 2.0 * c.psi(Q)), Q, atol=1e-12)


def test_energy_record_is_s_qp_of_the_marginals():
    c, rng = _problem(2)
    q0 = rng.dirichlet(np.ones(c.L), size=c.n)
    Q, e = mf.mean_field(c, q0, 3)
    np.testing.assert_allclose(e[0], c.s_qp(q0), rtol=1e-12)
    np.testing.assert_allclose(e[-1], c.s_qp(Q), rtol=1e-12)


def test_rounding_takes_the_lowest_label_on_ties_and_energy_is_eq1():
    y = np.array([[0.2, 0.5, 0.3], [0.4, 0.4, 0.2], [1 / 3, 1 / 3, 1 / 3]])
    np.testing.assert_array_equal(mf.round_labels(y), [1, 0, 0])
    c, rng = _problem(3, n=7)
    x = rng.integers(0, c.L, c.n)
    np.testing.assert_allclose(c.energy(x), crf.energy_pairs(c.phi, c.kernel.dense(), c.mu, x), rtol=1e-12)
