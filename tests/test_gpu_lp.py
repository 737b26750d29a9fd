"""GPU parity of the LP subgradient (Eq. 20, Appendix E), projection and Algorithm 3."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf, rel_err
from oracle import lp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle_subgrad(p, y):
    c = oracle_crf(p)
    return lp.subgradient_dc(c.phi, y.astype(np.float64), c.c, c.kernel.apply_partitioned)


def _case(dcrf, probs, ys, tol=1e-4):
    g = gpu_setup(dcrf, probs, torch)
    Y = torch.from_numpy(np.concatenate(ys)).cuda()
    G, e = dcrf.dcrf_lp_subgrad(g["phi"], Y, [g["lb"], g["ls"]], probs[0].weights)
    G = G.cpu().numpy()
    for b, (p, y) in enumerate(zip(probs, ys)):
        s, t = g["off"][b], g["off"][b + 1]
        Go = _oracle_subgrad(p, y)
        assert rel_err(G[s:t], Go) <= tol
        eo = lp.s_lp_from_g(y.astype(np.float64), Go)
        assert abs(e[b] - eo) <= 1e-4 * max(1.0, np.abs(Go).max() * y.shape[0])


def test_lp_subgrad_tiny(dcrf):
    p = S.make_problem(32, 24, 6, 21, seed=2)
    _case(dcrf, [p], [S.dirichlet_labels(p.n_pixels, 21, seed=5)])


def test_lp_subgrad_ties_and_ragged(dcrf):
    p = S.make_problem(37, 23, 5, 4, seed=3)
    y = S.dirichlet_labels(p.n_pixels, 4, seed=6)
    y[::3] = 0.25                      # exact ties, broken by pixel index
    _case(dcrf, [p], [y])


def test_lp_subgrad_batch(dcrf):
    probs = [S.make_problem(w, h, 5, 5, seed=40 + i) for i, (w, h) in enumerate([(20, 13), (1, 1), (2, 1), (31, 9)])]
    ys = [S.dirichlet_labels(q.n_pixels, 5, seed=50 + i) for i, q in enumerate(probs)]
    _case(dcrf, probs, ys)


def test_lp_subgrad_medium(dcrf):
    p = S.make_problem(120, 90, 12, 21, seed=4)
    _case(dcrf, [p], [S.dirichlet_labels(p.n_pixels, 21, seed=7)])


def test_simplex_projection_device(dcrf):
    rng = np.random.default_rng(3)
    for L in (2, 5, 21, 64):
        V = rng.normal(scale=2.0, size=(1000, L)).astype(np.float32)
        Y = dcrf.dcrf_simplex_project(torch.from_numpy(V).cuda()).cpu().numpy()
        np.testing.assert_allclose(Y, lp.project_simplex(V), atol=2e-6)


def test_lp_solve_small(dcrf):
    p = S.make_problem(32, 24, 6, 5, seed=8)
    g = gpu_setup(dcrf, [p], torch)
    y0 = S.dirichlet_labels(p.n_pixels, 5, seed=9)
    Y = torch.from_numpy(y0).cuda()
    e = dcrf.dcrf_lp_solve(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 30)[:, 0]
    c = oracle_crf(p)
    yb, eo = lp.lp_solve(c.phi, y0.astype(np.float64), c.c, c.kernel.apply_partitioned, 30)
    scale = np.abs(eo).max()
    assert abs(e[0] - eo[0]) <= 1e-4 * scale
    assert abs(e.min() - eo.min()) <= 1e-3 * scale
    Yg = Y.cpu().numpy()
    np.testing.assert_allclose(Yg.sum(1), 1.0, atol=1e-5)
    Gb = _oracle_subgrad(p, Yg)
    assert abs(lp.s_lp_from_g(Yg.astype(np.float64), Gb) - e.min()) <= 1e-3 * scale


def test_lp_solve_headline_200_steps(dcrf):
    # 200 projected-subgradient steps at 500x375, L=21 (the oracle's 200 steps
    # at this size would take hours; the subgradient itself is checked at
    # this size above: the iterate stays on the simplex, every energy is
    # finite, the best energy does not exceed the start and the returned y
    # has that energy)
    p = S.voc_shaped()
    g = gpu_setup(dcrf, [p], torch)
    y0 = S.dirichlet_labels(p.n_pixels, 21, seed=11)
    Y = torch.from_numpy(y0).cuda()
    e = dcrf.dcrf_lp_solve(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 200)[:, 0]
    assert np.isfinite(e).all()
    assert e.min() <= e[0]
    Yg = Y.cpu().numpy()
    np.testing.assert_allclose(Yg.sum(1), 1.0, atol=1e-5)
    assert Yg.min() >= 0.0
    _, e_best = dcrf.dcrf_lp_subgrad(g["phi"], Y, [g["lb"], g["ls"]], p.weights)
    assert abs(e_best[0] - e.min()) <= 1e-3 * abs(e.min())


def test_lp_subgrad_full_size_two_columns(dcrf):
    # 500x375, L=21, y ~ Dirichlet(0.5): the sorted columns of labels 0 and 20
    # through all 18 levels of the divide and conquer, against the oracle
    p = S.voc_shaped()
    g = gpu_setup(dcrf, [p], torch)
    y = S.dirichlet_labels(p.n_pixels, 21, seed=5)
    G, _ = dcrf.dcrf_lp_subgrad(g["phi"], torch.from_numpy(y).cuda(), [g["lb"], g["ls"]], p.weights)
    G = G.cpu().numpy()
    c = oracle_crf(p)
    for i in (0, 20):
        U = lp.upper_sums_dc(lp.label_rank(y[:, i].astype(np.float64)), c.kernel.apply_partitioned)
        assert rel_err(G[:, i], c.phi[:, i] + 2.0 * U - c.c) <= 1e-4


@pytest.mark.parametrize("shape", [(120, 90, 21), (37, 23, 4)])
def test_lp_own_sort_matches_cub(dcrf, shape, monkeypatch):
    # the per-label sort and the grouping of incidences by vertex are the
    # library's own segmented radix sort; CUB's radix sort, switched on by
    # DCRF_LP_SORT=cub, is the comparator: both are stable with the same key
    # order, so the subgradients agree up to the order of the float atomics
    # that sum the lattice values
    W, H, L = shape
    probs = [S.make_problem(W, H, 6, L, seed=20), S.make_problem(W // 2 + 1, H, 6, L, seed=21)]
    ys = [S.dirichlet_labels(q.n_pixels, L, seed=22 + i) for i, q in enumerate(probs)]
    ys[0][::5] = 1.0 / L                              # exact ties, kept in pixel order
    g = gpu_setup(dcrf, probs, torch)
    Y = torch.from_numpy(np.concatenate(ys)).cuda()
    G1, e1 = dcrf.dcrf_lp_subgrad(g["phi"], Y, [g["lb"], g["ls"]], probs[0].weights)
    monkeypatch.setenv("DCRF_LP_SORT", "cub")
    G2, e2 = dcrf.dcrf_lp_subgrad(g["phi"], Y, [g["lb"], g["ls"]], probs[0].weights)
    assert rel_err(G1.cpu().numpy(), G2.cpu().numpy()) <= 1e-6
    np.testing.assert_allclose(e1, e2, rtol=1e-6)
    for b, (p, y) in enumerate(zip(probs, ys)):
        s, t = g["off"][b], g["off"][b + 1]
        assert rel_err(G1.cpu().numpy()[s:t], _oracle_subgrad(p, y)) <= 1e-4
