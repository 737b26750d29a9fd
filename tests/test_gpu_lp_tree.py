"""GPU parity of the tree-metric (r-HST) LP of Appendix F: the subgradient on
every subtree column by the divide and conquer of Appendix E, its objective,
the projected subgradient solve, and the Potts model as the tree of single
labels."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf, rel_err
from oracle import lp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def two_level_tree(groups, top=2.0, leaf=1.0):
    """Root -> the given label groups -> single labels; edge lengths halve downwards."""
    L = sum(len(g) for g in groups)
    rows, c_t = [], []
    for g in groups:
        if len(g) > 1:                       # a group of one label is its own leaf
            m = np.zeros(L)
            m[list(g)] = 1
            rows.append(m)
            c_t.append(top)
    for i in range(L):
        m = np.zeros(L)
        m[i] = 1
        rows.append(m)
        c_t.append(leaf)
    return np.array(rows), np.array(c_t)


def _case(dcrf, probs, ys, members, c_t, tol=1e-4):
    g = gpu_setup(dcrf, probs, torch)
    Y = torch.from_numpy(np.concatenate(ys)).cuda()
    G, e = dcrf.dcrf_lp_subgrad_tree(g["phi"], Y, [g["lb"], g["ls"]], probs[0].weights, members, c_t)
    G = G.cpu().numpy()
    for b, (p, y) in enumerate(zip(probs, ys)):
        s, t = g["off"][b], g["off"][b + 1]
        c = oracle_crf(p)
        Go = lp.subgradient_tree_dc(c.phi, y.astype(np.float64), c.c, c.kernel.apply_partitioned, members, c_t)
        assert rel_err(G[s:t], Go) <= tol
        eo = lp.s_lp_from_g(y.astype(np.float64), Go)
        assert abs(e[b] - eo) <= 1e-4 * max(1.0, np.abs(Go).max() * y.shape[0])
    return g, G, e


def test_tree_subgrad_two_levels_six_labels(dcrf):
    members, c_t = two_level_tree([[0, 1, 2], [3, 4, 5]])
    p = S.make_problem(32, 24, 6, 6, seed=80)
    _case(dcrf, [p], [S.dirichlet_labels(p.n_pixels, 6, seed=81)], members, c_t)


def test_tree_subgrad_three_levels_21_labels_ragged(dcrf):
    members, c_t = S.hst_tree(21)
    p = S.make_problem(53, 29, 8, 21, seed=82)
    y = S.dirichlet_labels(p.n_pixels, 21, seed=83)
    y[::4] = 1.0 / 21                 # exact ties in every subtree column
    _case(dcrf, [p], [y], members, c_t)


def test_tree_subgrad_batch_with_tiny_images(dcrf):
    members, c_t = two_level_tree([[0, 1], [2], [3, 4]], top=3.0, leaf=0.5)
    sizes = [(20, 13), (1, 1), (2, 1), (31, 9)]
    probs = [S.make_problem(w, h, 5, 5, seed=84 + i) for i, (w, h) in enumerate(sizes)]
    ys = [S.dirichlet_labels(q.n_pixels, 5, seed=90 + i) for i, q in enumerate(probs)]
    _case(dcrf, probs, ys, members, c_t)


def test_tree_subgrad_64_labels(dcrf):
    # the top label bit of the 64-bit subtree masks
    members, c_t = S.hst_tree(64)
    p = S.make_problem(24, 18, 4, 64, seed=95)
    _case(dcrf, [p], [S.dirichlet_labels(p.n_pixels, 64, seed=96)], members, c_t)


def test_potts_tree_equals_the_potts_subgradient(dcrf):
    # the tree of single labels with unit edges is the Potts model: the same
    # sorts and sums, only phi + (2U - c) against (phi + 2U) - c in rounding
    L = 21
    p = S.make_problem(48, 36, 6, L, seed=97)
    g = gpu_setup(dcrf, [p], torch)
    Y = torch.from_numpy(S.dirichlet_labels(p.n_pixels, L, seed=98)).cuda()
    lats = [g["lb"], g["ls"]]
    G1, e1 = dcrf.dcrf_lp_subgrad(g["phi"], Y, lats, p.weights)
    G2, e2 = dcrf.dcrf_lp_subgrad_tree(g["phi"], Y, lats, p.weights, np.eye(L), np.ones(L))
    G1, G2 = G1.cpu().numpy(), G2.cpu().numpy()
    assert np.abs(G1 - G2).max() <= 1e-6 * np.abs(G1).max()
    np.testing.assert_allclose(e1, e2, rtol=1e-6)


def test_tree_subgrad_at_a_labelling(dcrf):
    # integer y: every subtree column holds only 0 and 1, the case of most ties
    members, c_t = two_level_tree([[0, 1, 2], [3, 4, 5]])
    p = S.make_problem(30, 20, 5, 6, seed=99)
    lab = np.random.default_rng(100).integers(0, 6, size=p.n_pixels)
    y = np.eye(6, dtype=np.float32)[lab]
    _case(dcrf, [p], [y], members, c_t)


def test_tree_solve_small(dcrf):
    members, c_t = two_level_tree([[0, 1, 2], [3, 4, 5]])
    p = S.make_problem(32, 24, 6, 6, seed=101)
    g = gpu_setup(dcrf, [p], torch)
    y0 = S.dirichlet_labels(p.n_pixels, 6, seed=102)
    Y = torch.from_numpy(y0).cuda()
    e = dcrf.dcrf_lp_solve_tree(g["phi"], [g["lb"], g["ls"]], p.weights, Y, members, c_t, 30)[:, 0]
    c = oracle_crf(p)
    _, eo = lp.lp_solve(c.phi, y0.astype(np.float64), c.c, c.kernel.apply_partitioned, 30, members=members,
                        c_t=c_t)
    scale = np.abs(eo).max()
    assert abs(e[0] - eo[0]) <= 1e-4 * scale
    assert abs(e.min() - eo.min()) <= 1e-3 * scale
    Yg = Y.cpu().numpy()
    np.testing.assert_allclose(Yg.sum(1), 1.0, atol=1e-5)
    Gb = lp.subgradient_tree_dc(c.phi, Yg.astype(np.float64), c.c, c.kernel.apply_partitioned, members, c_t)
    assert abs(lp.s_lp_from_g(Yg.astype(np.float64), Gb) - e.min()) <= 1e-3 * scale


@pytest.mark.parametrize("bad", ["empty", "out_of_range", "negative", "nan"])
def test_tree_invalid_subtrees_are_rejected(dcrf, bad):
    # a five-label tree; each case spoils one subtree and the call reports
    # DCRF_E_INVAL through the C ABI (masks passed as raw bits, no wrapper check)
    import ctypes
    members, c_t = two_level_tree([[0, 1, 2], [3, 4]])
    p = S.make_problem(8, 6, 3, 5, seed=103)
    g = gpu_setup(dcrf, [p], torch)
    Y = torch.from_numpy(S.dirichlet_labels(p.n_pixels, 5, seed=104)).cuda()
    masks, w = dcrf._tree(members, c_t, 5)
    if bad == "empty":
        masks[3] = 0
    elif bad == "out_of_range":
        masks[3] |= np.uint64(1) << np.uint64(5)      # label 5 of a 5-label problem
    elif bad == "negative":
        w[0] = -1.0
    else:
        w[1] = np.nan
    G = torch.empty_like(Y)
    st = dcrf.lib().dcrf_lp_subgrad_tree(dcrf._ptr(g["phi"]), dcrf._ptr(Y), dcrf._handles([g["lb"], g["ls"]]),
                                         dcrf._floats(p.weights), 2, 5, len(masks),
                                         masks.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                                         dcrf._ptr(G), None, dcrf._stream(None))
    assert st == -1                                   # DCRF_E_INVAL
    torch.cuda.synchronize()
    # the valid tree still runs afterwards
    dcrf.dcrf_lp_subgrad_tree(g["phi"], Y, [g["lb"], g["ls"]], p.weights, members, c_t)
