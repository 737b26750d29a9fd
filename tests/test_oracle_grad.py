"""Pins of the oracle's reverse mode through unrolled Frank-Wolfe: FP64 central differences."""
import numpy as np

from oracle import crf, qp
from oracle import permutohedral as P
from paper_1608_06192_gb300 import synthetic as S


def _crf(p, w=None, phi=None):
    fb, fs = crf.features(p.rgb, *p.thetas)
    lats = [P.Permutohedral(crf.to_fp32_features(fb)), P.Permutohedral(crf.to_fp32_features(fs))]
    ops = [(l.filter, l.filter_adjoint) for l in lats]
    return qp.WeightedCRF(p.unaries if phi is None else phi, ops, p.weights if w is None else w)


def _loss(p, ybar, iters, w=None, phi=None):
    c = _crf(p, w, phi)
    y, tape = qp.fw_tape(c, p.y0, iters)
    return float(np.sum(ybar * y)), tape


def test_weighted_crf_matches_dense_crf():
    p = S.crop(S.qp_small(), 16, 12)
    c = _crf(p)
    fb, fs = crf.features(p.rgb, *p.thetas)
    k = P.LatticeGaussian([crf.to_fp32_features(fb), crf.to_fp32_features(fs)], p.weights)
    d = crf.DenseCRF(p.unaries, k)
    v = np.random.default_rng(0).normal(size=(p.n_pixels, p.n_labels))
    np.testing.assert_allclose(c.op(v), d.psi_plus_D(v), rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(np.sum(v * c.op_T(v[::-1])), np.sum(c.op(v) * v[::-1]), rtol=1e-12)


def test_gradients_match_central_differences():
    base = S.make_problem(48, 40, 5, 4, seed=3)
    p = S.crop(base, 32, 24)
    iters = 10
    ybar = np.random.default_rng(1).normal(size=(p.n_pixels, p.n_labels))
    c = _crf(p)
    y, tape = qp.fw_tape(c, p.y0, iters)
    phibar, wbar, _ = qp.fw_backward(c, tape, ybar)
    h = 1e-4
    s_ref = [t[1] for t in tape]

    def same_path(tp):   # differences are valid only if no s^t flips and no alpha clips
        return all(np.array_equal(a[1], b) for a, b in zip(tp, s_ref)) and \
            all((0 < a[2] < 1) == (0 < b[2] < 1) for a, b in zip(tp, tape))

    # kernel weights
    for m in range(2):
        wp = np.array(p.weights, dtype=np.float64); wp[m] += h
        wm = np.array(p.weights, dtype=np.float64); wm[m] -= h
        fp, tp = _loss(p, ybar, iters, w=wp)
        fm, tm = _loss(p, ybar, iters, w=wm)
        assert same_path(tp) and same_path(tm)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - wbar[m]) <= 1e-4 * max(abs(fd), 1e-3), (m, fd, wbar[m])
    # unaries, sampled coordinates
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(12):
        a, i = int(rng.integers(p.n_pixels)), int(rng.integers(p.n_labels))
        php = p.unaries.astype(np.float64).copy(); php[a, i] += h
        phm = p.unaries.astype(np.float64).copy(); phm[a, i] -= h
        fp, tp = _loss(p, ybar, iters, phi=php)
        fm, tm = _loss(p, ybar, iters, phi=phm)
        if not (same_path(tp) and same_path(tm)):
            continue
        fd = (fp - fm) / (2 * h)
        assert abs(fd - phibar[a, i]) <= 1e-4 * max(abs(fd), 1e-6) + 1e-9, (a, i, fd, phibar[a, i])
        checked += 1
    assert checked >= 8


def test_gradients_along_given_decisions_match_central_differences_21_labels():
    # With 21 labels the FP64 path has argmin decisions within ~1e-7 of a tie,
    # so perturbing phi or w by h = 1e-4 changes s^t and plain differences
    # jump.  With the decisions held fixed (the smooth piece of the unrolled
    # map, the replay mode of the forward), central differences are the
    # derivative that the reverse mode computes.
    p = S.crop(S.make_problem(48, 40, 5, 21, seed=3), 32, 24)
    iters = 10
    ybar = np.random.default_rng(1).normal(size=(p.n_pixels, p.n_labels))
    c = _crf(p)
    y, tape = qp.fw_tape(c, p.y0, iters)
    dec = [np.argmax(t[1], axis=1) for t in tape]
    phibar, wbar, _ = qp.fw_backward(c, tape, ybar)
    # the replay of the run's own decisions is the run itself
    y_r, tape_r = qp.fw_tape(c, p.y0, iters, decisions=dec)
    np.testing.assert_array_equal(y, y_r)
    h = 1e-4

    def loss(w=None, phi=None):
        yy, tp = qp.fw_tape(_crf(p, w, phi), p.y0, iters, decisions=dec)
        assert all((0 < a[2] < 1) == (0 < b[2] < 1) for a, b in zip(tp, tape))
        return float(np.sum(ybar * yy))

    def central(**kw):
        """(difference quotient, its FP64 rounding floor 8 eps |f| / 2h)."""
        fp, fm = loss(**{k: v[0] for k, v in kw.items()}), loss(**{k: v[1] for k, v in kw.items()})
        return (fp - fm) / (2 * h), 8 * np.finfo(float).eps * max(abs(fp), abs(fm)) / (2 * h)

    for m in range(2):
        wp = np.array(p.weights, dtype=np.float64); wp[m] += h
        wm = np.array(p.weights, dtype=np.float64); wm[m] -= h
        fd, floor = central(w=(wp, wm))
        assert abs(fd - wbar[m]) <= 1e-4 * abs(fd) + floor, (m, fd, wbar[m])
    rng = np.random.default_rng(2)
    for _ in range(8):
        a, i = int(rng.integers(p.n_pixels)), int(rng.integers(p.n_labels))
        php = p.unaries.astype(np.float64).copy(); php[a, i] += h
        phm = p.unaries.astype(np.float64).copy(); phm[a, i] -= h
        fd, floor = central(phi=(php, phm))
        assert abs(fd - phibar[a, i]) <= 1e-4 * abs(fd) + floor, (a, i, fd, phibar[a, i], floor)
