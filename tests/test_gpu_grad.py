"""GPU reverse mode through unrolled Frank-Wolfe against the oracle and FP64 finite differences."""
import numpy as np
import pytest

from helpers import gpu_setup, rel_err
from oracle import crf, qp
from oracle import permutohedral as P
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _oracle(p, w=None, phi=None):
    fb, fs = crf.features(p.rgb, *p.thetas)
    lats = [P.Permutohedral(crf.to_fp32_features(fb)), P.Permutohedral(crf.to_fp32_features(fs))]
    return qp.WeightedCRF(p.unaries if phi is None else phi, [(l.filter, l.filter_adjoint) for l in lats],
                          p.weights if w is None else w)


def _min_margin(c, tape):
    """Smallest gap between the two lowest gradient entries along the path, relative to |g|."""
    lin = c.phi - c.d
    worst = np.inf
    for y, _, _, _, _ in tape:
        g = lin + 2.0 * c.op(y)
        gs = np.sort(g, axis=1)
        worst = min(worst, float(((gs[:, 1] - gs[:, 0]) / (np.abs(gs[:, 0]) + 1.0)).min()))
    return worst


def _robust_crop(L, iters, seeds=range(20)):
    """A 32x24 crop whose Frank-Wolfe path has no argmin within FP32 reach of a tie.

    The unrolled iteration is piecewise smooth: s^t is constant between ties of
    the gradient.  Its derivative is the same in FP32 and FP64 only where both
    follow the same path, so the comparison uses a crop whose smallest relative
    argmin margin is far above FP32 resolution.
    """
    for seed in seeds:
        p = S.crop(S.make_problem(48, 40, 5, L, seed=seed), 32, 24)
        c = _oracle(p)
        _, tape = qp.fw_tape(c, p.y0, iters)
        if _min_margin(c, tape) > 1e-5:
            return p, c, tape
    pytest.fail("no crop with a robust Frank-Wolfe path")


def _gpu_grad(dcrf, probs, ybar, iters):
    g = gpu_setup(dcrf, probs, torch)
    dYT = torch.from_numpy(ybar.astype(np.float32)).cuda()
    dphi, dw, _ = dcrf.dcrf_qp_fw_backward(g["phi"], [g["lb"], g["ls"]], probs[0].weights, g["y0"], dYT, iters)
    return g, dphi.cpu().numpy(), dw


def test_backward_matches_oracle_and_finite_differences(dcrf):
    iters = 10
    p, c, tape = _robust_crop(4, iters)
    ybar = np.random.default_rng(1).normal(size=(p.n_pixels, p.n_labels))
    _, dphi, dw = _gpu_grad(dcrf, [p], ybar, iters)
    phibar, wbar, _ = qp.fw_backward(c, tape, ybar)
    assert rel_err(dphi, phibar) <= 1e-4
    assert rel_err(dw, wbar) <= 1e-4
    # FP64 central differences (h = 1e-4) of the oracle's forward, where no s^t flips
    h = 1e-4

    def loss(w=None, phi=None):
        y, tp = qp.fw_tape(_oracle(p, w, phi), p.y0, iters)
        return float(np.sum(ybar * y)), tp

    for m in range(2):
        wp = np.array(p.weights, float); wp[m] += h
        wm = np.array(p.weights, float); wm[m] -= h
        (fp, tp), (fm, tm) = loss(w=wp), loss(w=wm)
        assert all(np.array_equal(a[1], b[1]) for a, b in zip(tp, tape))
        assert all(np.array_equal(a[1], b[1]) for a, b in zip(tm, tape))
        fd = (fp - fm) / (2 * h)
        assert abs(dw[m] - fd) <= 1e-4 * np.abs(wbar).max()
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(10):
        a, i = int(rng.integers(p.n_pixels)), int(rng.integers(p.n_labels))
        php = p.unaries.astype(np.float64).copy(); php[a, i] += h
        phm = p.unaries.astype(np.float64).copy(); phm[a, i] -= h
        (fp, tp), (fm, tm) = loss(phi=php), loss(phi=phm)
        if not all(np.array_equal(x[1], y[1]) for x, y in zip(tp + tm, tape + tape)):
            continue
        fd = (fp - fm) / (2 * h)
        assert abs(dphi[a, i] - fd) <= 1e-4 * max(abs(fd), np.abs(phibar).max() * 1e-2)
        checked += 1
    assert checked >= 6


def test_backward_21_labels_along_the_gpu_path(dcrf):
    # With 21 labels some argmin decisions of the path sit within FP32
    # rounding of a tie, so FP32 and FP64 runs may take different smooth
    # pieces of the unrolled map.  The GPU returns the decisions s^t of the
    # forward it differentiated; the oracle replays them (each must be an
    # argmin of the FP64 gradient up to the FP32 filter tolerance) and both
    # sides then differentiate the same piece: 1e-4 against the oracle's
    # reverse mode and against FP64 central differences (h = 1e-4) along it.
    iters = 10
    p = S.crop(S.make_problem(48, 40, 5, 21, seed=3), 32, 24)
    ybar = np.random.default_rng(1).normal(size=(p.n_pixels, p.n_labels))
    g = gpu_setup(dcrf, [p], torch)
    dYT = torch.from_numpy(ybar.astype(np.float32)).cuda()
    dphi, dw, _, st = dcrf.dcrf_qp_fw_backward(g["phi"], [g["lb"], g["ls"]], p.weights, g["y0"], dYT, iters,
                                               tape=True)
    dphi, dec = dphi.cpu().numpy(), st.cpu().numpy().astype(np.int64)
    c = _oracle(p)
    _, tape = qp.fw_tape(c, p.y0, iters, decisions=dec)
    bound = 4 * 1e-4 * float(sum(w * o for w, o in zip(c.w, c.o)).max())
    rows = np.arange(c.n)
    for t, (y, _, _, _, _) in enumerate(tape):
        gr = c.phi - c.d + 2.0 * c.op(y)
        assert float((gr[rows, dec[t]] - gr.min(axis=1)).max()) <= bound
    phibar, wbar, _ = qp.fw_backward(c, tape, ybar)
    assert rel_err(dphi, phibar) <= 1e-4
    assert rel_err(dw, wbar) <= 1e-4
    h = 1e-4

    def loss(w=None, phi=None):
        y, tp = qp.fw_tape(_oracle(p, w, phi), p.y0, iters, decisions=dec)
        assert all((0 < a[2] < 1) == (0 < b[2] < 1) for a, b in zip(tp, tape))
        return float(np.sum(ybar * y))

    def central(**kw):
        fp, fm = loss(**{k: v[0] for k, v in kw.items()}), loss(**{k: v[1] for k, v in kw.items()})
        return (fp - fm) / (2 * h), 8 * np.finfo(float).eps * max(abs(fp), abs(fm)) / (2 * h)

    for m in range(2):
        wp = np.array(p.weights, float); wp[m] += h
        wm = np.array(p.weights, float); wm[m] -= h
        fd, floor = central(w=(wp, wm))
        assert abs(dw[m] - fd) <= 1e-4 * abs(fd) + floor
    rng = np.random.default_rng(4)
    for _ in range(8):
        a, i = int(rng.integers(p.n_pixels)), int(rng.integers(p.n_labels))
        php = p.unaries.astype(np.float64).copy(); php[a, i] += h
        phm = p.unaries.astype(np.float64).copy(); phm[a, i] -= h
        fd, floor = central(phi=(php, phm))
        # the GPU value carries FP32 rounding: 1e-4 of the largest entry
        assert abs(dphi[a, i] - fd) <= 1e-4 * np.abs(phibar).max() + floor


def test_autograd_function_on_batch(dcrf, monkeypatch):
    # The one-hot splat sums fixed-point weights with integer reductions, so a
    # run does not depend on the order of the atomics, and an image of a batch
    # is processed exactly as alone when the same kernel variants run (forced
    # here: the tuners may choose others for other sizes), so the decisions
    # s^t agree.  The reverse sweep's filters still splat with float32
    # atomics, so every image gets the gradient it gets alone to 1e-5, and the
    # weight gradient, a sum over the images of terms that partly cancel, is
    # their sum to the gradient tolerance 1e-4.
    from paper_1608_06192_gb300.autograd import FrankWolfeQP
    monkeypatch.setenv("DCRF_PIXEL_VARIANT", "14")
    monkeypatch.setenv("DCRF_BLUR_VARIANT", "0")
    probs = [S.make_problem(320, 213, 30, 21, seed=60 + i) for i in range(8)]
    g = gpu_setup(dcrf, probs, torch)
    phi = g["phi"].clone().requires_grad_(True)
    w = torch.tensor(probs[0].weights, dtype=torch.float64, requires_grad=True)
    ybar = np.random.default_rng(2).normal(size=tuple(g["phi"].shape)).astype(np.float32)
    G = torch.from_numpy(ybar).cuda()
    y = FrankWolfeQP.apply(phi, w, g["y0"], [g["lb"], g["ls"]], 10)
    (y * G).sum().backward()
    dphi = phi.grad.cpu().numpy()
    assert np.isfinite(dphi).all() and torch.isfinite(w.grad).all()
    dw_sum = np.zeros(2)
    for b in range(8):
        s0, s1 = g["off"][b], g["off"][b + 1]
        _, dphi_b, dw_b = _gpu_grad(dcrf, [probs[b]], ybar[s0:s1], 10)
        dw_sum += dw_b
        assert rel_err(dphi[s0:s1], dphi_b) <= 1e-5
    assert rel_err(w.grad.numpy(), dw_sum) <= 1e-4
