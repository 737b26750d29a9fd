"""Element-wise parity of Frank-Wolfe (Algorithm 1, Appendix B) with the oracle.

The GPU returns its decisions s^t (dcrf_qp_fw_trace); the oracle replays them
in FP64.  What is unique is then compared element by element: every
per-iteration scalar (energy, gap, alpha, A, B) of every image and y^T per
pixel.  What is not unique, the argmin at a near-tie, is checked for
validity: at every iteration and pixel the GPU's label must be an argmin of
the oracle's gradient up to the gradient error that the filter tolerance
allows.  With Potts, g(i) - g(j) = lin(i) - lin(j) + 2 (X(j) - X(i)) + ...
with X = K~y - sum_w y, so a filter error of tol * max (K~y) moves a gradient
difference by at most 4 tol max (K~y) <= 4 tol max (K~1) (K~ has non-negative
entries and 0 <= y <= 1): a label whose oracle excess over the minimum exceeds
that bound could not have been chosen by a correct kernel.
"""
import numpy as np
import pytest

from helpers import check_replay, gpu_setup, replay_image
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(dcrf, probs, iters, storage):
    g = gpu_setup(dcrf, probs, torch)
    Y = g["y0"].clone()
    rec, trace = dcrf.dcrf_qp_fw_trace(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Y, iters, storage=storage)
    return g, Y.cpu().numpy(), rec, trace.cpu().numpy()


def _parity(dcrf, probs, iters, storage, images=None):
    g, Y, rec, trace = _run(dcrf, probs, iters, storage)
    assert trace.shape == (iters, Y.shape[0])
    out = []
    for b in (range(len(probs)) if images is None else images):
        s0, s1 = g["off"][b], g["off"][b + 1]
        p = probs[b]
        assert trace[:, s0:s1].max() < p.n_labels
        err = replay_image(p, Y[s0:s1], rec[:, b], trace[:, s0:s1], storage, iters)
        check_replay(err, f"{storage} image {b} ({p.width}x{p.height}, L={p.n_labels}, {iters} iterations)")
        out.append(err)
    return g, Y, rec, out


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_fw_elementwise_small(dcrf, storage):
    _parity(dcrf, [S.qp_small()], 50, storage)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_fw_elementwise_21_labels_uneven_batch(dcrf, storage):
    probs = [S.make_problem(w, h, 8, 21, seed=40 + i) for i, (w, h) in enumerate([(96, 64), (37, 23), (3, 2),
                                                                                     (120, 17)])]
    _parity(dcrf, probs, 30, storage)


def test_fw_elementwise_headline_configuration(dcrf):
    # the benchmarked configuration: 500x375, L=21, FP16 lattice storage,
    # 100 iterations (the per-iteration graph replay of the solver)
    _parity(dcrf, [S.voc_shaped()], 100, "f16")


def test_fw_elementwise_uneven_batch_at_size(dcrf):
    # 32 images of W ~ U[240,500] x H ~ U[160,500] in one call, FP16 lattice
    # storage, 100 iterations; four images replayed in full (the smallest, the
    # largest and two more), every image checked for a valid run
    probs = S.make_batch(32, 0)
    sizes = np.array([p.n_pixels for p in probs])
    pick = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 7, 21})
    g, Y, rec, _ = _parity(dcrf, probs, 100, "f16", images=pick)
    for b in range(len(probs)):
        s0, s1 = g["off"][b], g["off"][b + 1]
        e = rec[:, b, 0]
        scale = np.abs(e).max()
        assert np.all(np.isfinite(rec[:, b]))
        assert np.all(rec[:, b, 1] >= -1e-6 * scale)            # gap >= 0 up to rounding
        assert np.all(np.diff(e) <= 1e-4 * scale)                # energy non-increasing up to FP16
        np.testing.assert_allclose(Y[s0:s1].sum(1), 1.0, atol=1e-5)
        assert Y[s0:s1].min() >= -1e-6
