"""GPU parity of CCCP for negative semi-definite compatibilities (Section 5.2, Appendix C)."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf
from oracle import qp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tangent_nsd_mu(L, seed):
    # mu = 1 1^T - G with G positive definite: negative definite on zero-sum vectors
    rng = np.random.default_rng(seed)
    R = rng.normal(size=(L, L))
    return (np.ones((L, L)) - (R @ R.T / L + np.eye(L))).astype(np.float32)


def _run(dcrf, probs, outer, inner=0, mu=None, storage="f32"):
    g = gpu_setup(dcrf, probs, torch)
    Y = g["y0"].clone()
    e = dcrf.dcrf_dc_neg(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Y, outer, inner, compat=mu,
                         storage=storage)
    return g, Y.cpu().numpy(), e


def _check(probs, g, Y, e, outer, inner=0, mu=None, tol=1e-3):
    for b, p in enumerate(probs):
        c = oracle_crf(p, None if mu is None else mu.astype(np.float64))
        y_o, e_o = qp.cccp_dc_neg(c, p.y0, outer, inner)
        scale = np.abs(e_o).max()
        np.testing.assert_allclose(e[:, b], e_o, rtol=tol, atol=1e-6 * scale)
        # CCCP never raises S_QP (to FP32 rounding of the sums)
        assert np.all(np.diff(e[:, b]) <= 1e-5 * scale)
        s, t = g["off"][b], g["off"][b + 1]
        np.testing.assert_allclose(Y[s:t].sum(1), 1.0, atol=1e-5)
        assert Y[s:t].min() >= -1e-6
        # the labelling agrees with the oracle's on almost every pixel
        assert np.mean(Y[s:t].argmax(1) == y_o.argmax(1)) >= 0.99


def test_dcneg_potts_small(dcrf):
    p = S.qp_small()
    g, Y, e = _run(dcrf, [p], 6)
    _check([p], g, Y, e, 6)


def test_dcneg_potts_weak_pairwise(dcrf):
    # the filtered term mu F is large next to sum_w, so the projections land on
    # (or next to) vertices and CCCP settles within a few steps
    p = S.make_problem(48, 40, 6, 5, seed=21)
    p.weights = (0.5, 0.2)
    g, Y, e = _run(dcrf, [p], 8)
    _check([p], g, Y, e, 8)
    assert e[-1, 0] < e[0, 0]


def test_dcneg_fp16_storage(dcrf):
    p = S.make_problem(80, 60, 8, 21, seed=22)
    g, Y, e = _run(dcrf, [p], 5, storage="f16")
    _check([p], g, Y, e, 5, tol=2e-3)


def test_dcneg_general_mu(dcrf):
    p = S.crop(S.make_problem(48, 40, 5, 4, seed=23), 32, 24)
    p.weights = (0.6, 0.3)
    mu = _tangent_nsd_mu(4, 3)
    g, Y, e = _run(dcrf, [p], 4, inner=20, mu=mu)
    _check([p], g, Y, e, 4, inner=20, mu=mu)


def test_dcneg_batch_of_uneven_images(dcrf):
    probs = [S.make_problem(w, h, 5, 21, seed=30 + i) for i, (w, h) in enumerate([(40, 30), (7, 3), (33, 21)])]
    g, Y, e = _run(dcrf, probs, 4)
    _check(probs, g, Y, e, 4)


def test_dcneg_rejects_bad_arguments(dcrf):
    p = S.make_problem(16, 12, 3, 4, seed=24)
    g = gpu_setup(dcrf, [p], torch)
    asym = np.ones((4, 4), dtype=np.float32) - np.eye(4, dtype=np.float32)
    asym[0, 1] = 2.0
    with pytest.raises(dcrf.DcrfError) as err:
        dcrf.dcrf_dc_neg(g["phi"], [g["lb"], g["ls"]], p.weights, g["y0"].clone(), 2, 0, compat=asym)
    assert err.value.status == -1
    with pytest.raises(dcrf.DcrfError) as err:
        dcrf.dcrf_dc_neg(g["phi"], [g["lb"], g["ls"]], (0.0, 0.0), g["y0"].clone(), 2, 0)
    assert err.value.status == -1


def test_dcneg_headline_size(dcrf):
    # 500x375, L = 21 (no oracle at this size): monotone, finite, on the simplex
    p = S.voc_shaped()
    g, Y, e = _run(dcrf, [p], 10, storage="f16")
    assert np.isfinite(e).all()
    assert np.all(np.diff(e[:, 0]) <= 1e-5 * np.abs(e).max())
    np.testing.assert_allclose(Y.sum(1), 1.0, atol=1e-5)
    assert Y.min() >= -1e-6


@pytest.mark.parametrize("storage,tol", [("f32", 1e-4), ("f16", 2e-3)])
def test_dcneg_first_step_elementwise(dcrf, storage, tol):
    # One outer step from y0 is y1 = Proj(v), v = -(phi + mu F)/(2 sum_w),
    # F = K~y0 + K~^T y0 (Appendix C, Potts).  The projection onto the simplex
    # is 1-Lipschitz in the 2-norm, so |y1 - y1_oracle| <= sqrt(L) |dv|_inf
    # with |dv| <= (L - 1) |dF|_inf / (2 sum_w) and |dF| <= 2 tol max(K~1) by
    # the filter tolerance (K~ >= 0, 0 <= y0 <= 1): y1 is compared per
    # element against that bound.
    probs = [S.qp_small(), S.make_problem(80, 60, 8, 21, seed=22)]
    for p in probs:
        g, Y, e = _run(dcrf, [p], 1, storage=storage)
        c = oracle_crf(p)
        y_o, _ = qp.cccp_dc_neg(c, p.y0, 1, 0)
        L, sw = p.n_labels, c.kernel.sum_w
        bound = np.sqrt(L) * (L - 1) * 2 * tol * float((c.c_raw + sw).max()) / (2 * sw)
        err = float(np.abs(Y.astype(np.float64) - y_o).max())
        print(f"\n{storage} {p.width}x{p.height} L={L}: max |dy| {err:.3g} (bound {bound:.3g})")
        assert err <= bound
