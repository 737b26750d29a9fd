"""GPU parity of Frank-Wolfe (Algorithm 1, Appendix B) and CCCP (Algorithm 2)."""
import hashlib

import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf, rel_err
from oracle import qp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENERGY_TOL = 1e-3


def _run_fw(dcrf, probs, iters, storage="f32", mu=None):
    g = gpu_setup(dcrf, probs, torch)
    Y = g["y0"].clone()
    rec = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Y, iters, compat=mu, storage=storage)
    return g, Y.cpu().numpy(), rec


_ORACLE_RUNS = {}


def _oracle_fw(p, mu, iters):
    h = hashlib.sha1()
    for arr in (p.rgb, p.unaries, p.y0, np.asarray(p.weights), np.asarray(p.thetas)):
        h.update(np.ascontiguousarray(arr).tobytes())
    key = (h.hexdigest(), None if mu is None else np.asarray(mu).tobytes(), iters)
    if key not in _ORACLE_RUNS:
        c = oracle_crf(p, mu)
        _ORACLE_RUNS.clear()
        _ORACLE_RUNS[key] = (c,) + tuple(qp.frank_wolfe(c, p.y0, iters))
    c, y_o, _, rec_o = _ORACLE_RUNS[key]
    return c, y_o, rec_o


def _check_against_oracle(probs, g, Y, rec, iters, mu=None, tol=ENERGY_TOL, mono=1e-6):
    for b, p in enumerate(probs):
        c, y_o, rec_o = _oracle_fw(p, mu, iters)
        e_o = rec_o[:, 0]
        scale = np.abs(e_o).max()
        # per-iteration energy and the final relaxed energy
        assert np.abs(rec[:, b, 0] - e_o).max() <= tol * scale
        s, e = g["off"][b], g["off"][b + 1]
        assert abs(c.s_cvx(Y[s:e].astype(np.float64)) - c.s_cvx(y_o)) <= tol * abs(c.s_cvx(y_o))
        # gap non-negative (to rounding) and the energy never rises
        assert np.all(rec[:, b, 1] >= -1e-6 * scale)
        assert np.all(np.diff(rec[:, b, 0]) <= mono * scale)
        # the iterate stays on the simplex
        np.testing.assert_allclose(Y[s:e].sum(1), 1.0, atol=1e-5)
        assert Y[s:e].min() >= -1e-6


def test_fw_small_fp32(dcrf):
    p = S.qp_small()
    g, Y, rec = _run_fw(dcrf, [p], 50)
    _check_against_oracle([p], g, Y, rec, 50)


def test_fw_small_fp16_storage(dcrf):
    p = S.qp_small()
    g, Y, rec = _run_fw(dcrf, [p], 50, storage="f16")
    # float16 lattice values: the energy is non-increasing to float16 rounding
    _check_against_oracle([p], g, Y, rec, 50, mono=1e-4)


def test_fw_general_compatibility(dcrf):
    p = S.make_problem(48, 40, 6, 4, seed=9)
    rng = np.random.default_rng(1)
    mu = rng.uniform(0.0, 1.5, (4, 4))
    mu = (mu + mu.T) / 2
    np.fill_diagonal(mu, 0.0)
    g, Y, rec = _run_fw(dcrf, [p], 30, mu=mu)
    _check_against_oracle([p], g, Y, rec, 30, mu=mu)


def test_fw_batch_uneven(dcrf):
    probs = [S.make_problem(w, h, 7, 5, seed=30 + i) for i, (w, h) in enumerate([(40, 30), (3, 2), (64, 17)])]
    g, Y, rec = _run_fw(dcrf, probs, 25)
    _check_against_oracle(probs, g, Y, rec, 25)


def test_fw_headline_size(dcrf):
    p = S.voc_shaped()
    g, Y, rec = _run_fw(dcrf, [p], 8, storage="f16")
    _check_against_oracle([p], g, Y, rec, 8, mono=1e-4)


def test_fw_zero_iterations_leaves_y(dcrf):
    p = S.qp_small()
    g, Y, rec = _run_fw(dcrf, [p], 0)
    np.testing.assert_array_equal(Y, p.y0)


def test_cccp_medium(dcrf):
    p = S.qp_cccp_medium()
    g = gpu_setup(dcrf, [p], torch)
    Y = g["y0"].clone()
    # QP Frank-Wolfe first, then CCCP from its result (10 outer x 50 inner)
    dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 50, records=False)
    yq = Y.cpu().numpy().astype(np.float64)
    e = dcrf.dcrf_dc_cccp(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 10, 50)[:, 0]
    c = oracle_crf(p)
    y_o, _, _ = qp.frank_wolfe(c, p.y0, 50)
    y_c, e_o = qp.cccp_dc_gen(c, y_o, 10, 50)
    scale = np.abs(e_o).max()
    assert np.all(np.diff(e) <= 1e-5 * scale)                    # monotone (Section 5.1)
    assert abs(e[0] - c.s_qp(yq)) <= ENERGY_TOL * scale
    assert abs(e[-1] - e_o[-1]) <= ENERGY_TOL * scale
    yg = Y.cpu().numpy().astype(np.float64)
    assert abs(c.s_qp(yg) - e[-1]) <= ENERGY_TOL * scale


def test_cccp_medium_elementwise(dcrf):
    # C2: QP Frank-Wolfe (50 iterations) then CCCP 10 x 50 at 320x213, L=21,
    # FP32.  The oracle replays the GPU's decisions of both phases (each an
    # argmin of the FP64 gradient up to the FP32 filter tolerance: see
    # tests/test_gpu_fw_parity.py), and S_QP after every outer step and the
    # final y are compared element by element.
    p = S.qp_cccp_medium()
    g = gpu_setup(dcrf, [p], torch)
    Y = g["y0"].clone()
    _, tq = dcrf.dcrf_qp_fw_trace(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 50)
    yq = Y.cpu().numpy()
    e, tc = dcrf.dcrf_dc_cccp_trace(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 10, 50)
    c = oracle_crf(p)
    bound = 4.0 * 1e-4 * float((c.c_raw + c.kernel.sum_w).max())
    rows = np.arange(c.n)
    worst = [0.0]

    def on_step(t, gr, s):
        worst[0] = max(worst[0], float((gr[rows, s] - gr.min(axis=1)).max()))

    y_o, _, _ = qp.frank_wolfe(c, p.y0, 50, decisions=tq.cpu().numpy().astype(np.int64), on_step=on_step)
    assert np.abs(yq - y_o).max() <= 1e-3
    y_c, e_o = qp.cccp_dc_gen(c, yq.astype(np.float64), 10, 50, decisions=tc.cpu().numpy().astype(np.int64),
                              on_step=on_step)
    scale = np.abs(e_o).max()
    print(f"\nCCCP 320x213: energies {np.abs(e[:, 0] - e_o).max() / scale:.3g}, "
          f"y {np.abs(Y.cpu().numpy() - y_c).max():.3g}, excess/bound {worst[0] / bound:.3g}")
    assert worst[0] <= bound
    assert np.abs(e[:, 0] - e_o).max() <= ENERGY_TOL * scale
    assert np.all(np.diff(e[:, 0]) <= 1e-5 * scale)                # monotone (Section 5.1)
    assert np.abs(Y.cpu().numpy() - y_c).max() <= 1e-3


def test_fw_graph_path_matches_eager(dcrf):
    # a non-default stream takes the captured two-iteration graph path
    p = S.make_problem(64, 48, 5, 5, seed=12)
    g = gpu_setup(dcrf, [p], torch)
    Y1 = g["y0"].clone()
    r1 = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y1, 21)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Y2 = g["y0"].clone()
        r2 = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y2, 21, stream=s)
    s.synchronize()
    # the same kernels in the same order, and the one-hot splat sums integers:
    # the replayed graph reproduces the eager run bit for bit
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(Y1.cpu().numpy(), Y2.cpu().numpy())


@pytest.mark.parametrize("variant", range(19))
def test_fw_every_pixel_variant(dcrf, variant, monkeypatch):
    # the autotuner chooses among these layouts of the pixel pass (block
    # shapes, index prefetch, packed FMAs, three lanes per pixel, gather
    # during the tile copy, bulk tile copies, the label count fixed at 21);
    # each must follow the oracle
    monkeypatch.setenv("DCRF_PIXEL_VARIANT", str(variant))
    p = S.make_problem(96, 64, 8, 21, seed=13)
    for storage in ("f32", "f16"):
        g, Y, rec = _run_fw(dcrf, [p], 15, storage=storage)
        _check_against_oracle([p], g, Y, rec, 15, mono=1e-6 if storage == "f32" else 1e-4)


@pytest.mark.parametrize("variant", [12, 13, 14, 15, 16])
def test_fw_bulk_variant_on_unaligned_batch(dcrf, variant, monkeypatch):
    # chunks whose rows do not start or end on 16 bytes fall back to cp.async
    # (image 0 ends after 851 pixels: 851 x 21 floats is not a multiple of 4)
    monkeypatch.setenv("DCRF_PIXEL_VARIANT", str(variant))
    probs = [S.make_problem(37, 23, 5, 21, seed=71), S.make_problem(41, 19, 5, 21, seed=72)]
    for storage in ("f32", "f16"):
        g, Y, rec = _run_fw(dcrf, probs, 12, storage=storage)
        _check_against_oracle(probs, g, Y, rec, 12, mono=1e-6 if storage == "f32" else 1e-4)


@pytest.mark.parametrize("blur", [0, 1, 2])
@pytest.mark.parametrize("L", [5, 21, 40])
def test_fw_each_blur_kernel(dcrf, blur, L, monkeypatch):
    # the blur tuner chooses a row per thread (0), label-split rows (1) or the
    # persistent form (2); each follows the oracle for 8-, 24- and 64-wide rows
    monkeypatch.setenv("DCRF_BLUR_VARIANT", str(blur))
    p = S.make_problem(64, 48, 6, L, seed=80 + L)
    for storage in ("f32", "f16"):
        g, Y, rec = _run_fw(dcrf, [p], 10, storage=storage)
        _check_against_oracle([p], g, Y, rec, 10, mono=1e-6 if storage == "f32" else 1e-4)


def test_fw_persistent_blur_strides_over_many_rows(dcrf, monkeypatch):
    # 10 images of 500x375: ~460k vertex rows, more than one row per thread of
    # the persistent blur's resident grid; two sampled images follow the oracle
    monkeypatch.setenv("DCRF_BLUR_VARIANT", "2")
    B, iters = 10, 6
    probs = [S.make_problem(500, 375, 30, 21, seed=200 + i) for i in range(B)]
    g = gpu_setup(dcrf, probs, torch)
    assert g["lb"].m + g["ls"].m > 152 * 8 * 256
    Y = g["y0"].clone()
    rec = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Y, iters, storage="f16")
    for b in (0, B - 1):
        c = oracle_crf(probs[b])
        _, _, rec_o = qp.frank_wolfe(c, probs[b].y0, iters)
        scale = np.abs(rec_o[:, 0]).max()
        assert np.abs(rec[:, b, 0] - rec_o[:, 0]).max() <= 1e-3 * scale


def test_fw_fixed_label_count_variant_falls_back(dcrf, monkeypatch):
    # the variants compiled for L = 21 are never used for another label count:
    # forcing one with L = 5 runs the generic layout
    monkeypatch.setenv("DCRF_PIXEL_VARIANT", "16")
    p = S.qp_small()
    g, Y, rec = _run_fw(dcrf, [p], 20)
    _check_against_oracle([p], g, Y, rec, 20)
