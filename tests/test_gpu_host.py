"""The host-buffer entry point (features, both lattices, Frank-Wolfe and the
copies in one C call) against the oracle, per image of a ragged batch."""
import numpy as np
import pytest

from helpers import oracle_crf
from oracle import qp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(probs):
    rgb = np.ascontiguousarray(np.concatenate([p.rgb.reshape(-1, 3) for p in probs]).astype(np.float32))
    phi = np.ascontiguousarray(np.concatenate([p.unaries for p in probs]))
    y0 = np.ascontiguousarray(np.concatenate([p.y0 for p in probs]))
    return rgb, phi, y0, [p.width for p in probs], [p.height for p in probs]


def _check_against_oracle(probs, Y, rec, iters):
    off = np.concatenate([[0], np.cumsum([p.n_pixels for p in probs])])
    np.testing.assert_allclose(Y.sum(1), 1.0, atol=1e-5)
    for b, p in enumerate(probs):
        if p.n_pixels == 0:
            continue
        c = oracle_crf(p)
        y_o, _, rec_o = qp.frank_wolfe(c, p.y0, iters)
        scale = np.abs(rec_o[:, 0]).max()
        assert np.abs(rec[:, b, 0] - rec_o[:, 0]).max() <= 1e-3 * scale
        assert abs(c.s_cvx(Y[off[b]:off[b + 1]].astype(np.float64)) - c.s_cvx(y_o)) <= 1e-3 * scale


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_host_path_pageable_ragged_batch(dcrf, storage):
    probs = [S.make_problem(w, h, 5, 6, seed=110 + i) for i, (w, h) in enumerate([(40, 30), (17, 23), (33, 9)])]
    rgb, phi, y0, ws, hs = _inputs(probs)
    y0_keep = y0.copy()
    Y, rec = dcrf.dcrf_qp_fw_host(rgb, phi, y0, ws, hs, probs[0].thetas, probs[0].weights, 12, storage=storage,
                                  records=True)
    np.testing.assert_array_equal(y0, y0_keep)          # the input is not written
    _check_against_oracle(probs, Y, rec, 12)


def test_host_path_pinned_in_place_with_an_empty_image(dcrf):
    probs = [S.make_problem(36, 28, 5, 5, seed=120), S.make_problem(25, 19, 5, 5, seed=121)]
    rgb, phi, y0, ws, hs = _inputs(probs)
    ws = [ws[0], 0, ws[1]]
    hs = [hs[0], 7, hs[1]]
    rgb_t = torch.from_numpy(rgb).pin_memory()
    phi_t = torch.from_numpy(phi).pin_memory()
    y_t = torch.from_numpy(y0).pin_memory()
    Y, rec = dcrf.dcrf_qp_fw_host(rgb_t, phi_t, y_t, ws, hs, probs[0].thetas, probs[0].weights, 10, Y=y_t,
                                  records=True)
    assert Y is y_t
    assert np.all(rec[:, 1, 0] == 0.0)
    rec = rec[:, [0, 2]]
    _check_against_oracle(probs, y_t.numpy(), rec, 10)


def test_host_path_matches_the_device_path(dcrf):
    # the same calls a user would make with device tensors give the same energies
    probs = [S.make_problem(48, 36, 6, 21, seed=130), S.make_problem(30, 41, 6, 21, seed=131)]
    rgb, phi, y0, ws, hs = _inputs(probs)
    _, rec_h = dcrf.dcrf_qp_fw_host(rgb, phi, y0, ws, hs, probs[0].thetas, probs[0].weights, 15, storage="f16",
                                    records=True)
    fb, fs = dcrf.dcrf_features(torch.from_numpy(rgb).cuda(), ws, hs, *probs[0].thetas)
    off = np.concatenate([[0], np.cumsum([p.n_pixels for p in probs])])
    lb, ls = dcrf.dcrf_lattice_build(fb, off), dcrf.dcrf_lattice_build(fs, off)
    Yd = torch.from_numpy(y0).cuda()
    rec_d = dcrf.dcrf_qp_fw(torch.from_numpy(phi).cuda(), [lb, ls], probs[0].weights, Yd, 15, storage="f16")
    scale = np.abs(rec_d[:, :, 0]).max()
    assert np.abs(rec_h[:, :, 0] - rec_d[:, :, 0]).max() <= 1e-5 * scale


def test_host_path_rejects_mismatched_buffers(dcrf):
    p = S.make_problem(10, 8, 3, 4, seed=140)
    rgb, phi, y0, ws, hs = _inputs([p])
    with pytest.raises(ValueError):
        dcrf.dcrf_qp_fw_host(rgb[:-1], phi, y0, ws, hs, p.thetas, p.weights, 2)
    with pytest.raises(ValueError):
        dcrf.dcrf_qp_fw_host(rgb, phi, y0[:, :3].copy(), ws, hs, p.thetas, p.weights, 2)
    with pytest.raises(ValueError):
        dcrf.dcrf_qp_fw_host(rgb, phi.astype(np.float64), y0, ws, hs, p.thetas, p.weights, 2)


def test_pool_trim_between_calls(dcrf):
    # the cached scratch can be handed back; later calls map it again
    p = S.make_problem(30, 20, 4, 5, seed=150)
    rgb, phi, y0, ws, hs = _inputs([p])
    _, r1 = dcrf.dcrf_qp_fw_host(rgb, phi, y0, ws, hs, p.thetas, p.weights, 8, records=True)
    torch.cuda.synchronize()
    dcrf.pool_trim()
    _, r2 = dcrf.dcrf_qp_fw_host(rgb, phi, y0, ws, hs, p.thetas, p.weights, 8, records=True)
    np.testing.assert_allclose(r1[:, :, 0], r2[:, :, 0], rtol=1e-5)
