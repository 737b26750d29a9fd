"""GPU parity of the mean-field baseline, rounding and labelling energy (Section 1, Section 6.2)."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf, rel_err
from oracle import mf
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mf_case(dcrf, probs, iters, storage="f32", tol=1e-3, qtol=1e-3):
    g = gpu_setup(dcrf, probs, torch)
    Q = g["y0"].clone()                        # softmax(-phi), the usual start
    e = dcrf.dcrf_mean_field(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Q, iters, storage=storage)
    Qg = Q.cpu().numpy()
    for b, p in enumerate(probs):
        c = oracle_crf(p)
        Qo, eo = mf.mean_field(c, p.y0, iters)
        np.testing.assert_allclose(e[:, b], eo, rtol=tol, atol=1e-6 * np.abs(eo).max())
        s, t = g["off"][b], g["off"][b + 1]
        assert np.abs(Qg[s:t] - Qo).max() <= qtol
        np.testing.assert_allclose(Qg[s:t].sum(1), 1.0, atol=1e-5)
    return g, Qg


def test_mean_field_small(dcrf):
    _mf_case(dcrf, [S.qp_small()], 5)


def test_mean_field_mf5_21_labels_fp16(dcrf):
    _mf_case(dcrf, [S.make_problem(96, 64, 8, 21, seed=41)], 5, storage="f16", tol=2e-3, qtol=5e-3)


def test_mean_field_batch(dcrf):
    probs = [S.make_problem(w, h, 5, 21, seed=42 + i) for i, (w, h) in enumerate([(40, 30), (9, 4), (31, 22)])]
    _mf_case(dcrf, probs, 5)


def test_round_and_labelling_energy(dcrf):
    probs = [S.make_problem(48, 36, 6, 21, seed=50), S.make_problem(20, 17, 4, 21, seed=51)]
    g = gpu_setup(dcrf, probs, torch)
    Y = g["y0"].clone()
    Y[::7] = 1.0 / 21                          # exact ties: the lowest label wins
    labels, onehot = dcrf.dcrf_round(Y, onehot=True)
    lab = labels.cpu().numpy()
    np.testing.assert_array_equal(lab, mf.round_labels(Y.cpu().numpy()))
    np.testing.assert_array_equal(onehot.cpu().numpy(), np.eye(21, dtype=np.float32)[lab])
    e = dcrf.dcrf_labelling_energy(g["phi"], [g["lb"], g["ls"]], probs[0].weights, labels)
    for b, p in enumerate(probs):
        s, t = g["off"][b], g["off"][b + 1]
        eo = oracle_crf(p).energy(lab[s:t])
        assert rel_err(e[b], eo) <= 1e-4


def test_labelling_energy_rejects_out_of_range_labels(dcrf):
    p = S.make_problem(16, 12, 3, 4, seed=52)
    g = gpu_setup(dcrf, [p], torch)
    labels = torch.zeros(p.n_pixels, dtype=torch.int32, device="cuda")
    labels[3] = 4
    with pytest.raises(dcrf.DcrfError) as err:
        dcrf.dcrf_labelling_energy(g["phi"], [g["lb"], g["ls"]], p.weights, labels)
    assert err.value.status == -1
