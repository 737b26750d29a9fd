"""The paper's best pipeline, QP -> DC_neg -> LP -> rounding (Section 6.1, the
QP-DC_neg-LP rows), on the GPU, checked stage by stage against the oracle
started from the GPU's previous stage."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf
from oracle import lp, mf, qp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_qp_dcneg_lp_pipeline(dcrf):
    p = S.make_problem(48, 36, 6, 5, seed=70)
    g = gpu_setup(dcrf, [p], torch)
    lats = [g["lb"], g["ls"]]
    c = oracle_crf(p)
    Y = g["y0"].clone()

    # 1. convex QP by Frank-Wolfe
    dcrf.dcrf_qp_fw(g["phi"], lats, p.weights, Y, 30, records=False)
    y_qp = Y.cpu().numpy().astype(np.float64)
    y_o, _, _ = qp.frank_wolfe(c, p.y0, 30)
    assert abs(c.s_cvx(y_qp) - c.s_cvx(y_o)) <= 1e-3 * abs(c.s_cvx(y_o))

    # 2. DC_neg from the QP solution: S_QP does not rise, and matches the oracle
    e_dc = dcrf.dcrf_dc_neg(g["phi"], lats, p.weights, Y, 4, 0)[:, 0]
    _, e_dc_o = qp.cccp_dc_neg(c, y_qp, 4)
    np.testing.assert_allclose(e_dc, e_dc_o, rtol=1e-3)
    assert e_dc[-1] <= e_dc[0] + 1e-5 * abs(e_dc[0])
    y_dc = Y.cpu().numpy().astype(np.float64)

    # 3. LP projected subgradient from the DC solution (best iterate kept)
    e_lp = dcrf.dcrf_lp_solve(g["phi"], lats, p.weights, Y, 10)[:, 0]
    _, e_lp_o = lp.lp_solve(c.phi, y_dc, c.c, c.kernel.apply_partitioned, 10)
    scale = np.abs(e_lp_o).max()
    assert abs(e_lp[0] - e_lp_o[0]) <= 1e-4 * scale
    assert abs(e_lp.min() - e_lp_o.min()) <= 1e-3 * scale

    # 4. rounding and the energy of the labelling (Eq. 1)
    labels = dcrf.dcrf_round(Y)
    lab = labels.cpu().numpy()
    np.testing.assert_array_equal(lab, mf.round_labels(Y.cpu().numpy()))
    E = dcrf.dcrf_labelling_energy(g["phi"], lats, p.weights, labels)[0]
    np.testing.assert_allclose(E, c.energy(lab), rtol=1e-4)
    # the pipeline ends at least as low as rounding the QP solution directly
    E_qp = c.energy(mf.round_labels(y_qp))
    assert E <= E_qp + 1e-3 * abs(E_qp)
