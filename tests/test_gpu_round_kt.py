"""GPU parity of the Kleinberg-Tardos rounding (end of Section 5): labels are
integers decided in FP32 on both sides, so they must agree bit for bit."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_crf
from oracle import lp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,L,T", [(1037, 21, 60), (4099, 5, 12), (300, 64, 400), (1, 3, 2)])
def test_kt_rounding_matches_the_oracle(dcrf, n, L, T):
    y = S.dirichlet_labels(n, L, seed=n + L)
    pl, pt = S.kt_phases(L, T, seed=T)
    lab, left = dcrf.dcrf_round_kt(torch.from_numpy(y).cuda(), pl, pt)
    ref = lp.kt_round(y, pl, pt)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)
    assert left == int((ref < 0).sum())


def test_kt_rounding_continued_with_more_phases(dcrf):
    y = S.dirichlet_labels(5000, 21, seed=1)
    pl, pt = S.kt_phases(21, 300, seed=2)
    Y = torch.from_numpy(y).cuda()
    lab, left = dcrf.dcrf_round_kt(Y, pl[:15], pt[:15])
    assert 0 < left < 5000
    lab2, left2 = dcrf.dcrf_round_kt(Y, pl[15:], pt[15:], labels=lab)
    assert lab2.data_ptr() == lab.data_ptr()
    ref = lp.kt_round(y, pl, pt)
    np.testing.assert_array_equal(lab2.cpu().numpy(), ref)
    assert left2 == int((ref < 0).sum())


def test_kt_rounding_full_image_and_its_energy(dcrf):
    # one 500x375 image, L=21: 700 phases leave a pixel unlabelled with
    # probability (20/21)^700 ~ 1e-15; the labelling's energy (Eq. 1) through
    # the lattices matches the oracle's energy of the same labelling
    y = S.dirichlet_labels(500 * 375, 21, seed=3)
    pl, pt = S.kt_phases(21, 700, seed=4)
    lab, left = dcrf.dcrf_round_kt(torch.from_numpy(y).cuda(), pl, pt)
    ref = lp.kt_round(y, pl, pt)
    np.testing.assert_array_equal(lab.cpu().numpy(), ref)
    assert left == int((ref < 0).sum()) == 0
    small = S.make_problem(64, 48, 5, 21, seed=5)
    gs = gpu_setup(dcrf, [small], torch)
    ys = S.dirichlet_labels(small.n_pixels, 21, seed=6)
    lab_s, _ = dcrf.dcrf_round_kt(torch.from_numpy(ys).cuda(), pl, pt)
    E = dcrf.dcrf_labelling_energy(gs["phi"], [gs["lb"], gs["ls"]], small.weights, lab_s)[0]
    np.testing.assert_allclose(E, oracle_crf(small).energy(lab_s.cpu().numpy()), rtol=1e-4)


def test_kt_rounding_edges(dcrf):
    # no pixels; one label (y = 1 beats every threshold); a labelling
    lab, left = dcrf.dcrf_round_kt(torch.zeros((0, 4), device="cuda"), [1], [0.5])
    assert lab.numel() == 0 and left == 0
    lab, left = dcrf.dcrf_round_kt(torch.ones((77, 1), device="cuda"), [0, 0], [0.999, 0.0])
    assert left == 0 and torch.all(lab == 0)
    x = np.random.default_rng(7).integers(0, 6, size=999)
    pl, pt = S.kt_phases(6, 500, seed=8)
    lab, left = dcrf.dcrf_round_kt(torch.from_numpy(np.eye(6, dtype=np.float32)[x]).cuda(), pl, pt)
    np.testing.assert_array_equal(lab.cpu().numpy(), x)
    # no phases at all: every pixel stays unlabelled
    lab, left = dcrf.dcrf_round_kt(torch.full((10, 3), 1.0 / 3, device="cuda"), [], [])
    assert left == 10 and torch.all(lab == -1)


@pytest.mark.parametrize("labels,thresholds", [([3], [0.5]), ([-1], [0.5]), ([0], [1.0]), ([0], [-0.1]),
                                               ([0], [np.nan])])
def test_kt_rounding_rejects_bad_phases(dcrf, labels, thresholds):
    Y = torch.full((10, 3), 1.0 / 3, device="cuda")
    with pytest.raises(RuntimeError):
        dcrf.dcrf_round_kt(Y, labels, thresholds)
