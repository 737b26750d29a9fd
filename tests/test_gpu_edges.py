"""Edge cases at the limits of the boundary: label counts 1, 25 and 64, d = 8,
an empty image inside a batch, and the full 32-image batch of the benchmark
(sampled images against the oracle run alone)."""
import numpy as np
import pytest

from helpers import check_replay, gpu_setup, oracle_crf, rel_err, replay_image
from oracle import permutohedral as P
from oracle import qp
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L", [1, 25, 64])
def test_filter_label_counts(dcrf, L):
    # L = 1 (one channel), 25 (first count above the 24-wide rows) and 64 (the maximum)
    p = S.make_problem(40, 30, 4, max(L, 2), seed=60 + L)
    g = gpu_setup(dcrf, [p], torch)
    Y = np.random.default_rng(L).uniform(size=(p.n_pixels, L)).astype(np.float32)
    for key, fkey in (("lb", "fb"), ("ls", "fs")):
        out = dcrf.dcrf_filter(g[key], torch.from_numpy(Y).cuda()).cpu().numpy()
        ref = P.Permutohedral(g[fkey].cpu().numpy()).filter(Y)
        assert rel_err(out, ref) <= 1e-4


def test_lattice_at_the_maximum_dimension(dcrf):
    # d = 8, the largest feature dimension of the boundary
    rng = np.random.default_rng(61)
    f = rng.normal(scale=1.0, size=(3000, 8)).astype(np.float32)
    lat = dcrf.dcrf_lattice_build(torch.from_numpy(f).cuda())
    ora = P.Permutohedral(f)
    assert lat.m == ora.m
    Y = rng.uniform(size=(3000, 3)).astype(np.float32)
    out = dcrf.dcrf_filter(lat, torch.from_numpy(Y).cuda()).cpu().numpy()
    assert rel_err(out, ora.filter(Y)) <= 1e-4


@pytest.mark.parametrize("L", [2, 64])
def test_fw_label_counts(dcrf, L):
    p = S.make_problem(32, 24, 4, L, seed=62 + L)
    g = gpu_setup(dcrf, [p], torch)
    Y = g["y0"].clone()
    rec = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 12)
    c = oracle_crf(p)
    y_o, _, rec_o = qp.frank_wolfe(c, p.y0, 12)
    scale = np.abs(rec_o[:, 0]).max()
    assert np.abs(rec[:, 0, 0] - rec_o[:, 0]).max() <= 1e-3 * scale
    np.testing.assert_allclose(Y.cpu().numpy().sum(1), 1.0, atol=1e-5)


def test_fw_single_label_is_fixed(dcrf):
    # L = 1: the simplex is a point, y stays 1 and every step has gap 0
    p = S.make_problem(20, 15, 3, 2, seed=64)
    g = gpu_setup(dcrf, [p], torch)
    phi = g["phi"][:, :1].contiguous()
    Y = torch.ones((p.n_pixels, 1), device="cuda")
    rec = dcrf.dcrf_qp_fw(phi, [g["lb"], g["ls"]], p.weights, Y, 4)
    assert torch.all(Y == 1.0)
    assert np.abs(rec[:, 0, 1]).max() <= 1e-6 * np.abs(rec[:, 0, 0]).max()


def test_fw_batch_with_an_empty_image(dcrf):
    # image 1 of three has no pixels; the others match their single-image runs
    probs = [S.make_problem(30, 20, 4, 5, seed=65), S.make_problem(25, 18, 4, 5, seed=66)]
    g = gpu_setup(dcrf, probs, torch)
    n0, n1 = probs[0].n_pixels, probs[1].n_pixels
    off = [0, n0, n0, n0 + n1]
    lb = dcrf.dcrf_lattice_build(g["fb"], off)
    ls = dcrf.dcrf_lattice_build(g["fs"], off)
    Y = g["y0"].clone()
    rec = dcrf.dcrf_qp_fw(g["phi"], [lb, ls], probs[0].weights, Y, 10)
    assert rec.shape[1] == 3
    assert np.all(rec[:, 1, 0] == 0.0)
    for b, p in ((0, probs[0]), (2, probs[1])):
        c = oracle_crf(p)
        _, _, rec_o = qp.frank_wolfe(c, p.y0, 10)
        scale = np.abs(rec_o[:, 0]).max()
        assert np.abs(rec[:, b, 0] - rec_o[:, 0]).max() <= 1e-3 * scale


def test_fw_benchmark_batch_sampled_images(dcrf):
    # the benchmark's launch configuration (32 x 500x375, FP16 storage, 100
    # iterations, the autotuned pixel kernel, graph replay on a side stream):
    # the first and the last image, replayed along the GPU's decisions, match
    # the oracle element by element
    B, iters = 32, 100
    probs = [S.make_problem(500, 375, 30, 21, seed=i) for i in range(B)]
    g = gpu_setup(dcrf, probs, torch)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        Y = g["y0"].clone()
        rec, trace = dcrf.dcrf_qp_fw_trace(g["phi"], [g["lb"], g["ls"]], probs[0].weights, Y, iters, storage="f16",
                                           stream=s)
    s.synchronize()
    Y, trace = Y.cpu().numpy(), trace.cpu().numpy()
    for b in (0, B - 1):
        s0, s1 = g["off"][b], g["off"][b + 1]
        err = replay_image(probs[b], Y[s0:s1], rec[:, b], trace[:, s0:s1], "f16", iters)
        check_replay(err, f"benchmark batch image {b}")


def test_fw_rejects_y0_off_the_simplex(dcrf):
    # y^0 must lie on the simplex; a row summing to 2 or a negative entry is
    # reported as DCRF_E_INVAL by the call that reads the records
    p = S.make_problem(24, 16, 3, 4, seed=67)
    g = gpu_setup(dcrf, [p], torch)
    for bad in ("sum", "negative"):
        Y = g["y0"].clone()
        if bad == "sum":
            Y[5] *= 2.0
        else:
            Y[7, 0] = -0.25
            Y[7, 1] += 0.25
        with pytest.raises(dcrf.DcrfError) as ei:
            dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 3)
        assert ei.value.status == -1
        with pytest.raises(dcrf.DcrfError):   # the status word keeps the error until it is read
            g["lb"].status()
    # the lattices are still usable afterwards
    Y = g["y0"].clone()
    dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 3)


def test_fw_is_reproducible_bit_for_bit(dcrf):
    # lattices built twice from the same points, solver run on each: the
    # splats sum fixed-point integers, so records and y agree exactly
    p = S.make_problem(160, 120, 12, 21, seed=68)
    out = []
    for _ in range(2):
        g = gpu_setup(dcrf, [p], torch)
        Y = g["y0"].clone()
        rec = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 20, storage="f16")
        out.append((rec, Y.cpu().numpy()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_bounded_wait_runs_out_and_the_context_survives(dcrf):
    # The pixel pass waits for its tile copies with a bounded number of polls.
    # The self-test arms an mbarrier for bytes that nothing sends (no copy in
    # flight): the wait must run out, DCRF_E_TIMEOUT must reach the status
    # word, and the next calls must run normally.
    p = S.make_problem(24, 16, 3, 3, seed=90)
    g = gpu_setup(dcrf, [p], torch)
    dcrf.dcrf_selftest_bounded_wait(g["lb"], 1000, True)
    with pytest.raises(dcrf.DcrfError) as ei:
        g["lb"].status()
    assert ei.value.status == -6
    dcrf.dcrf_selftest_bounded_wait(g["lb"], 1000, False)
    g["lb"].status()
    out = dcrf.dcrf_filter(g["lb"], g["y0"]).cpu().numpy()
    ref = P.Permutohedral(g["fb"].cpu().numpy()).filter(p.y0.astype(np.float64))
    assert rel_err(out, ref) <= 1e-4
    Y = g["y0"].clone()
    rec = dcrf.dcrf_qp_fw(g["phi"], [g["lb"], g["ls"]], p.weights, Y, 5)
    assert np.all(np.isfinite(rec))


def test_check_mode_on_lattice_tables(dcrf):
    # the tables the kernels index with pass the check mode, and host-made
    # faults in them are counted: a corner pointing into another image, a
    # vertex id past the end, a negative weight, weights not summing to one,
    # a blur neighbour past the end
    probs = [S.make_problem(40, 30, 4, 5, seed=91), S.make_problem(20, 10, 3, 5, seed=92)]
    g = gpu_setup(dcrf, probs, torch)
    po = g["off"]
    for lat in (g["lb"], g["ls"]):
        assert dcrf.dcrf_lattice_validate(lat) == 0
        ex = dcrf.dcrf_lattice_export(lat)
        vo = lat.vertex_offsets
        pv, pw, nb = ex["point_vertex"], ex["point_weight"], ex["neighbours"]
        assert dcrf.dcrf_check_lattice_tables(pv, pw, nb, po, vo) == 0

        def bad(pv_=pv, pw_=pw, nb_=nb):
            return dcrf.dcrf_check_lattice_tables(pv_, pw_, nb_, po, vo)

        x = pv.clone(); x[0, 0] = int(vo[1]); assert bad(pv_=x) >= 1           # image 1's vertex for a point of image 0
        x = pv.clone(); x[-1, 1] = int(lat.m); assert bad(pv_=x) >= 1          # past the last vertex
        w = pw.clone(); w[3, 0] = -0.5; w[3, 1] += 0.5; assert bad(pw_=w) >= 1  # negative weight (sum kept)
        w = pw.clone(); w[5, 0] += 0.25; assert bad(pw_=w) >= 1                # weights sum to 1.25
        n2 = nb.clone(); n2[2, 0, 1] = int(lat.m) + 7; assert bad(nb_=n2) >= 1
        with pytest.raises(ValueError):
            dcrf.dcrf_check_lattice_tables(pv.float(), pw, nb, po, vo)
