"""GPU parity of features, lattice build, filter and adjoint against the oracle."""
import numpy as np
import pytest

from helpers import gpu_setup, oracle_features, rel_err
from oracle import crf
from oracle import permutohedral as P
from paper_1608_06192_gb300 import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(64, 48, 5, 5), (37, 23, 4, 3), (320, 213, 30, 21)]


def _keyset(keys):
    return {tuple(r) for r in np.asarray(keys).tolist()}


@pytest.mark.parametrize("w,h,regions,L", SHAPES)
def test_features_bit_exact(dcrf, w, h, regions, L):
    p = S.make_problem(w, h, regions, L, seed=3)
    g = gpu_setup(dcrf, [p], torch)
    fb, fs = oracle_features(p)
    np.testing.assert_array_equal(g["fb"].cpu().numpy(), fb)
    np.testing.assert_array_equal(g["fs"].cpu().numpy(), fs)


@pytest.mark.parametrize("w,h,regions,L", SHAPES)
def test_lattice_structure_identical(dcrf, w, h, regions, L):
    p = S.make_problem(w, h, regions, L, seed=4)
    g = gpu_setup(dcrf, [p], torch)
    for key, f in (("lb", g["fb"]), ("ls", g["fs"])):
        lat = g[key]
        ora = P.Permutohedral(f.cpu().numpy())
        ex = dcrf.dcrf_lattice_export(lat)
        keys = ex["keys"].cpu().numpy()
        assert lat.m == ora.m
        assert _keyset(keys) == _keyset(ora.vertex_keys)
        # every point's corners: same vertex keys, same weights
        pv = ex["point_vertex"].cpu().numpy()
        got = keys[pv]                                     # [n, d+1, d]
        np.testing.assert_array_equal(got, ora.point_verts[:, :, :lat.d])
        np.testing.assert_allclose(ex["point_weight"].cpu().numpy(), ora.bary, atol=2e-7)
        # neighbour structure, compared through keys
        nb = ex["neighbours"].cpu().numpy()
        order = {k: i for i, k in enumerate(map(tuple, ora.vertex_keys.tolist()))}
        remap = np.array([order[tuple(k)] for k in keys.tolist()])
        exp = ora.nbr[remap]
        got_nb = np.where(nb >= 0, remap[np.maximum(nb, 0)], -1)
        np.testing.assert_array_equal(got_nb, exp)


def _filter_case(dcrf, problems, L, storage, tol, adjoint=False):
    g = gpu_setup(dcrf, problems, torch)
    rng = np.random.default_rng(11)
    n = int(g["off"][-1])
    Y = rng.uniform(0.0, 1.0, (n, L)).astype(np.float32)
    Yd = torch.from_numpy(Y).cuda()
    for key, fkey in (("lb", "fb"), ("ls", "fs")):
        fn = dcrf.dcrf_filter_adjoint if adjoint else dcrf.dcrf_filter
        out = fn(g[key], Yd, storage=storage).cpu().numpy()
        for b in range(len(problems)):
            s, e = g["off"][b], g["off"][b + 1]
            ora = P.Permutohedral(g[fkey][s:e].cpu().numpy())
            ref = ora.filter_adjoint(Y[s:e]) if adjoint else ora.filter(Y[s:e])
            assert rel_err(out[s:e], ref) <= tol, (key, b)


@pytest.mark.parametrize("w,h,regions,L", SHAPES)
def test_filter_fp32(dcrf, w, h, regions, L):
    _filter_case(dcrf, [S.make_problem(w, h, regions, L, seed=5)], L, "f32", 1e-4)


@pytest.mark.parametrize("w,h,regions,L", SHAPES)
def test_filter_fp16_storage(dcrf, w, h, regions, L):
    _filter_case(dcrf, [S.make_problem(w, h, regions, L, seed=6)], L, "f16", 2e-3)


def test_filter_adjoint_fp32(dcrf):
    _filter_case(dcrf, [S.make_problem(96, 64, 8, 7, seed=7)], 7, "f32", 1e-4, adjoint=True)


def test_filter_batch_of_uneven_images(dcrf):
    probs = [S.make_problem(w, h, 6, 6, seed=20 + i) for i, (w, h) in enumerate([(50, 31), (1, 1), (17, 64)])]
    _filter_case(dcrf, probs, 6, "f32", 1e-4)


def test_filter_headline_size(dcrf):
    _filter_case(dcrf, [S.voc_shaped()], 21, "f32", 1e-4)


def test_adjoint_identity_on_device(dcrf):
    p = S.make_problem(80, 60, 6, 4, seed=8)
    g = gpu_setup(dcrf, [p], torch)
    rng = np.random.default_rng(0)
    u = torch.from_numpy(rng.normal(size=(p.n_pixels, 4)).astype(np.float32)).cuda()
    v = torch.from_numpy(rng.normal(size=(p.n_pixels, 4)).astype(np.float32)).cuda()
    for key in ("lb", "ls"):
        lhs = float(torch.sum(u.double() * dcrf.dcrf_filter(g[key], v).double()))
        rhs = float(torch.sum(dcrf.dcrf_filter_adjoint(g[key], u).double() * v.double()))
        assert abs(lhs - rhs) <= 1e-4 * max(1.0, abs(lhs))


def test_empty_image_in_batch(dcrf):
    f = torch.zeros((5, 2), dtype=torch.float32, device="cuda")
    f[:, 0] = torch.arange(5, dtype=torch.float32, device="cuda")
    lat = dcrf.dcrf_lattice_build(f, [0, 3, 3, 5])
    assert lat.batch == 3
    assert lat.vertex_offsets[1] == lat.vertex_offsets[2]
    out = dcrf.dcrf_filter(lat, torch.ones((5, 1), device="cuda")).cpu().numpy()[:, 0]
    ref = np.concatenate([P.Permutohedral(f[:3].cpu().numpy()).filter(np.ones(3)),
                          P.Permutohedral(f[3:].cpu().numpy()).filter(np.ones(2))])
    assert rel_err(out, ref) < 1e-5


def test_key_range_and_nonfinite_are_reported(dcrf):
    big = torch.full((4, 5), 1.0e5, dtype=torch.float32, device="cuda")
    big[1:, 0] = torch.tensor([2.0e5, 3.0e5, 4.0e5], device="cuda")
    with pytest.raises(dcrf.DcrfError) as e:
        dcrf.dcrf_lattice_build(big)
    assert e.value.status == -5
    bad = torch.zeros((3, 2), dtype=torch.float32, device="cuda")
    bad[1, 1] = float("nan")
    with pytest.raises(dcrf.DcrfError) as e:
        dcrf.dcrf_lattice_build(bad)
    assert e.value.status == -7
    # the context stays usable afterwards
    ok = dcrf.dcrf_lattice_build(torch.zeros((3, 2), dtype=torch.float32, device="cuda"))
    assert ok.m >= 1


def test_invalid_arguments_rejected(dcrf):
    f = torch.zeros((3, 9), dtype=torch.float32, device="cuda")
    with pytest.raises(dcrf.DcrfError):
        dcrf.dcrf_lattice_build(f)                       # d > 8
    lat = dcrf.dcrf_lattice_build(torch.zeros((3, 2), dtype=torch.float32, device="cuda"))
    with pytest.raises(dcrf.DcrfError):
        dcrf.dcrf_filter(lat, torch.zeros((3, 65), device="cuda"))   # L > 64


def test_table_full_is_reported(dcrf, monkeypatch):
    # a table segment smaller than the vertex count: bounded probing gives up
    # and the build returns DCRF_E_TABLE_FULL; the context stays usable
    p = S.make_problem(40, 30, 5, 4, seed=14)
    fb, fs = oracle_features(p)
    f = torch.from_numpy(fs).cuda()
    monkeypatch.setenv("DCRF_TABLE_SLOTS", "64")
    with pytest.raises(dcrf.DcrfError) as e:
        dcrf.dcrf_lattice_build(f)
    assert e.value.status == -4
    monkeypatch.delenv("DCRF_TABLE_SLOTS")
    assert dcrf.dcrf_lattice_build(f).m > 64
