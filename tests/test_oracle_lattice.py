"""Pins of the oracle's permutohedral lattice against geometry and the exact sum."""
import numpy as np
import pytest

from oracle import crf
from oracle import permutohedral as P
from paper_1608_06192_gb300 import synthetic as S


def _feats(d, n, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    return (rng.uniform(-spread, spread, (n, d))).astype(np.float32)


@pytest.mark.parametrize("d", [1, 2, 3, 5])
def test_elevation_is_scaled_isometry_onto_hyperplane(d):
    f = _feats(d, 200, d)
    x = P.elevate(f)
    alpha, _, _ = P.lattice_constants(d)
    assert np.abs(x.sum(axis=1)).max() < 1e-12
    i, j = np.triu_indices(len(f), 1)
    dx = np.sum((x[i] - x[j]) ** 2, axis=1)
    df = np.sum((f[i].astype(np.float64) - f[j]) ** 2, axis=1)
    np.testing.assert_allclose(dx, alpha ** 2 * df, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_enclosing_simplex_contains_point(d):
    f = _feats(d, 500, 10 + d, spread=6.0)
    x = P.elevate(f)
    verts, b, rank = P.enclosing_simplex(x)
    d1 = d + 1
    # barycentric weights are a partition of unity, non-negative, and reproduce x
    assert b.min() > -1e-12
    np.testing.assert_allclose(b.sum(axis=1), 1.0, atol=1e-12)
    rec = np.einsum("nk,nkc->nc", b, verts.astype(np.float64))
    np.testing.assert_allclose(rec, x, atol=1e-9)
    # vertex k is a remainder-k point of the lattice A*_d on the hyperplane
    for k in range(d1):
        assert np.all((verts[:, k, :] - k) % d1 == 0)
        assert np.all(verts[:, k, :].sum(axis=1) == 0)
    # consecutive vertices differ by a canonical simplex edge: one coordinate
    # drops by d, the others rise by 1
    for k in range(d):
        step = verts[:, k + 1, :] - verts[:, k, :]
        assert np.all(np.sort(step, axis=1)[:, 0] == -d)
        assert np.all(np.sort(step, axis=1)[:, 1:] == 1)


def test_special_point_on_lattice_vertex():
    # f = 0 elevates to the origin, a remainder-0 point: all weight on vertex 0
    lat = P.Permutohedral(np.zeros((1, 3), dtype=np.float32))
    np.testing.assert_allclose(lat.bary[0], [1, 0, 0, 0], atol=1e-15)
    assert np.all(lat.point_verts[0, 0] == 0)


def test_neighbours_are_lattice_steps():
    lat = P.Permutohedral(_feats(3, 400, 3, spread=2.0))
    d, d1 = lat.d, lat.d + 1
    full = np.concatenate([lat.vertex_keys, -lat.vertex_keys.sum(1, keepdims=True)], axis=1)
    found = 0
    for j in range(d1):
        w = -np.ones(d1, dtype=np.int64)
        w[j] = d
        for side, sgn in ((0, -1), (1, 1)):
            nb = lat.nbr[:, j, side]
            ok = nb >= 0
            found += ok.sum()
            np.testing.assert_array_equal(full[nb[ok]], full[ok] + sgn * w)
            # an absent neighbour is really absent from the vertex set
            keys = {tuple(r) for r in lat.vertex_keys}
            for v in np.nonzero(~ok)[0][:50]:
                assert tuple((full[v] + sgn * w)[:d]) not in keys
    assert found > 0


@pytest.mark.parametrize("d", [2, 5])
def test_adjoint_identity(d):
    lat = P.Permutohedral(_feats(d, 300, 7, spread=2.0))
    rng = np.random.default_rng(1)
    u, v = rng.normal(size=(300, 3)), rng.normal(size=(300, 3))
    lhs = np.sum(u * lat.filter(v))
    rhs = np.sum(lat.filter_adjoint(u) * v)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_blur_weights_on_complete_row():
    # d = 1: points on a line; the lattice is a 1-D chain and each blur pass is
    # the [1/4, 1/2, 1/4] stencil, so interior vertex values of a constant field stay constant
    f = (np.arange(400, dtype=np.float64) * 0.05).astype(np.float32)[:, None]
    lat = P.Permutohedral(f)
    vl = np.ones(lat.m)
    out = lat.blur(vl.copy())
    inner = np.all(lat.nbr >= 0, axis=(1, 2))
    np.testing.assert_allclose(out[inner & (np.convolve(inner, np.ones(5), "same") == 5)], 1.0, atol=1e-15)


def test_uniform_density_matches_exact_gaussian_sum():
    # dense regular grid (d = 2): the output scale s0 makes the lattice reproduce the
    # exact sum of the unnormalised Gaussian away from the border
    h = 0.25
    g = np.arange(0, 60) * h
    xx, yy = np.meshgrid(g, g)
    f = np.stack([xx.ravel(), yy.ravel()], 1)
    lat = P.Permutohedral(f.astype(np.float32))
    ones = np.ones((len(f), 1))
    approx = lat.filter(ones)[:, 0]
    inner = (np.abs(f[:, 0] - g.mean()) < 2.0) & (np.abs(f[:, 1] - g.mean()) < 2.0)
    exact = crf.BruteGaussian([f], [1.0]).rows(np.nonzero(inner)[0]).sum(axis=1)
    ratio = approx[inner] / exact
    assert abs(ratio.mean() - 1.0) < 0.02


def test_impulse_response_has_unit_variance():
    # the lattice kernel should approximate exp(-|df|^2/2): per-dimension second
    # moment of the impulse response close to 1
    h = 0.2
    g = np.arange(0, 70) * h
    xx, yy = np.meshgrid(g, g)
    f = np.stack([xx.ravel(), yy.ravel()], 1)
    lat = P.Permutohedral(f.astype(np.float32))
    c = np.argmin(np.sum((f - g.mean()) ** 2, 1))
    e = np.zeros((len(f), 1))
    e[c] = 1.0
    r = lat.filter(e)[:, 0]
    var = np.sum(r * np.sum((f - f[c]) ** 2, 1)) / np.sum(r) / 2.0
    assert 0.85 < var < 1.15


def test_partitioned_filter_is_block_diagonal_and_reduces_to_full():
    lat = P.Permutohedral(_feats(2, 200, 5, spread=2.0))
    rng = np.random.default_rng(2)
    v = rng.normal(size=200)
    np.testing.assert_allclose(lat.filter_partitioned(v, np.zeros(200, dtype=np.int64)), lat.filter(v),
                               rtol=1e-12, atol=1e-12)
    part = rng.integers(0, 3, 200)
    for p in range(3):
        out = lat.filter_partitioned(np.where(part == p, v, 0.0), part)
        assert np.all(out[part != p] == 0.0)


def test_lattice_tracks_brute_force_on_small_image():
    p = S.qp_small()
    fb, fs = crf.features(p.rgb, *p.thetas)
    for f, min_cos in ((fb, 0.98), (fs, 0.99)):
        lat = P.Permutohedral(crf.to_fp32_features(f))
        rng = np.random.default_rng(0)
        v = rng.uniform(size=(lat.n, 2))
        kv = crf.BruteGaussian([f], [1.0]).apply(v)
        lv = lat.filter(v)
        cos = np.sum(kv * lv) / np.linalg.norm(kv) / np.linalg.norm(lv)
        assert cos > min_cos


@pytest.mark.parametrize("d", [2, 5])
def test_lattice_operator_is_slightly_asymmetric_and_its_adjoint_is_the_transpose(d):
    # reading c4: the per-axis blurs are symmetric but do not commute where
    # vertices are missing, so K~ = S^T B_d ... B_0 S is not symmetric; the
    # reverse-order blur gives exactly K~^T
    lat = P.Permutohedral(_feats(d, 120, 20 + d, spread=2.0))
    eye = np.eye(lat.n)
    K = lat.filter(eye)
    KT = lat.filter_adjoint(eye)
    np.testing.assert_allclose(KT, K.T, rtol=0, atol=1e-12 * np.abs(K).max())
    asym = np.linalg.norm(K - K.T) / np.linalg.norm(K)
    assert asym > 1e-9
