"""Seeded synthetic inputs shaped like the paper's segmentation workloads.

The paper evaluates on PASCAL VOC 2010 (500x375 images, 21 labels, Section 7)
and Middlebury stereo; neither dataset nor the trained unaries are available,
so every workload here is synthetic:

* an RGB image made of ``regions`` Voronoi cells (seeds uniform in the image,
  ties to the lowest seed index), each with a colour drawn from U[0,255]^3,
  plus N(0, noise^2) per channel and pixel, not clipped;
* region r carries label ``r mod L``;
* unaries ``phi = -log softmax(3 * onehot(label) + N(0,1))`` per pixel;
* the Frank-Wolfe start point ``y0 = softmax(-phi)`` per pixel;
* LP inputs: ``y ~ Dirichlet(0.5 * 1_L)`` per pixel.

All draws come from numpy's PCG64 generator with the given seed.  This module
only produces inputs: it holds none of the CRF arithmetic, and both the CUDA
path and the CPU oracle take its arrays as given.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Kernel parameters of the experiments (Appendix G, in the theta form of Eq. 4).
THETA_ALPHA = 80.0   # bilateral kernel, position scale
THETA_BETA = 13.0    # bilateral kernel, colour scale
THETA_GAMMA = 3.0    # spatial kernel, position scale
W_BILATERAL = 10.0
W_SPATIAL = 3.0


@dataclass
class Problem:
    """One synthetic dense-CRF instance (pixel order: row-major, a = y*W + x)."""
    width: int
    height: int
    n_labels: int
    rgb: np.ndarray          # (H, W, 3) float32
    region: np.ndarray       # (H, W) int32
    unaries: np.ndarray      # (N, L) float32
    y0: np.ndarray           # (N, L) float32, rows on the simplex
    seed: int
    weights: tuple = (W_BILATERAL, W_SPATIAL)
    thetas: tuple = (THETA_ALPHA, THETA_BETA, THETA_GAMMA)
    extra: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


def voronoi_image(width: int, height: int, regions: int, rng: np.random.Generator,
                  noise_std: float = 10.0):
    sx = rng.uniform(0.0, width, regions)
    sy = rng.uniform(0.0, height, regions)
    colours = rng.uniform(0.0, 255.0, (regions, 3))
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    best = np.full((height, width), np.inf)
    region = np.zeros((height, width), dtype=np.int32)
    for r in range(regions):                      # strict < keeps the lowest index on ties
        d2 = (xx - sx[r]) ** 2 + (yy - sy[r]) ** 2
        closer = d2 < best
        best[closer] = d2[closer]
        region[closer] = r
    rgb = colours[region] + rng.normal(0.0, noise_std, (height, width, 3))
    return rgb.astype(np.float32), region


def make_problem(width: int, height: int, regions: int, n_labels: int, seed: int,
                 noise_std: float = 10.0) -> Problem:
    rng = np.random.default_rng(seed)
    rgb, region = voronoi_image(width, height, regions, rng, noise_std)
    label = (region.reshape(-1) % n_labels).astype(np.int64)
    n = width * height
    logits = rng.normal(0.0, 1.0, (n, n_labels))
    logits[np.arange(n), label] += 3.0
    z = logits - logits.max(axis=1, keepdims=True)
    lse = np.log(np.exp(z).sum(axis=1, keepdims=True))
    log_sm = z - lse
    unaries = (-log_sm).astype(np.float32)
    y0 = np.exp(log_sm)
    y0 /= y0.sum(axis=1, keepdims=True)
    return Problem(width, height, n_labels, rgb, region, unaries,
                   y0.astype(np.float32), seed)


def dirichlet_labels(n: int, n_labels: int, seed: int, concentration: float = 0.5) -> np.ndarray:
    rng = np.random.default_rng(seed)
    y = rng.dirichlet(np.full(n_labels, concentration), size=n)
    y /= y.sum(axis=1, keepdims=True)
    return y.astype(np.float32)


def kt_phases(n_labels: int, count: int, seed: int):
    """Random draws of the Kleinberg-Tardos rounding: `count` labels uniform
    in [0, n_labels) (int32) and thresholds uniform in [0, 1) (float32)."""
    rng = np.random.default_rng(seed)
    return (rng.integers(0, n_labels, size=count).astype(np.int32),
            rng.random(count, dtype=np.float32))


def batch_sizes(count: int, seed: int, w_range=(240, 500), h_range=(160, 500)):
    """Image sizes W ~ U[240,500], H ~ U[160,500] (integers, inclusive)."""
    rng = np.random.default_rng(seed)
    ws = rng.integers(w_range[0], w_range[1] + 1, count)
    hs = rng.integers(h_range[0], h_range[1] + 1, count)
    return [(int(w), int(h)) for w, h in zip(ws, hs)]


def make_batch(count: int, seed: int, n_labels: int = 21, regions: int = 30,
               sizes=None) -> list[Problem]:
    if sizes is None:
        sizes = batch_sizes(count, seed)
    return [make_problem(w, h, regions, n_labels, seed * 1000 + k)
            for k, (w, h) in enumerate(sizes)]


def crop(p: Problem, width: int, height: int, x0: int = 0, y0: int = 0) -> Problem:
    """A window of a problem (used for the small finite-difference cases)."""
    rgb = p.rgb[y0:y0 + height, x0:x0 + width].copy()
    region = p.region[y0:y0 + height, x0:x0 + width].copy()
    idx = ((np.arange(height)[:, None] + y0) * p.width + (np.arange(width)[None, :] + x0)).reshape(-1)
    return Problem(width, height, p.n_labels, rgb, region, p.unaries[idx].copy(),
                   p.y0[idx].copy(), p.seed, p.weights, p.thetas)


def hst_tree(n_labels: int, group: int = 4):
    """A synthetic three-level r-HST (r = 2) over the labels, given as the
    subtrees below the root: two halves (edge length 4), groups of up to
    `group` consecutive labels inside each half (length 2, groups of one
    label omitted) and the single labels (length 1).  Returns the 0/1 matrix
    [subtrees][labels] of the label sets and the edge lengths."""
    halves = [list(range(0, n_labels // 2)), list(range(n_labels // 2, n_labels))]
    rows, lengths = [], []

    def add(labels, length):
        m = np.zeros(n_labels)
        m[labels] = 1.0
        rows.append(m)
        lengths.append(length)

    for h in halves:
        if len(h) > 1:
            add(h, 4.0)
        for s in range(0, len(h), group):
            if len(h[s:s + group]) > 1:
                add(h[s:s + group], 2.0)
    for i in range(n_labels):
        add([i], 1.0)
    return np.array(rows), np.array(lengths)

# The five workloads, by what they are.
def qp_small():        # 64x48, 5 regions, L=5, seed 0
    return make_problem(64, 48, 5, 5, 0)


def qp_cccp_medium():  # 320x213, 30 regions, L=21
    return make_problem(320, 213, 30, 21, 0)


def voc_shaped():      # 500x375, 30 regions, L=21
    return make_problem(500, 375, 30, 21, 0)
