"""Permutohedral-lattice Gaussian filter, FP64 (test infrastructure).

The paper computes sum_b k(f_a, f_b) v_b (Eq. 6) approximately in O(N) with the
filter of Adams et al. that it cites (Section 3 and Appendix A), WITHOUT the
per-pixel normalisation that Kraehenbuehl and Koltun add (Appendix A).  The
paper only cites that method, so the lattice is written here from its
geometry; the same written conventions are implemented independently by the
CUDA path:

1. Scale: c_j = f_j * alpha / sqrt((j+1)(j+2)), j = 0..d-1, with
   alpha = (d+1) sqrt(2/3).  The d+1 axis blurs with weights [1/4, 1/2, 1/4]
   along the lattice vectors w_j = (d+1) e_j - 1 add up to the covariance
   (d+1)^2/2 * P_H (P_H the projector onto the hyperplane H_d), i.e. 3/4 of a
   unit variance in feature units; the remaining 1/4 is the smoothing of the
   linear splat and slice (exact for d = 1).
2. Elevation onto H_d = {x in R^{d+1} : sum x = 0} with the Helmert basis
   u_j = (1,...,1, -j, 0,...,0)/sqrt(j(j+1)), an isometry:
   running sum sm = 0; for i = d..1: x_i = sm - i*c_{i-1}; sm += c_{i-1};
   x_0 = sm.  Every operation is one IEEE FP64 rounding, in this order.
3. Nearest remainder-0 point: m_i = rint(x_i / (d+1)) (ties to even),
   delta_i = x_i - (d+1) m_i; rank_i = #{j: delta_j > delta_i} +
   #{j < i: delta_j == delta_i}; with s = sum m_i, if s > 0 the s coordinates
   of largest rank get m_i -= 1 (rank_i -= d+1-s, others rank += s); if s < 0
   the -s coordinates of smallest rank get m_i += 1 (rank_i += d+1+s, others
   rank += s).  delta is then recomputed from the corrected m.
4. Enclosing simplex: with y_p the delta of rank p, vertex k (k = 0..d) has
   coordinates (d+1) m_i + k - (d+1)[rank_i >= d+1-k] and barycentric weight
   b_k = (y_{d-k} - y_{d+1-k})/(d+1) for k >= 1, b_0 = 1 - (y_0 - y_d)/(d+1).
5. The lattice holds exactly the vertices touched by some point.  Splat:
   V[v] = sum of b_k(a) * value_a.  Blur: for j = 0..d in order,
   V[v] <- V[v]/2 + (V[v + w_j] + V[v - w_j])/4, a Jacobi pass, absent
   neighbours read as 0 and are never created.  Slice: out_a =
   s0 * sum_k b_k(a) V[vertex_k(a)].
6. Output scale s0 = (2 pi)^{d/2} alpha^d / (d+1)^{d-1/2}: the lattice A*_d
   above has (d+1)^{d-1/2} volume per vertex, so this makes a uniform point
   cloud give the exact sum of the unnormalised Gaussian.

The operator is K~ = s0 S^T B_d ... B_0 S (S the splat matrix); each B_j is
symmetric, so its adjoint is the same chain with the blur axes reversed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def lattice_constants(d: int):
    d1 = d + 1
    alpha = float(d1) * np.sqrt(2.0 / 3.0)
    sig = np.array([alpha / np.sqrt(float((j + 1) * (j + 2))) for j in range(d)])
    s0 = (2.0 * np.pi) ** (d / 2.0) * alpha ** d / float(d1) ** (d - 0.5)
    return alpha, sig, s0


def elevate(f32: np.ndarray) -> np.ndarray:
    """Step 1-2: scaled, elevated coordinates x (N, d+1), FP64."""
    n, d = f32.shape
    _, sig, _ = lattice_constants(d)
    c = np.asarray(f32, dtype=np.float64) * sig[None, :]
    x = np.zeros((n, d + 1))
    sm = np.zeros(n)
    for i in range(d, 0, -1):
        x[:, i] = sm - float(i) * c[:, i - 1]
        sm = sm + c[:, i - 1]
    x[:, 0] = sm
    return x


def enclosing_simplex(x: np.ndarray):
    """Steps 3-4: vertex coordinates (N, d+1, d+1) int64 and weights (N, d+1)."""
    n, d1 = x.shape
    d = d1 - 1
    m = np.rint(x / float(d1))
    delta = x - float(d1) * m
    gt = delta[:, None, :] > delta[:, :, None]          # [a, i, j] = delta_j > delta_i
    eq = delta[:, None, :] == delta[:, :, None]
    earlier = np.tril(np.ones((d1, d1), dtype=bool), -1)  # [i, j] = j < i
    rank = gt.sum(axis=2) + (eq & earlier[None]).sum(axis=2)
    s = m.sum(axis=1).astype(np.int64)
    mi = m.astype(np.int64)
    sc = s[:, None]
    pos = (sc > 0) & (rank >= d1 - sc)          # s > 0: the s largest ranks move down a level
    neg = (sc < 0) & (rank < -sc)               # s < 0: the -s smallest ranks move up a level
    mi = mi - pos + neg
    rank = np.where(pos, rank - (d1 - sc), np.where(neg, rank + d1 + sc, rank + sc))
    delta = x - float(d1) * mi.astype(np.float64)
    ys = np.zeros_like(delta)
    np.put_along_axis(ys, rank, delta, axis=1)
    b = np.zeros((n, d1))
    for k in range(1, d1):
        b[:, k] = (ys[:, d - k] - ys[:, d + 1 - k]) / float(d1)
    b[:, 0] = 1.0 - (ys[:, 0] - ys[:, d]) / float(d1)
    k = np.arange(d1)
    verts = (d1 * mi[:, None, :] + k[None, :, None]
             - d1 * (rank[:, None, :] >= (d1 - k)[None, :, None]).astype(np.int64))
    return verts, b, rank


class _Codec:
    """Maps integer key rows (first d coordinates) to sortable int64 codes."""

    def __init__(self, rows: np.ndarray, margin: int):
        self.lo = int(rows.min()) - margin
        self.base = int(rows.max()) - self.lo + margin + 1
        if self.base ** rows.shape[1] >= 2 ** 62:
            raise ValueError("lattice key range too large for the oracle codec")

    def encode(self, rows: np.ndarray) -> np.ndarray:
        code = np.zeros(rows.shape[0], dtype=np.int64)
        for i in range(rows.shape[1] - 1, -1, -1):
            code = code * self.base + (rows[:, i] - self.lo)
        return code


class Permutohedral:
    """The lattice of one Gaussian kernel over N points with d features."""

    def __init__(self, features_f32: np.ndarray):
        f = np.asarray(features_f32)
        if f.dtype != np.float32:
            raise TypeError("the lattice takes FP32 features")
        self.n, self.d = f.shape
        d, d1 = self.d, self.d + 1
        self.alpha, _, self.s0 = lattice_constants(d)
        self.x = elevate(f)
        verts, self.bary, self.rank = enclosing_simplex(self.x)
        self.point_verts = verts                          # (N, d+1, d+1)
        rows = verts[:, :, :d].reshape(-1, d)
        self._codec = _Codec(rows, margin=d1 + 1)
        codes = self._codec.encode(rows)
        self.codes, inv = np.unique(codes, return_inverse=True)
        self.m = len(self.codes)
        self.vid = inv.reshape(self.n, d1)                # vertex id of (a, k)
        first = np.zeros(self.m, dtype=np.int64)
        first[inv] = np.arange(len(inv))
        self.vertex_keys = rows[first]                    # (M, d), sorted by code
        full = np.concatenate([self.vertex_keys, -self.vertex_keys.sum(axis=1, keepdims=True)], axis=1)
        self.nbr = np.full((self.m, d1, 2), -1, dtype=np.int64)
        for j in range(d1):
            w = -np.ones(d1, dtype=np.int64)
            w[j] = d
            for side, sgn in ((0, -1), (1, 1)):
                nb = full + sgn * w[None, :]
                c = self._codec.encode(nb[:, :d])
                pos = np.searchsorted(self.codes, c)
                pos = np.minimum(pos, self.m - 1)
                hit = self.codes[pos] == c
                self.nbr[hit, j, side] = pos[hit]
        self.S = sp.csr_matrix((self.bary.reshape(-1), (self.vid.reshape(-1), np.repeat(np.arange(self.n), d1))),
                               shape=(self.m, self.n))

    # pieces
    def splat(self, v):
        return self.S @ np.asarray(v, dtype=np.float64)

    def blur(self, vl, reverse: bool = False, nbr=None):
        nbr = self.nbr if nbr is None else nbr
        axes = range(self.d, -1, -1) if reverse else range(self.d + 1)
        for j in axes:
            out = 0.5 * vl
            for side in (0, 1):
                idx = nbr[:, j, side]
                ok = idx >= 0
                out[ok] += 0.25 * vl[idx[ok]]
            vl = out
        return vl

    def slice(self, vl):
        return self.s0 * (self.S.T @ vl)

    def filter(self, v):
        """K~ v (Eq. 6 through the lattice), v of shape (N,) or (N, C)."""
        return self.slice(self.blur(self.splat(v)))

    def filter_adjoint(self, v):
        """K~^T v: the blur axes in reverse order."""
        return self.slice(self.blur(self.splat(v), reverse=True))

    def filter_partitioned(self, v, part):
        """Sum over groups g of K~^(g) v restricted to group g.

        K~^(g) is the lattice built over the points of group g only: the same
        vertices and weights as the full lattice, restricted to the vertices
        those points touch (the sub-problems of the LP divide-and-conquer).
        """
        part = np.asarray(part, dtype=np.int64)
        d1 = self.d + 1
        tag = part[:, None] * self.m + self.vid
        tcodes, tinv = np.unique(tag.reshape(-1), return_inverse=True)
        mt = len(tcodes)
        tpart = tcodes // self.m
        tvid = tcodes % self.m
        tnbr = np.full((mt, d1, 2), -1, dtype=np.int64)
        for j in range(d1):
            for side in (0, 1):
                u = self.nbr[tvid, j, side]
                ok = u >= 0
                c = tpart[ok] * self.m + u[ok]
                pos = np.minimum(np.searchsorted(tcodes, c), mt - 1)
                hit = tcodes[pos] == c
                sel = np.nonzero(ok)[0][hit]
                tnbr[sel, j, side] = pos[hit]
        S = sp.csr_matrix((self.bary.reshape(-1), (tinv, np.repeat(np.arange(self.n), d1))), shape=(mt, self.n))
        vl = S @ np.asarray(v, dtype=np.float64)
        vl = self.blur(vl, nbr=tnbr)
        return self.s0 * (S.T @ vl)


class LatticeGaussian:
    """K~ = sum_m w_m K~^(m): the pixel operator built from one lattice per kernel."""

    def __init__(self, feats_f32, weights):
        self.lattices = [Permutohedral(f) for f in feats_f32]
        self.weights = [float(w) for w in weights]
        self.n = self.lattices[0].n
        self.sum_w = float(sum(self.weights))

    def apply(self, v):
        return sum(w * lat.filter(v) for w, lat in zip(self.weights, self.lattices))

    def apply_T(self, v):
        return sum(w * lat.filter_adjoint(v) for w, lat in zip(self.weights, self.lattices))

    def apply_partitioned(self, v, part):
        return sum(w * lat.filter_partitioned(v, part) for w, lat in zip(self.weights, self.lattices))
