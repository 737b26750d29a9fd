"""Exact dense-CRF definitions, FP64 (test infrastructure; see package header).

Everything here is the plain definition from Section 3-4 of the paper:

* Eq. 3-4: psi_ab(i,j) = mu(i,j) * sum_m w_m exp(-|f_a^m - f_b^m|^2 / 2).
* Appendix G: the two kernels are a bilateral one on (position, colour) and a
  spatial one on position; with theta scales the features are
  f_bil = (x/theta_alpha, y/theta_alpha, rgb/theta_beta), f_sp = (x, y)/theta_gamma.
* Eq. 6: v'_a = sum_b k(f_a, f_b) v_b, including b = a.
* Eq. 7: Psi = mu (x) (sum_m w_m K_m - (sum_m w_m) I), i.e. exactly the b != a
  pairs of Eq. 1 (the weights are dropped in the printed Eq. 7; reading c1).
* Eq. 11: d_a(i) = sum_{b!=a} sum_j |psi_ab(i,j)| = (sum_j |mu_ij|) * c_a with
  c_a = sum_{b!=a} K_ab, clamped at 0 when K is approximated (reading c16).
* Eq. 10: S_cvx(y) = (phi - d)^T y + y^T (Psi + D) y.
* Eq. 8:  S_QP(y) = phi^T y + y^T Psi y.
* Eq. 1:  E(x) = sum_a phi_a(x_a) + sum_a sum_{b!=a} psi_ab(x_a, x_b).
* Eq. 18: S_LP(y) = phi^T y + sum_a sum_{b!=a} sum_i K_ab |y_a(i) - y_b(i)| / 2.

A "pixel operator" is any object with ``apply(V)`` (= K V, K the N x N mixture
sum including the diagonal), ``apply_T(V)``, ``sum_w`` and ``n``.  The exact one
is :class:`BruteGaussian`; the lattice one lives in ``permutohedral``.
"""
from __future__ import annotations

import numpy as np


def potts(n_labels: int) -> np.ndarray:
    """mu_potts(i, j) = [i != j] (Section 3)."""
    return 1.0 - np.eye(n_labels)


def features(rgb: np.ndarray, theta_alpha: float, theta_beta: float, theta_gamma: float):
    """Bilateral (d=5) and spatial (d=2) features of Appendix G, FP64.

    Pixel a = y*W + x sits at position (x, y).
    """
    h, w, _ = rgb.shape
    yy, xx = np.mgrid[0:h, 0:w]
    x = xx.reshape(-1).astype(np.float64)
    y = yy.reshape(-1).astype(np.float64)
    col = rgb.reshape(-1, 3).astype(np.float64)
    f_bil = np.stack([x / theta_alpha, y / theta_alpha,
                      col[:, 0] / theta_beta, col[:, 1] / theta_beta, col[:, 2] / theta_beta], axis=1)
    f_sp = np.stack([x / theta_gamma, y / theta_gamma], axis=1)
    return f_bil, f_sp


def to_fp32_features(f: np.ndarray) -> np.ndarray:
    """The FP32 features the lattice consumes.

    Each FP64 quotient above is rounded once to FP32; since FP64 carries more
    than 2*24+2 bits this equals the correctly rounded FP32 quotient.
    """
    return np.ascontiguousarray(f.astype(np.float32))


class BruteGaussian:
    """Exact K = sum_m w_m K^(m), K^(m)_ab = exp(-|f_a^m - f_b^m|^2 / 2), O(N^2)."""

    def __init__(self, feats, weights, block_bytes: int = 1 << 26):
        self.feats = [np.asarray(f, dtype=np.float64) for f in feats]
        self.weights = [float(w) for w in weights]
        self.n = self.feats[0].shape[0]
        self.sum_w = float(sum(self.weights))
        self.block_bytes = block_bytes

    def _rows(self, i0, i1):
        k = np.zeros((i1 - i0, self.n))
        for f, w in zip(self.feats, self.weights):
            diff = f[i0:i1, None, :] - f[None, :, :]
            k += w * np.exp(-0.5 * np.sum(diff * diff, axis=2))
        return k

    def dense(self) -> np.ndarray:
        return self._rows(0, self.n)

    def apply(self, v: np.ndarray) -> np.ndarray:
        v = np.asarray(v, dtype=np.float64)
        out = np.zeros_like(v)
        dmax = max(f.shape[1] for f in self.feats)
        step = max(1, self.block_bytes // (8 * self.n * (dmax + 1)))
        for i0 in range(0, self.n, step):
            i1 = min(self.n, i0 + step)
            out[i0:i1] = self._rows(i0, i1) @ v
        return out

    apply_T = apply   # K is symmetric

    def rows(self, idx: np.ndarray) -> np.ndarray:
        """K restricted to the given rows (for sampled checks)."""
        out = np.zeros((len(idx), self.n))
        for f, w in zip(self.feats, self.weights):
            diff = f[idx][:, None, :] - f[None, :, :]
            out += w * np.exp(-0.5 * np.sum(diff * diff, axis=2))
        return out


class DenseCRF:
    """Unaries phi (N x L), label compatibility mu (L x L) and a pixel operator."""

    def __init__(self, unaries: np.ndarray, kernel, mu: np.ndarray | None = None, clamp: bool = True):
        self.phi = np.asarray(unaries, dtype=np.float64)
        self.n, self.L = self.phi.shape
        self.kernel = kernel
        self.mu = potts(self.L) if mu is None else np.asarray(mu, dtype=np.float64)
        ones = np.ones((self.n, 1))
        c = kernel.apply(ones)[:, 0] - kernel.sum_w          # sum_{b != a} K_ab
        self.c_raw = c
        self.c = np.maximum(c, 0.0) if clamp else c
        self.d = np.abs(self.mu).sum(axis=1)[None, :] * self.c[:, None]   # Eq. 11

    # Psi v with Psi = mu (x) (K - sum_w I)   (Eq. 7, reading c1)
    def psi(self, v: np.ndarray) -> np.ndarray:
        x = self.kernel.apply(v) - self.kernel.sum_w * v
        return x @ self.mu.T

    def psi_T(self, v: np.ndarray) -> np.ndarray:
        x = self.kernel.apply_T(v) - self.kernel.sum_w * v
        return x @ self.mu

    def psi_plus_D(self, v: np.ndarray) -> np.ndarray:
        return self.psi(v) + self.d * v

    def psi_plus_D_T(self, v: np.ndarray) -> np.ndarray:
        return self.psi_T(v) + self.d * v

    # objectives
    def s_cvx(self, y: np.ndarray) -> float:
        """Eq. 10."""
        return float(np.sum((self.phi - self.d) * y) + np.sum(y * self.psi_plus_D(y)))

    def s_qp(self, y: np.ndarray) -> float:
        """Eq. 8 (the non-convex QP objective)."""
        return float(np.sum(self.phi * y) + np.sum(y * self.psi(y)))

    def energy(self, labels: np.ndarray) -> float:
        """Eq. 1 at an integer labelling, through the operator: phi + sum mu K (b != a)."""
        y = np.zeros((self.n, self.L))
        y[np.arange(self.n), labels] = 1.0
        return self.s_qp(y)


def energy_pairs(unaries: np.ndarray, k_dense: np.ndarray, mu: np.ndarray, labels: np.ndarray) -> float:
    """Eq. 1 written as the double sum over ordered pairs (pure Python; tiny N only)."""
    n = len(labels)
    e = sum(float(unaries[a, labels[a]]) for a in range(n))
    for a in range(n):
        for b in range(n):
            if b != a:
                e += float(mu[labels[a], labels[b]]) * float(k_dense[a, b])
    return e


def s_lp_pairs(unaries: np.ndarray, k_dense: np.ndarray, y: np.ndarray) -> float:
    """Eq. 18 over ordered pairs with exact K (Potts); O(N^2 L)."""
    y = np.asarray(y, dtype=np.float64)
    pair = 0.0
    for i in range(y.shape[1]):
        diff = np.abs(y[:, i][:, None] - y[:, i][None, :])
        np.fill_diagonal(diff, 0.0)
        pair += float(np.sum(k_dense * diff)) / 2.0
    return float(np.sum(unaries * y)) + pair
