"""LP relaxation: subgradient, divide and conquer, projection (test infrastructure).

Section 6 of the paper, Potts model, FP64:

* Eq. 18: S_LP(y) = phi^T y + sum_a sum_{b!=a} sum_i K_ab |y_a(i) - y_b(i)| / 2.
* Eq. 19 / Appendix D: with the pixels of label i sorted by descending y(i)
  the pairwise term is linear in y; ties are broken by ascending pixel index
  (reading c12) -- any tie order gives a valid subgradient.
* Eq. 20: dS/dy_c(k) = phi_c(k) + sum_{a after c} K_ac - sum_{a before c} K_ac.
* Appendix E: the upper sums U_c = sum_{b after c} K_cb by divide and conquer
  with power-of-two splits of the sorted order (reading c11): with B =
  ceil(log2 N) levels and r(a) the 0-based rank, at level l the node of a is
  r >> (B - l) and a is in the right child when bit B - l - 1 of r is set; the
  left-child points receive the filter of the right child's indicator, taken
  over the node's own points only (reading c13).
* The lower sums follow from L_c = c_c - U_c with c_c = sum_{b != c} K_cb (the
  same clamped c as Eq. 11), so G = phi + 2U - c.
* S_LP(y) = <y, G(y)> since the pairwise term is positively 1-homogeneous.
* Algorithm 3: y <- Proj_M(y - beta_t G), beta_t = beta0 / (1 + t), with
  beta0 = 0.1 / max |G0_a(i) - mean_i G0_a(i)| by default (reading c14); the
  projection onto the simplex (Condat's problem) is computed here by the
  sort-based closed form, which gives the same unique point.
* Section 5 (end): the LP point is turned into a labelling by the randomised
  rounding of Kleinberg and Tardos (uniform metric): repeatedly draw a label i
  uniformly and a threshold alpha uniformly in [0, 1), and give label i to
  every still unlabelled pixel a with y_a(i) > alpha.  The draws are inputs
  here (phase_labels, phase_thresholds); the comparison is taken in FP32, the
  precision y is stored in (reading: the decision of an integer in the
  kernel's precision).  Pixel a gets label i with probability y_a(i), and two
  pixels are separated with probability at most 2d/(1+d), d = |y_a - y_b|_1 / 2,
  which is at most twice their LP distance: the factor 2 for the Potts model.
"""
from __future__ import annotations

import math

import numpy as np


def label_rank(v: np.ndarray) -> np.ndarray:
    """0-based rank of every pixel in descending order of v, ties by index."""
    idx = np.arange(len(v))
    order = np.lexsort((idx, -np.asarray(v, dtype=np.float64)))
    rank = np.empty(len(v), dtype=np.int64)
    rank[order] = np.arange(len(v))
    return rank


def subgradient_pairs(phi: np.ndarray, k_dense: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Eq. 20 by explicit sums over the sorted order (exact K, O(N^2 L))."""
    G = np.array(phi, dtype=np.float64)
    for i in range(y.shape[1]):
        r = label_rank(y[:, i])
        after = r[None, :] > r[:, None]      # [c, b]: b comes after c
        before = r[None, :] < r[:, None]
        G[:, i] += np.sum(k_dense * after, axis=1) - np.sum(k_dense * before, axis=1)
    return G


def levels(n: int) -> int:
    return int(math.ceil(math.log2(n))) if n > 1 else 0


def upper_sums_dc(rank: np.ndarray, filter_partitioned) -> np.ndarray:
    """U_a = sum_{b after a} K_ab by the divide and conquer of Appendix E."""
    n = len(rank)
    nb = levels(n)
    U = np.zeros(n)
    for lev in range(nb):
        node = rank >> (nb - lev)
        bit = (rank >> (nb - lev - 1)) & 1
        out = filter_partitioned(bit.astype(np.float64), node)
        U += np.where(bit == 0, out, 0.0)
    return U


def brute_partitioned(k_dense: np.ndarray):
    """v -> sum_b K_ab v_b over b in the same group as a (exact sub-matrices)."""
    def f(v, part):
        same = part[:, None] == part[None, :]
        return (k_dense * same) @ v
    return f


def subgradient_dc(phi: np.ndarray, y: np.ndarray, c: np.ndarray, filter_partitioned) -> np.ndarray:
    """G = phi + 2U - c with U from the divide and conquer, per label."""
    G = np.array(phi, dtype=np.float64)
    for i in range(y.shape[1]):
        U = upper_sums_dc(label_rank(y[:, i]), filter_partitioned)
        G[:, i] += 2.0 * U - c
    return G


def s_lp_from_g(y: np.ndarray, G: np.ndarray) -> float:
    return float(np.sum(np.asarray(y, dtype=np.float64) * G))


def project_simplex(V: np.ndarray) -> np.ndarray:
    """Euclidean projection of each row onto {y >= 0, sum y = 1} (closed form)."""
    V = np.asarray(V, dtype=np.float64)
    n, L = V.shape
    u = -np.sort(-V, axis=1)
    css = np.cumsum(u, axis=1)
    j = np.arange(1, L + 1)[None, :]
    cond = u - (css - 1.0) / j > 0
    rho = L - np.argmax(cond[:, ::-1], axis=1)          # largest j with cond true
    tau = (css[np.arange(n), rho - 1] - 1.0) / rho
    return np.maximum(V - tau[:, None], 0.0)


def default_beta0(G0: np.ndarray) -> float:
    dev = np.abs(G0 - G0.mean(axis=1, keepdims=True)).max()
    return 0.1 / dev if dev > 0 else 0.1


def lp_solve(phi, y0, c, filter_partitioned, steps: int, beta0: float | None = None, members=None, c_t=None):
    """Algorithm 3 (Potts) or Appendix F's algorithm (tree metric, when `members`
    and `c_t` are given); returns (best y, energies[steps+1] of every iterate)."""
    y = np.array(y0, dtype=np.float64)

    def subgrad(y):
        if members is None:
            return subgradient_dc(phi, y, c, filter_partitioned)
        return subgradient_tree_dc(phi, y, c, filter_partitioned, members, c_t)

    G = subgrad(y)
    beta0 = default_beta0(G) if beta0 is None or beta0 <= 0 else beta0
    energies = [s_lp_from_g(y, G)]
    best_y, best_e = y.copy(), energies[0]
    for t in range(steps):
        y = project_simplex(y - (beta0 / (1.0 + t)) * G)
        G = subgrad(y)
        e = s_lp_from_g(y, G)
        energies.append(e)
        if e < best_e:
            best_e, best_y = e, y.copy()
    return best_y, np.array(energies)


# ---------------------------------------------------------------------------
# r-HST (tree) metrics, Appendix F: the LP of Eq. (rHST-LP) over the subtrees
# T of a given tree, with y_a(T) = sum_{i in L(T)} y_a(i) and weights c_T:
#   S(y) = phi^T y + sum_T c_T sum_{a, b != a} K_ab |y_a(T) - y_b(T)| / 2.
# Per subtree the pixels are sorted by descending y(T) (ties by index), and
#   dS/dy_c(k) = phi_c(k) + sum_{T containing k} c_T (sum_{a after c} K_ac
#                                                    - sum_{a before c} K_ac),
# the Potts model being the tree whose subtrees are the single labels with
# c_T = 1.  `members` is the 0/1 matrix [subtrees][labels] of L(T).


def subtree_values(y: np.ndarray, members: np.ndarray) -> np.ndarray:
    """y_a(T) for every pixel and subtree: [N][n_subtrees]."""
    return np.asarray(y, dtype=np.float64) @ np.asarray(members, dtype=np.float64).T


def subgradient_tree_pairs(phi, k_dense, y, members, c_t):
    """The Appendix F subgradient by explicit sums over each subtree's order (exact K)."""
    Z = subtree_values(y, members)
    G = np.array(phi, dtype=np.float64)
    for t in range(Z.shape[1]):
        r = label_rank(Z[:, t])
        after = r[None, :] > r[:, None]
        before = r[None, :] < r[:, None]
        gt = c_t[t] * (np.sum(k_dense * after, axis=1) - np.sum(k_dense * before, axis=1))
        G += gt[:, None] * np.asarray(members[t], dtype=np.float64)[None, :]
    return G


def subgradient_tree_dc(phi, y, c, filter_partitioned, members, c_t):
    """The same with the divide and conquer of Appendix E on every subtree column."""
    Z = subtree_values(y, members)
    G = np.array(phi, dtype=np.float64)
    for t in range(Z.shape[1]):
        U = upper_sums_dc(label_rank(Z[:, t]), filter_partitioned)
        G += (c_t[t] * (2.0 * U - c))[:, None] * np.asarray(members[t], dtype=np.float64)[None, :]
    return G


def s_lp_tree_pairs(phi, k_dense, y, members, c_t) -> float:
    """The r-HST LP objective by pairs (exact K, tiny N only)."""
    Z = subtree_values(y, members)
    K = np.array(k_dense, dtype=np.float64)
    np.fill_diagonal(K, 0.0)
    pair = sum(c_t[t] * np.sum(K * np.abs(Z[:, t][:, None] - Z[:, t][None, :])) / 2.0 for t in range(Z.shape[1]))
    return float(np.sum(phi * y) + pair)


# ---------------------------------------------------------------------------
# Kleinberg-Tardos rounding of an LP point (uniform metric).


def kt_round(y: np.ndarray, phase_labels, phase_thresholds, labels=None) -> np.ndarray:
    """Labels after the given phases; -1 marks a pixel no phase has labelled.

    Phase t gives label phase_labels[t] to every unlabelled pixel a with
    y_a(phase_labels[t]) > phase_thresholds[t] (both in FP32).  `labels`
    (optional) is a previous result to continue from: its entries >= 0 stay.
    """
    y32 = np.asarray(y, dtype=np.float32)
    out = np.full(y32.shape[0], -1, dtype=np.int32) if labels is None else np.array(labels, dtype=np.int32)
    for i, alpha in zip(np.asarray(phase_labels), np.asarray(phase_thresholds, dtype=np.float32)):
        hit = (out < 0) & (y32[:, int(i)] > alpha)
        out[hit] = int(i)
    return out


def kt_separation_probability(ya: np.ndarray, yb: np.ndarray) -> float:
    """Exact probability that the rounding gives two pixels different labels.

    Until one of them is labelled, a phase labels both (label i, threshold
    below min(ya(i), yb(i))) or exactly one of them; the first such event
    decides.  Both together: the same label.  One alone with label i: the
    other later draws its label from its own marginal, equal to i with
    probability y(i).  The events of one phase have weights min_i, (ya-yb)+_i
    and (yb-ya)+_i, summing to 1 + d with d = |ya - yb|_1 / 2.
    """
    a = np.asarray(ya, np.float64)
    b = np.asarray(yb, np.float64)
    d = 0.5 * float(np.abs(a - b).sum())
    same = float(np.sum(np.minimum(a, b) + np.maximum(a - b, 0.0) * b + np.maximum(b - a, 0.0) * a))
    return 1.0 - same / (1.0 + d)
