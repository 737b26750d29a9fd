"""Frank-Wolfe on S_cvx and CCCP on the generic DC relaxation, FP64 (test infrastructure).

Frank-Wolfe (Algorithm 1, Section 4) with the step of Appendix B, written in
the update convention y <- y + alpha (s - y) of Appendix B (reading c2):

    g     = lin + 2 P_y                      gradient, Eq. 12 (lin = phi - d)
    s     = onehot(argmin_i g_a(i))          conditional gradient, Eq. 14
                                              (lowest label on ties, reading c6)
    gap   = <g, y - s>
    P_s   = (Psi + D) s                      the one filter of the iteration
    A     = <s - y, P_s - P_y>
    B     = <lin, s - y> + <y, P_s - P_y> + <s - y, P_y>
    alpha = argmin over [0,1] of A a^2 + B a (reading c3)
    y    += alpha (s - y);  P_y += alpha (P_s - P_y)   (product reuse, App. B)

B is the exact derivative at a = 0 of S_cvx(y + a (s - y)) for the evaluated
operator; for a symmetric operator it equals the printed
(phi - d)^T (s - y) + 2 y^T (Psi + D)(s - y) (reading c4).

CCCP (Algorithm 2, Section 5.1): p(y) = phi^T y + y^T (Psi + D) y,
q(y) = y^T D y; each outer step replaces the linear term by
phi - grad q(y^t) = phi - 2 d o y^t and runs Frank-Wolfe warm-started at y^t.

CCCP for negative semi-definite compatibilities (Section 5.2, Appendix C):
one filter per outer step, then a per-pixel convex problem; see cccp_dc_neg.
"""
from __future__ import annotations

import numpy as np


def step_size(A: float, B: float) -> float:
    """Minimiser of A a^2 + B a over a in [0, 1] (reading c3)."""
    if A > 0.0:
        return float(min(1.0, max(0.0, -B / (2.0 * A))))
    return 1.0 if A + B < 0.0 else 0.0


def frank_wolfe(crf, y0, iters: int, lin=None, P_y=None, decisions=None, on_step=None):
    """Returns (y, P_y, records); records[t] = (energy, gap, alpha, A, B) at y^t.

    decisions: optional [iters][n] label indices to use as s^t instead of the
    argmin (a replay of another run's choices, which may differ from the FP64
    argmin only where g is within rounding of a tie); on_step(t, g, s_idx) is
    called with the gradient of every iteration and the vertex taken.
    """
    lin = crf.phi - crf.d if lin is None else lin
    y = np.array(y0, dtype=np.float64)
    P_y = crf.psi_plus_D(y) if P_y is None else P_y.copy()
    rows = np.arange(crf.n)
    recs = []
    for t in range(iters):
        g = lin + 2.0 * P_y
        s_idx = np.argmin(g, axis=1) if decisions is None else np.asarray(decisions[t], dtype=np.int64)
        if on_step is not None:
            on_step(t, g, s_idx)
        s = np.zeros_like(y)
        s[rows, s_idx] = 1.0
        gap = float(np.sum(g * (y - s)))
        energy = float(np.sum(lin * y) + np.sum(y * P_y))
        P_s = crf.psi_plus_D(s)
        delta = s - y
        dP = P_s - P_y
        A = float(np.sum(delta * dP))
        B = float(np.sum(lin * delta) + np.sum(y * dP) + np.sum(delta * P_y))
        alpha = step_size(A, B)
        y = y + alpha * delta
        P_y = P_y + alpha * dP
        recs.append((energy, gap, alpha, A, B))
    return y, P_y, np.array(recs).reshape(-1, 5)


def cccp_dc_gen(crf, y0, outer: int, inner: int, decisions=None, on_step=None):
    """Returns (y, qp_energies[outer+1]) with S_QP after every outer step.

    decisions: optional [outer * inner][n] vertices replayed by the inner
    Frank-Wolfe runs (row o * inner + i for inner iteration i of outer step o);
    on_step(o * inner + t, g, s_idx) as in frank_wolfe.
    """
    y = np.array(y0, dtype=np.float64)
    P_y = crf.psi_plus_D(y)

    def s_qp(y, P_y):
        return float(np.sum(crf.phi * y) + np.sum(y * P_y) - np.sum(crf.d * y * y))

    energies = [s_qp(y, P_y)]
    for o in range(outer):
        lin = crf.phi - 2.0 * crf.d * y
        dec = None if decisions is None else decisions[o * inner:(o + 1) * inner]
        step = None if on_step is None else (lambda t, g, s, o=o: on_step(o * inner + t, g, s))
        y, P_y, _ = frank_wolfe(crf, y, inner, lin=lin, P_y=P_y, decisions=dec, on_step=step)
        energies.append(s_qp(y, P_y))
    return y, np.array(energies)


# ---------------------------------------------------------------------------
# CCCP on the DC relaxation for negative semi-definite compatibilities
# (Section 5.2 and Appendix C).
#
# S_QP(y) = phi^T y + y^T Psi y with Psi = mu (x) (K - sum_w I) (reading c1)
# splits into
#   convex:   phi^T y - sum_w y^T (mu (x) I) y     (mu negative semi-definite on
#                                                  the zero-sum directions of M)
#   concave:  y^T (mu (x) K) y                     (K positive semi-definite)
# Each outer step replaces the concave part by its linearisation at y^t, whose
# gradient is (mu (x) K) y^t + (mu (x) K)^T y^t (exact for the evaluated,
# slightly non-symmetric lattice operator; reading c4), and solves the convex
# problem, which decouples over pixels (Appendix C):
#   min_{y_a in simplex}  lin_a^T y_a - sum_w y_a^T mu y_a,
#   lin_a = phi_a + mu (K y^t + K^T y^t)_a        (mu symmetric).
# Potts (mu = 1 1^T - I): on the simplex - y^T mu y = |y|^2 - 1, so the
# minimiser is the Euclidean projection of -lin_a / (2 sum_w) (closed form).
# Other mu: `inner` Frank-Wolfe steps per pixel with the exact step of the
# per-pixel quadratic, warm-started at y^t_a.


def dc_neg_pixel_fw(lin, y0, mu, sum_w, inner: int):
    """Frank-Wolfe on min lin_a^T y_a - sum_w y_a^T mu y_a for every pixel a."""
    y = np.array(y0, dtype=np.float64)
    rows = np.arange(y.shape[0])
    for _ in range(inner):
        g = lin - sum_w * (y @ (mu + mu.T))
        s = np.zeros_like(y)
        s[rows, np.argmin(g, axis=1)] = 1.0
        d = s - y
        A = -sum_w * np.einsum("ai,ij,aj->a", d, mu, d)
        B = np.sum(g * d, axis=1)
        al = np.array([step_size(a_, b_) for a_, b_ in zip(A, B)])
        y = y + al[:, None] * d
    return y


def cccp_dc_neg(crf, y0, outer: int, inner: int = 0):
    """Returns (y, qp_energies[outer+1]) with S_QP after every outer step."""
    from oracle.lp import project_simplex
    y = np.array(y0, dtype=np.float64)
    mu = crf.mu
    sw = crf.kernel.sum_w
    potts = np.array_equal(mu, 1.0 - np.eye(crf.L))
    energies = []
    for t in range(outer + 1):
        F = crf.kernel.apply(y) + crf.kernel.apply_T(y)          # K y + K^T y
        # S_QP = phi^T y + 1/2 y^T mu F - sum_w y^T mu y  (y^T K y = y^T K^T y)
        energies.append(float(np.sum(crf.phi * y) + 0.5 * np.sum(y * (F @ mu.T)) - sw * np.sum(y * (y @ mu.T))))
        if t == outer:
            break
        lin = crf.phi + F @ mu.T
        if potts:
            y = project_simplex(-lin / (2.0 * sw))
        else:
            y = dc_neg_pixel_fw(lin, y, mu, sw, inner)
    return y, np.array(energies)


# ---------------------------------------------------------------------------
# Reverse mode through unrolled Frank-Wolfe (differentiation of T iterations)
#
# With P = Op(y) = (Psi + D) y exact, one iteration is
#   y+ = y + alpha (s - y),  alpha = -B / (2A) when 0 < alpha < 1 and A > 0,
# s piecewise constant in (y, phi, w) and alpha constant when clipped.  With
# Delta = s - y and u = y - (1 - 2 alpha) Delta:
#   d alpha / d y   = (lin + Op u + Op^T u) / (2A)
#   d alpha / d phi = -Delta / (2A)
#   d alpha / d w_m = -(dB_m + 2 alpha dA_m) / (2A),
#     dA_m = <Delta, Op_m' Delta>,
#     dB_m = -<d_m', Delta> + <y, Op_m' Delta> + <Delta, Op_m' y>,
#   where Op_m' v = mu (K_m v - v) + d_m' o v is the derivative of Op in w_m and
#   d_m' = (sum_j |mu_ij|) (K_m 1 - 1) [c > 0] that of d (lin = phi - d).
# The adjoint step is  ybar <- (1 - alpha) ybar + abar d alpha/dy,  abar = <ybar, Delta>.


class WeightedCRF:
    """Dense CRF whose kernel weights are explicit: K = sum_m w_m K_m (K_m unweighted)."""

    def __init__(self, unaries, ops, weights, mu=None):
        """ops: per kernel (apply, apply_T) of the unweighted K_m (diagonal included)."""
        from oracle.crf import potts
        self.phi = np.asarray(unaries, dtype=np.float64)
        self.n, self.L = self.phi.shape
        self.ops = ops
        self.w = np.asarray(weights, dtype=np.float64)
        self.mu = potts(self.L) if mu is None else np.asarray(mu, dtype=np.float64)
        self.musum = np.abs(self.mu).sum(axis=1)
        ones = np.ones((self.n, 1))
        self.o = [op(ones)[:, 0] for op, _ in ops]
        c = sum(w * o for w, o in zip(self.w, self.o)) - self.w.sum()
        self.active = c > 0
        self.c = np.maximum(c, 0.0)
        self.d = self.musum[None, :] * self.c[:, None]
        self.dd = [self.musum[None, :] * ((o - 1.0) * self.active)[:, None] for o in self.o]

    def op(self, v):
        x = sum(w * f(v) for w, (f, _) in zip(self.w, self.ops)) - self.w.sum() * v
        return x @ self.mu.T + self.d * v

    def op_T(self, v):
        x = sum(w * ft(v) for w, (_, ft) in zip(self.w, self.ops)) - self.w.sum() * v
        return x @ self.mu + self.d * v

    def dop(self, m, v):
        return (self.ops[m][0](v) - v) @ self.mu.T + self.dd[m] * v

    psi_plus_D = op


def fw_tape(crf, y0, iters, decisions=None):
    """Forward pass keeping y^t, s^t and (alpha, A, B) of every iteration.

    decisions: optional [iters][n] label indices taken as s^t instead of the
    argmin, which fixes the smooth piece of the unrolled map (see frank_wolfe).
    """
    lin = crf.phi - crf.d
    y = np.array(y0, dtype=np.float64)
    P = crf.op(y)
    rows = np.arange(crf.n)
    tape = []
    for t in range(iters):
        g = lin + 2.0 * P
        s = np.zeros_like(y)
        s_idx = np.argmin(g, axis=1) if decisions is None else np.asarray(decisions[t], dtype=np.int64)
        s[rows, s_idx] = 1.0
        Ps = crf.op(s)
        delta, dP = s - y, Ps - P
        A = float(np.sum(delta * dP))
        B = float(np.sum(lin * delta) + np.sum(y * dP) + np.sum(delta * P))
        alpha = step_size(A, B)
        tape.append((y.copy(), s, alpha, A, B))
        y = y + alpha * delta
        P = P + alpha * dP
    return y, tape


def fw_backward(crf, tape, ybar):
    """Gradients of <ybar, y^T> w.r.t. phi, the kernel weights and y^0."""
    lin = crf.phi - crf.d
    ybar = np.array(ybar, dtype=np.float64)
    phibar = np.zeros_like(lin)
    wbar = np.zeros(len(crf.w))
    for y, s, alpha, A, B in reversed(tape):
        delta = s - y
        abar = float(np.sum(ybar * delta))
        interior = A > 0.0 and 0.0 < alpha < 1.0
        if interior:
            u = y - (1.0 - 2.0 * alpha) * delta
            da_dy = (lin + crf.op(u) + crf.op_T(u)) / (2.0 * A)
            phibar += -abar * delta / (2.0 * A)
            for m in range(len(crf.w)):
                dA = float(np.sum(delta * crf.dop(m, delta)))
                dB = float(-np.sum(crf.dd[m] * delta) + np.sum(y * crf.dop(m, delta)) + np.sum(delta * crf.dop(m, y)))
                wbar[m] += abar * (-(dB + 2.0 * alpha * dA) / (2.0 * A))
            ybar = (1.0 - alpha) * ybar + abar * da_dy
        else:
            ybar = (1.0 - alpha) * ybar
    return phibar, wbar, ybar
