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
"""
from __future__ import annotations

import numpy as np


def step_size(A: float, B: float) -> float:
    """Minimiser of A a^2 + B a over a in [0, 1] (reading c3)."""
    if A > 0.0:
        return float(min(1.0, max(0.0, -B / (2.0 * A))))
    return 1.0 if A + B < 0.0 else 0.0


def frank_wolfe(crf, y0, iters: int, lin=None, P_y=None):
    """Returns (y, P_y, records); records[t] = (energy, gap, alpha, A, B) at y^t."""
    lin = crf.phi - crf.d if lin is None else lin
    y = np.array(y0, dtype=np.float64)
    P_y = crf.psi_plus_D(y) if P_y is None else P_y.copy()
    rows = np.arange(crf.n)
    recs = []
    for _ in range(iters):
        g = lin + 2.0 * P_y
        s_idx = np.argmin(g, axis=1)
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


def cccp_dc_gen(crf, y0, outer: int, inner: int):
    """Returns (y, qp_energies[outer+1]) with S_QP after every outer step."""
    y = np.array(y0, dtype=np.float64)
    P_y = crf.psi_plus_D(y)

    def s_qp(y, P_y):
        return float(np.sum(crf.phi * y) + np.sum(y * P_y) - np.sum(crf.d * y * y))

    energies = [s_qp(y, P_y)]
    for _ in range(outer):
        lin = crf.phi - 2.0 * crf.d * y
        y, P_y, _ = frank_wolfe(crf, y, inner, lin=lin, P_y=P_y)
        energies.append(s_qp(y, P_y))
    return y, np.array(energies)
