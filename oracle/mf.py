"""Mean-field baseline and rounding, FP64 (test infrastructure).

The paper compares its relaxations with the parallel mean-field algorithm of
the dense-CRF filtering work it builds on (Section 1; MF and MF5 = five
iterations, Section 6.2) and reports the energy of the final labelling.  Mean
field approximates P(x) proportional to exp(-E(x)) with E of Eq. 1, whose
pairwise sum runs over ordered pairs (a, b != a); for a factorised Q the
expected energy is phi^T Q + Q^T Psi Q with Psi = mu (x) (K - sum_w I)
(reading c1), and its stationarity conditions give the parallel update

    Q = softmax_rows(-phi - (Psi + Psi^T) Q)

(2 Psi Q for a symmetric kernel; the transpose keeps it exact for the
evaluated lattice operator, reading c4).  The record per iteration is the
relaxed energy S_QP(Q) = phi^T Q + Q^T Psi Q of the current marginals.
Rounding takes the most probable label of every pixel (lowest label on ties);
the energy of a labelling is Eq. 1, S_QP at the one-hot rows.
"""
from __future__ import annotations

import numpy as np


def softmax_rows(Z: np.ndarray) -> np.ndarray:
    Z = Z - Z.max(axis=1, keepdims=True)
    E = np.exp(Z)
    return E / E.sum(axis=1, keepdims=True)


def mean_field(crf, q0, iters: int):
    """Returns (Q, energies[iters+1]): S_QP(Q^t) before each update and at the end."""
    Q = np.array(q0, dtype=np.float64)
    energies = []
    for t in range(iters + 1):
        m = crf.psi(Q)
        energies.append(float(np.sum(crf.phi * Q) + np.sum(Q * m)))
        if t == iters:
            break
        Q = softmax_rows(-crf.phi - m - crf.psi_T(Q))
    return Q, np.array(energies)


def round_labels(y: np.ndarray) -> np.ndarray:
    """Most probable label per row, lowest label on ties (np.argmax keeps the first)."""
    return np.argmax(np.asarray(y), axis=1)
