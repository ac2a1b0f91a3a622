"""Exact inner solves and the per-shift direct comparator (oracle).

ExactInner applies (K + tau M)^{-1} by a sparse LU factorisation of each distinct
tau_bar, as the paper's "Flexible" variant does with SuperLU (Section 2.2.1,
Section 6.1); ||p_k|| is still computed as ||v - (K + tau M) z||.
direct_solve factorises K + sigma_j M for every shift ("Direct", Section 6.1).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


class ExactInner:
    def __init__(self, op, taus):
        self.A = [op.shifted(t).tocsc() for t in taus]
        self.lu = [spla.splu(A) for A in self.A]

    def __call__(self, v, p, k, eps=None):  # exact: a tolerance does not apply
        z = self.lu[p].solve(v)
        return z, 0, float(np.linalg.norm(v - self.A[p] @ z))


def direct_solve(op, b, sigmas):
    """x_j = (K + sigma_j M)^{-1} b for every shift, one factorisation per shift."""
    out = np.zeros((op.n, len(sigmas)), dtype=np.complex128)
    for j, s in enumerate(sigmas):
        out[:, j] = spla.splu(op.shifted(s).tocsc()).solve(b)
    return out
