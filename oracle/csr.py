"""General sparse operator and BiCGSTAB inner solve (oracle).

The paper applies (K + tau_k M)^{-1} inexactly with BiCGSTAB (Section 6, with an
algebraic-multigrid preconditioner; Section 4, Eq. zmmoditer). For operators
given as general sparse matrices (finite-element K and M, Section 5.1) this
build's inner solve is the same stationary defect correction as for grids,
z <- z + C(v - A z) from z = 0 with ||p|| = ||v - A z|| computed exactly, where one
"cycle" C is s steps of BiCGSTAB (van der Vorst's method) with Jacobi
preconditioning D^{-1}, D = diag(K + tau M), started from e = 0 on A e = r:

    r = r_hat = f, p = v = 0, rho_old = alpha = omega = 1
    repeat s times:
        rho = <r_hat, r>;  beta = (rho / rho_old) (alpha / omega)
        p = r + beta (p - omega v);  p_hat = D^{-1} p;  v = A p_hat
        alpha = rho / <r_hat, v>;  s_ = r - alpha v;  s_hat = D^{-1} s_;  t = A s_hat
        omega = <t, s_> / <t, t>;  e += alpha p_hat + omega s_hat;  r = s_ - omega t
        rho_old = rho
    (<a, b> = a^* b; a step whose denominator vanishes leaves e unchanged and
    ends the cycle)

The oracle uses scipy sparse products and NumPy vector operations only.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

STEPS = 8


@dataclasses.dataclass
class CSROperator:
    K: sp.csr_matrix
    M: sp.csr_matrix

    @property
    def n(self) -> int:
        return self.K.shape[0]

    def shifted(self, s: complex) -> sp.csr_matrix:
        return (self.K + s * self.M).tocsr()


def csr_operator(n, rowptr, col, kval, m_rowptr, m_col, mval) -> CSROperator:
    K = sp.csr_matrix((np.asarray(kval, float), np.asarray(col), np.asarray(rowptr)), shape=(n, n))
    M = sp.csr_matrix((np.asarray(mval, float), np.asarray(m_col), np.asarray(m_rowptr)), shape=(n, n))
    return CSROperator(K, M)


def bicgstab_cycle(A, dinv, f, steps):
    """`steps` preconditioned BiCGSTAB steps on A e = f from e = 0. The
    preconditioner `dinv` is the Jacobi diagonal D^{-1} (an array, applied
    elementwise) or a callable (the AMG V-cycle of oracle.amg)."""
    prec = dinv if callable(dinv) else (lambda x: dinv * x)
    e = np.zeros_like(f)
    r = f.copy()
    rh = f.copy()
    p = np.zeros_like(f)
    v = np.zeros_like(f)
    rho_old = alpha = omega = 1.0 + 0j
    for _ in range(steps):
        rho = np.vdot(rh, r)
        if rho == 0 or omega == 0:
            break
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = prec(p)
        v = A @ ph
        den = np.vdot(rh, v)
        if den == 0:
            break
        alpha = rho / den
        s = r - alpha * v
        sh = prec(s)
        t = A @ sh
        tt = np.vdot(t, t)
        if tt == 0:
            e = e + alpha * ph
            break
        omega = np.vdot(t, s) / tt
        e = e + alpha * ph + omega * sh
        r = s - omega * t
        rho_old = rho
    return e


class BiCGStabInner:
    """Inner solve callable for the shifted solver: (v, tau_index, k) -> (z, cycles, ||p||)."""

    def __init__(self, op: CSROperator, taus, eps, steps=STEPS, max_cycles=50, replay_cycles=None):
        self.A = [op.shifted(t) for t in taus]
        self.dinv = [1.0 / A.diagonal() for A in self.A]
        self.eps = eps
        self.steps = steps
        self.max_cycles = max_cycles
        self.replay = None if replay_cycles is None else list(replay_cycles)

    def solve(self, v, p, cycles=None):
        A = self.A[p]
        z = np.zeros_like(v)
        r = v.copy()
        nr = np.linalg.norm(r)
        nv = np.linalg.norm(v)
        c = 0
        while (c < cycles) if cycles is not None else (nr > self.eps * nv and c < self.max_cycles):
            z = z + bicgstab_cycle(A, self.dinv[p], r, self.steps)
            c += 1
            r = v - A @ z
            nr = np.linalg.norm(r)
        return z, c, nr

    def __call__(self, v, p, k, eps=None):
        cyc = None if self.replay is None else int(self.replay[k - 1])
        if eps is None:
            return self.solve(v, p, cyc)
        keep, self.eps = self.eps, eps
        try:
            return self.solve(v, p, cyc)
        finally:
            self.eps = keep
