"""Smoothed-aggregation algebraic multigrid for K + tau M and the
AMG-preconditioned BiCGSTAB inner solve (oracle).

Test infrastructure: imported by the tests and the benchmark's CPU legs only,
never by the product path.

Section 6 inverts each preconditioner K + tau_k M with BiCGSTAB preconditioned
by smoothed-aggregation AMG (PyAMG) and names no parameters. This module states
the method from its definition (Vanek, Mandel & Brezina, Computing 56, 1996),
with the choices below (each a reading of the paper's silence):

  strength graph   every stored off-diagonal connection is strong (theta = 0).
                   Level 0 takes the entries where K or M is nonzero; level l+1
                   the pattern that P_l^T A_l P_l has structurally, i.e. the
                   pattern of |P_l|^T |A_l| |P_l| (nonnegative products never
                   cancel), so the graph, and with it the aggregates, does not
                   depend on tau
  aggregation      pass 1, nodes in ascending order: a node none of whose
                   neighbours is aggregated forms an aggregate with all of its
                   neighbours (a node without neighbours forms one alone);
                   pass 2: every node left joins the aggregate of its first
                   neighbour, in ascending order, that pass 1 aggregated (one
                   always exists: a node skipped by pass 1 had one)
  tentative T_l    the near-null-space vector B_l (B_0 = 1) cut to each
                   aggregate and normalised: T[i, a] = B_l[i] / ||B_l|a||, and
                   B_{l+1}[a] = ||B_l|a||
  smoothed P_l     (I - omega_l D_l^{-1} A_l) T_l with omega_l = 4 / (3 rho_l),
                   rho_l = max_i sum_j |a_ij| / |a_ii| (the Gershgorin bound of
                   the spectral radius of D^{-1} A)
  coarse operator  A_{l+1} = P_l^T A_l P_l (the plain transpose, so that a
                   complex-symmetric A_l gives a complex-symmetric A_{l+1})
  coarsest level   level l becomes the coarsest when n_l <= max_coarse, when
                   l = max_levels - 1, or when aggregation no longer shrinks the
                   level; it is solved exactly (its dense inverse, at most
                   4096 unknowns)
  V-cycle          nu damped-Jacobi sweeps (weight omega_l; nu = 2 by default)
                   from zero before the coarse correction and nu after it:
                       x = omega D^{-1} f, then nu - 1 times x += omega D^{-1} (f - A x)
                       r = f - A x;  x = x + P V_{l+1}(P^T r)
                       nu times x += omega D^{-1} (f - A x);  V_l(f) = x

The inner solve is the defect correction of oracle.csr (z <- z + C(v - A z),
||p|| exact), with one cycle C = s BiCGSTAB steps whose preconditioner is one
V-cycle.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .csr import BiCGStabInner, CSROperator

MAX_DENSE = 4096


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix            # A_l (complex)
    dinv: np.ndarray            # 1 / diag(A_l)
    omega: float                # 4 / (3 rho_l)
    P: sp.csr_matrix | None     # n_l x n_{l+1} (None on the coarsest level)
    agg: np.ndarray | None      # aggregate of every node (None on the coarsest level)


@dataclasses.dataclass
class AMGHierarchy:
    levels: list
    coarse_inv: np.ndarray      # dense inverse of the coarsest A

    @property
    def sizes(self):
        return [lv.A.shape[0] for lv in self.levels]


def _offdiag_pattern(S: sp.csr_matrix):
    """CSR row pointers and sorted column indices of the off-diagonal entries of S."""
    S = sp.csr_matrix(S, copy=True)
    S.setdiag(0)
    S.eliminate_zeros()
    S.sort_indices()
    return S.indptr, S.indices


def aggregate(S: sp.csr_matrix) -> tuple[np.ndarray, int]:
    """Standard aggregation (passes 1 and 2) on the off-diagonal pattern of S."""
    ptr, idx = _offdiag_pattern(S)
    n = S.shape[0]
    agg = np.full(n, -1, dtype=np.int64)
    first_pass = np.zeros(n, dtype=bool)
    na = 0
    for i in range(n):
        nb = idx[ptr[i]:ptr[i + 1]]
        if agg[i] == -1 and np.all(agg[nb] == -1):
            agg[i] = na
            agg[nb] = na
            first_pass[i] = True
            first_pass[nb] = True
            na += 1
    for i in range(n):
        if agg[i] != -1:
            continue
        for j in idx[ptr[i]:ptr[i + 1]]:
            if first_pass[j]:
                agg[i] = agg[j]
                break
        assert agg[i] != -1
    return agg, na


def tentative(agg: np.ndarray, na: int, B: np.ndarray) -> tuple[sp.csr_matrix, np.ndarray]:
    """T[i, agg[i]] = B[i] / ||B restricted to the aggregate||; the coarse B is that norm."""
    norms = np.sqrt(np.bincount(agg, weights=B * B, minlength=na))
    n = len(agg)
    T = sp.csr_matrix((B / norms[agg], (np.arange(n), agg)), shape=(n, na))
    return T, norms


def gershgorin_omega(A: sp.csr_matrix) -> float:
    d = np.abs(A.diagonal())
    rho = float(np.max(np.asarray(abs(A).sum(axis=1)).ravel() / d))
    return 4.0 / (3.0 * rho)


def sa_hierarchy(A0: sp.csr_matrix, S0: sp.csr_matrix, max_levels: int = 10, max_coarse: int = 256) -> AMGHierarchy:
    """The hierarchy of A0 (complex) on the strength pattern S0 (nonnegative, with the diagonal)."""
    A = sp.csr_matrix(A0, dtype=np.complex128)
    S = sp.csr_matrix(abs(S0), dtype=np.float64)
    S.data[:] = 1.0
    B = np.ones(A.shape[0])
    levels = []
    while True:
        n = A.shape[0]
        d = A.diagonal()
        if np.any(d == 0):
            raise ValueError("AMG: zero diagonal entry")
        om = gershgorin_omega(A)
        last = n <= max_coarse or len(levels) == max_levels - 1
        if not last:
            agg, na = aggregate(S)
            last = na >= n
        if last:
            if n > MAX_DENSE:
                raise ValueError(f"AMG: coarsest level has {n} > {MAX_DENSE} unknowns")
            levels.append(Level(A, 1.0 / d, om, None, None))
            return AMGHierarchy(levels, np.linalg.inv(A.toarray()))
        T, B = tentative(agg, na, B)
        Dinv = sp.diags(1.0 / d)
        P = (T - om * (Dinv @ (A @ T))).tocsr()
        levels.append(Level(A, 1.0 / d, om, P, agg))
        A = (P.T @ A @ P).tocsr()
        Ts = sp.csr_matrix(T, copy=True)
        Ts.data[:] = 1.0
        Ps = S @ Ts                       # structural pattern of P
        Ps.data[:] = 1.0
        S = (Ps.T @ S @ Ps).tocsr()
        S.data[:] = 1.0


def strength0(K: sp.spmatrix, M: sp.spmatrix) -> sp.csr_matrix:
    """Level-0 pattern: the entries where K or M is nonzero, with the diagonal."""
    S = (abs(sp.csr_matrix(K)) + abs(sp.csr_matrix(M))).tocsr()
    S.eliminate_zeros()
    return S + sp.identity(S.shape[0], format="csr")


def vcycle(h: AMGHierarchy, f: np.ndarray, l: int = 0, nu: int = 2) -> np.ndarray:
    """V_l(f), the V-cycle of the module docstring."""
    lv = h.levels[l]
    if lv.P is None:
        return h.coarse_inv @ f
    x = lv.omega * (lv.dinv * f)
    for _ in range(nu - 1):
        x = x + lv.omega * (lv.dinv * (f - lv.A @ x))
    r = f - lv.A @ x
    x = x + lv.P @ vcycle(h, lv.P.T @ r, l + 1, nu)
    for _ in range(nu):
        x = x + lv.omega * (lv.dinv * (f - lv.A @ x))
    return x


class AMGBiCGStabInner(BiCGStabInner):
    """Inner solve callable for the shifted solver: defect correction whose cycles
    are s BiCGSTAB steps preconditioned by one V-cycle of K + tau M's hierarchy."""

    def __init__(self, op: CSROperator, taus, eps, steps=4, max_cycles=50, replay_cycles=None, max_levels=10,
                 max_coarse=256, nu=2):
        super().__init__(op, taus, eps, steps=steps, max_cycles=max_cycles, replay_cycles=replay_cycles)
        S0 = strength0(op.K, op.M)
        self.h = [sa_hierarchy(A, S0, max_levels, max_coarse) for A in self.A]
        self.dinv = [(lambda v, h=h: vcycle(h, v, 0, nu)) for h in self.h]
