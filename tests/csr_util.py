"""Sparse-operator fixtures shared by the oracle and GPU tests of the CSR path:
a finite-element-like operator (bilinear-element stiffness with random element
coefficients and a consistent mass matrix) and the CSR arrays of any K, M."""
import dataclasses

import numpy as np
import scipy.sparse as sp

from oracle.csr import CSROperator

# bilinear (Q1) element matrices on a unit square, nodes (0,0), (1,0), (0,1), (1,1)
KE = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
ME = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36.0


def fe_like(n_side=12, seed=0, anchor=1e-3):
    """n_side x n_side nodes; K gets `anchor` * I so that it is SPD (a zero-head anchoring)."""
    rng = np.random.default_rng(seed)
    n = n_side * n_side
    idx = np.arange(n).reshape(n_side, n_side)
    nodes = np.stack([idx[:-1, :-1].ravel(), idx[:-1, 1:].ravel(), idx[1:, :-1].ravel(), idx[1:, 1:].ravel()], 1)
    c = np.exp(rng.standard_normal(len(nodes)))
    rows = np.repeat(nodes, 4, axis=1).ravel()
    cols = np.tile(nodes, (1, 4)).ravel()
    kdat = (c[:, None] * KE.ravel()[None, :]).ravel()
    mdat = np.tile(ME.ravel(), len(nodes))
    K = sp.coo_matrix((kdat, (rows, cols)), shape=(n, n)).tocsr() + anchor * sp.identity(n, format="csr")
    M = sp.coo_matrix((mdat, (rows, cols)), shape=(n, n)).tocsr()
    return CSROperator(K.tocsr(), M.tocsr())


def csr_arrays(K, M):
    """(k_rowptr, k_col, k_val, m_rowptr, m_col, m_val) as the C ABI takes them."""
    K, M = sp.csr_matrix(K), sp.csr_matrix(M)
    return (K.indptr.astype(np.int64), K.indices.astype(np.int32), K.data.astype(np.float64),
            M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float64))


@dataclasses.dataclass
class SparseProblem:
    """Shifts, schedule, tolerance and point sources for a K, M given as matrices."""
    n: int
    sigma: np.ndarray
    tau_bar: np.ndarray
    schedule: np.ndarray
    src_cells: np.ndarray
    tol: float = 1e-8
    m_max: int = 100
    q0: float = 1.0

    def rhs(self):
        b = np.zeros((self.n, len(self.src_cells)), dtype=np.complex128)
        b[self.src_cells, np.arange(len(self.src_cells))] = self.q0
        return b


def sparse_problem(n, n_f=6, omega=(1e-2, 1e2), taus=(0.1, 10.0), n_src=1, seed=0, m_max=100, tol=1e-8):
    rng = np.random.default_rng(seed)
    src = rng.choice(n, size=n_src, replace=False).astype(np.int64)
    return SparseProblem(n=n, sigma=1j * np.logspace(np.log10(omega[0]), np.log10(omega[1]), n_f),
                         tau_bar=1j * np.asarray(taus, float), schedule=np.arange(len(taus), dtype=np.int32),
                         src_cells=src, tol=tol, m_max=m_max)
