"""Sparse-operator fixtures shared by the oracle and GPU tests of the CSR path:
a finite-element-like operator (bilinear-element stiffness with random element
coefficients and a consistent mass matrix) and the CSR arrays of any K, M."""
import dataclasses

import numpy as np
import scipy.sparse as sp

from oracle.csr import CSROperator
from paper_1212_3660_gb300 import synth

def fe_like(n_side=12, seed=0, anchor=1e-3):
    """n_side x n_side nodes; K gets `anchor` * I so that it is SPD (a zero-head anchoring)."""
    K, M = synth.fe_matrices(n_side, seed, anchor)
    return CSROperator(K, M)


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
