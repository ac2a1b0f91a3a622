"""Pins of the oracle's sparse-operator path: BiCGSTAB cycles against SciPy's
own bicgstab (Jacobi preconditioner, zero initial guess, the same number of
steps), the inner solve against sparse LU, and the whole shifted solve on a
general sparse (non-grid) operator against dense solves."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle.csr import CSROperator, bicgstab_cycle, BiCGStabInner, csr_operator
from paper_1212_3660_gb300 import synth

from csr_util import fe_like


@pytest.mark.parametrize("steps", [1, 3, 8])
def test_bicgstab_cycle_equals_scipy_bicgstab(steps):
    op = fe_like()
    A = op.shifted(0.7j)
    dinv = 1.0 / A.diagonal()
    rng = np.random.default_rng(3)
    f = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    e = bicgstab_cycle(A, dinv, f, steps)
    Mop = spla.LinearOperator(A.shape, matvec=lambda x: dinv * x, dtype=complex)
    e_ref, _ = spla.bicgstab(A, f, x0=np.zeros_like(f), rtol=1e-300, atol=0.0, maxiter=steps, M=Mop)
    assert np.linalg.norm(e - e_ref) <= 1e-10 * np.linalg.norm(e_ref)


def test_bicgstab_inner_reaches_eps_and_matches_lu():
    op = fe_like(seed=5)
    tau = 0.2j
    inner = BiCGStabInner(op, [tau], 1e-10)
    v = np.random.default_rng(1).standard_normal(op.n) + 0j
    v /= np.linalg.norm(v)
    z, c, pn = inner(v, 0, 1)
    A = op.shifted(tau)
    assert pn <= 1e-10 and abs(pn - np.linalg.norm(v - A @ z)) <= 1e-14
    z_lu = spla.spsolve(A.tocsc(), v)
    sv_min = np.linalg.svd(A.toarray(), compute_uv=False).min()
    assert np.linalg.norm(z - z_lu) <= 1.01 * pn / sv_min


def test_shifted_solve_on_general_sparse_operator_matches_dense():
    op = fe_like(n_side=10, seed=7)
    b = np.zeros(op.n, complex)
    b[op.n // 2 + 5] = 1.0
    sig = 1j * np.array([0.05, 0.3, 1.0, 2.5])
    taus = 1j * np.array([0.1, 1.0])
    inner = BiCGStabInner(op, taus, 1e-12)
    res = oracle.shifted_solve(op, b, sig, taus, [0, 1], 1e-10, 80, inner)
    for j, s in enumerate(sig):
        A = op.shifted(s).toarray()
        x = np.linalg.solve(A, b)
        assert np.linalg.norm(b - A @ res.x[:, j]) <= 1.0001e-10 * np.linalg.norm(b)
        assert np.linalg.norm(res.x[:, j] - x) <= 1e-10 * np.linalg.cond(A) * np.linalg.norm(x)


def test_csr_operator_from_arrays_equals_grid_operator():
    pr = synth.make_problem((9, 7), n_f=2, periods=(10.0, 1000.0), n_p=1, seed=3)
    g = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    K, M = g.K.tocsr(), g.M.tocsr()
    c = csr_operator(g.n, K.indptr, K.indices, K.data, M.indptr, M.indices, M.data)
    x = np.random.default_rng(0).standard_normal(g.n) + 0j
    assert np.allclose(c.shifted(0.3j) @ x, g.shifted(0.3j) @ x, rtol=1e-15, atol=0)
