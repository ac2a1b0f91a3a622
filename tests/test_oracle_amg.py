"""Pins of the smoothed-aggregation AMG oracle (oracle/amg.py) against facts
that do not come from the oracle itself: aggregates of small graphs worked by
hand from the two-pass rule, the tentative prolongator's orthonormality and
reproduction of the near-null-space vector, the Gershgorin weight of a
Laplacian, constants in the kernel of a Neumann operator carried to the coarse
level, the Galerkin identities of the coarse-grid correction, the V-cycle's error
propagation against the two-grid product formula, and the AMG-BiCGSTAB inner
solve against a sparse direct solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle.amg import (AMGBiCGStabInner, aggregate, gershgorin_omega, sa_hierarchy, strength0, tentative,
                        vcycle)
from oracle.csr import bicgstab_cycle

from csr_util import fe_like, sparse_problem


def lap1d(n):
    return sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def lap2d(nx, ny):
    return (sp.kron(sp.identity(ny), lap1d(nx)) + sp.kron(lap1d(ny), sp.identity(nx))).tocsr()


def test_aggregates_of_a_path_by_hand():
    # pass 1: 0 takes {0,1}; 3 takes {2,3,4}; 6 takes {5,6,7}; 9 takes {8,9}
    agg, na = aggregate(lap1d(10))
    assert na == 4
    assert agg.tolist() == [0, 0, 1, 1, 1, 2, 2, 2, 3, 3]


def test_aggregates_of_a_3x3_grid_by_hand():
    # nodes row-major; pass 1: 0 takes {0,1,3}; 2 and 4 see aggregated
    # neighbours; 5 takes {2,4,5,8}; pass 2: 6 joins 3's aggregate, 7 joins 4's
    agg, na = aggregate(lap2d(3, 3))
    assert na == 2
    assert agg.tolist() == [0, 0, 1, 0, 1, 1, 0, 1, 1]


def test_isolated_nodes_form_their_own_aggregates():
    S = sp.block_diag([lap1d(3), sp.identity(2), lap1d(2)], format="csr")
    agg, na = aggregate(S)
    assert agg.tolist() == [0, 0, 0, 1, 2, 3, 3] and na == 4


def test_aggregates_cover_and_are_connected():
    op = fe_like(20, seed=1)
    S = strength0(op.K, op.M)
    agg, na = aggregate(S)
    assert agg.min() == 0 and agg.max() == na - 1 and len(np.unique(agg)) == na
    G = sp.csr_matrix(S)
    for a in range(na):
        nodes = np.flatnonzero(agg == a)
        sub = G[nodes][:, nodes]
        ncomp, _ = sp.csgraph.connected_components(sub, directed=False)
        assert ncomp == 1, a


def test_tentative_is_orthonormal_and_reproduces_b():
    op = fe_like(16, seed=2)
    agg, na = aggregate(strength0(op.K, op.M))
    B = np.random.default_rng(0).uniform(0.5, 2.0, op.n)   # a non-constant B, as on level 1 and below
    T, Bc = tentative(agg, na, B)
    assert np.allclose((T.T @ T).toarray(), np.eye(na), atol=1e-14)
    assert np.allclose(T @ Bc, B, rtol=1e-14)


def test_gershgorin_weight_of_laplacians():
    # D^{-1} A of tridiag(-1, 2, -1): row sums of moduli 2, so omega = 2/3
    assert gershgorin_omega(lap1d(9).astype(complex)) == pytest.approx(2.0 / 3.0, rel=1e-15)
    # 5-point Laplacian: 8 / 4 = 2 as well; shifted by i: |4 + i| on the diagonal
    A = (lap2d(5, 5) + 1j * sp.identity(25)).tocsr()
    assert gershgorin_omega(A) == pytest.approx(4.0 / (3.0 * (1 + 4 / abs(4 + 1j))), rel=1e-14)


def test_neumann_constants_reach_the_coarse_level():
    """K without anchoring annihilates constants; the smoothed prolongator then
    reproduces them (P B_1 = 1) and the coarse operator annihilates B_1, up to the
    tiny shift 1e-13 i M that keeps the coarsest level invertible. A slip in the
    near-null-space bookkeeping (T, B_{l+1}) breaks this."""
    K, M = fe_matrices_no_anchor(14)
    assert np.abs(K @ np.ones(K.shape[0])).max() <= 1e-13
    A = (K + 1e-13j * M).tocsr()
    h = sa_hierarchy(A, strength0(K, M), max_levels=3, max_coarse=4)
    lv0, lv1 = h.levels[0], h.levels[1]
    _, B1 = tentative(lv0.agg, lv0.P.shape[1], np.ones(K.shape[0]))
    assert np.allclose(lv0.P @ B1, 1.0, rtol=0, atol=1e-12)
    assert np.linalg.norm(lv1.A @ B1) <= 1e-11 * abs(lv1.A).sum()


def test_smoothed_prolongator_of_a_path_by_hand():
    """tridiag(-1, 2, -1) on 10 nodes, aggregates {0,1} {2,3,4} ..., B = 1:
    T = 1/sqrt(2) and 1/sqrt(3) on the first two, omega D^{-1} = 1/3, so
    P = T - (A T) / 3 gives P[0,0] = 2/(3 sqrt 2), P[2,0] = 1/(3 sqrt 2),
    P[2,1] = 2/(3 sqrt 3), P[3,1] = 1/sqrt 3 and P[0,1] = 0."""
    h = sa_hierarchy(lap1d(10).astype(complex), lap1d(10), max_levels=2, max_coarse=1)
    P = h.levels[0].P.toarray()
    r2, r3 = np.sqrt(2.0), np.sqrt(3.0)
    assert P[0, 0] == pytest.approx(2 / (3 * r2), rel=1e-15)
    assert P[2, 0] == pytest.approx(1 / (3 * r2), rel=1e-15)
    assert P[2, 1] == pytest.approx(2 / (3 * r3), rel=1e-15)
    assert P[3, 1] == pytest.approx(1 / r3, rel=1e-15)
    assert P[0, 1] == 0 and P.shape == (10, 4)


def fe_matrices_no_anchor(n_side):
    from paper_1212_3660_gb300 import synth
    return synth.fe_matrices(n_side, 5, 0.0)


@pytest.mark.parametrize("tau", [0.05j, 3.0 - 2.0j])
def test_coarse_correction_is_a_galerkin_projector(tau):
    """E = I - P A_c^{-1} P^T A is a projection (E^2 = E) with P^T A E = 0, and
    A_c is complex symmetric like A (P^T, not P^H)."""
    op = fe_like(12, seed=3)
    A = op.shifted(tau)
    h = sa_hierarchy(A, strength0(op.K, op.M), max_levels=2, max_coarse=1)
    P, Ac = h.levels[0].P.toarray(), h.levels[1].A.toarray()
    Ad = A.toarray()
    assert np.abs(P.imag).max() > 0                      # smoothing with a complex A
    assert np.allclose(Ac, Ac.T, rtol=0, atol=1e-13 * np.abs(Ac).max())
    E = np.eye(op.n) - P @ np.linalg.solve(Ac, P.T @ Ad)
    assert np.allclose(E @ E, E, atol=1e-10)
    assert np.abs(P.T @ Ad @ E).max() <= 1e-11 * np.abs(Ad).max()


@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_error_propagation_is_the_two_grid_formula(nu):
    """On two levels, I - V A = S^nu (I - P A_c^{-1} P^T A) S^nu with the Jacobi
    error propagator S = I - omega D^{-1} A (textbook two-grid identity)."""
    op = fe_like(10, seed=4)
    A = op.shifted(0.7j)
    h = sa_hierarchy(A, strength0(op.K, op.M), max_levels=2, max_coarse=1)
    lv = h.levels[0]
    Ad = A.toarray()
    P, Ac = lv.P.toarray(), h.levels[1].A.toarray()
    S = np.eye(op.n) - lv.omega * (lv.dinv[:, None] * Ad)
    Snu = np.linalg.matrix_power(S, nu)
    E2 = Snu @ (np.eye(op.n) - P @ np.linalg.solve(Ac, P.T @ Ad)) @ Snu
    VA = np.stack([vcycle(h, Ad[:, j], 0, nu) for j in range(op.n)], axis=1)
    assert np.allclose(np.eye(op.n) - VA, E2, atol=1e-11)


def test_single_level_vcycle_is_the_exact_inverse():
    op = fe_like(8, seed=6)
    A = op.shifted(0.2 + 1j)
    h = sa_hierarchy(A, strength0(op.K, op.M), max_levels=1)
    f = np.random.default_rng(1).standard_normal(op.n) + 0j
    assert len(h.levels) == 1
    assert np.linalg.norm(A @ vcycle(h, f) - f) <= 1e-13 * np.linalg.norm(f)


def test_hierarchy_shape_and_contraction():
    """Q1 elements (9-point stencil) aggregate into about 3 x 3 blocks; the
    aggregates are the same for every tau; on the SPD case the V-cycle (the same
    convergent Jacobi sweeps before and after a Galerkin correction) has an
    A-self-adjoint error propagation with eigenvalues in [0, 1)."""
    op = fe_like(40, seed=7)
    S0 = strength0(op.K, op.M)
    hs = [sa_hierarchy(op.shifted(t), S0, max_coarse=64) for t in (0.01j, 1j, 100j)]
    assert hs[0].sizes == hs[1].sizes == hs[2].sizes
    for a, b in zip(hs[0].levels[:-1], hs[2].levels[:-1]):
        assert np.array_equal(a.agg, b.agg)
    sz = hs[0].sizes
    assert all(6 <= sz[i] / sz[i + 1] <= 12 for i in range(len(sz) - 1)), sz
    h = sa_hierarchy(op.K.astype(complex), S0, max_coarse=64)
    Kd = op.K.toarray()
    E = np.eye(op.n) - np.stack([vcycle(h, Kd[:, j] + 0j) for j in range(op.n)], axis=1)
    lam = np.linalg.eigvals(E)
    assert np.abs(lam.imag).max() <= 1e-10 and lam.real.min() >= -1e-10
    assert lam.real.max() < 0.9


def test_amg_bicgstab_inner_solve_reaches_the_direct_solution():
    op = fe_like(48, seed=8)
    for tau in (0.01j, 10j):
        inner = AMGBiCGStabInner(op, [tau], 1e-12, steps=4)
        v = np.random.default_rng(2).standard_normal(op.n) + 1j * np.random.default_rng(3).standard_normal(op.n)
        z, c, pn = inner(v, 0, 1)
        xd = spla.spsolve(op.shifted(tau).tocsc(), v)
        assert pn <= 1e-12 * np.linalg.norm(v) and c <= 6
        assert np.linalg.norm(z - xd) <= 1e-9 * np.linalg.norm(xd)
        # the defect it reports is the exact one
        assert abs(np.linalg.norm(v - op.shifted(tau) @ z) - pn) <= 1e-15 * np.linalg.norm(v)


def test_amg_preconditioning_beats_jacobi_per_step():
    op = fe_like(48, seed=9)
    A = op.shifted(0.05j)
    f = np.random.default_rng(4).standard_normal(op.n) + 0j
    inner = AMGBiCGStabInner(op, [0.05j], 1e-10)
    ea = bicgstab_cycle(A, inner.dinv[0], f, 6)
    ej = bicgstab_cycle(A, 1.0 / A.diagonal(), f, 6)
    ra, rj = (np.linalg.norm(f - A @ e) / np.linalg.norm(f) for e in (ea, ej))
    assert ra < 1e-4 and ra < 1e-3 * rj


def test_shifted_solve_with_amg_inner_is_certified():
    op = fe_like(32, seed=10)
    pr = sparse_problem(op.n, n_f=8, omega=(1e-2, 1e2), taus=(0.1, 10.0), seed=4, m_max=60)
    b = pr.rhs()[:, 0]
    inner = AMGBiCGStabInner(op, pr.tau_bar, 1e-10)
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max, inner)
    assert np.all(res.status == 0)
    tr = oracle.true_residuals(op, b, pr.sigma, res.x)
    assert np.all(tr <= pr.tol * 1.0001)
    xd = oracle.direct_solve(op, b, pr.sigma)
    for j in range(len(pr.sigma)):
        assert np.linalg.norm(res.x[:, j] - xd[:, j]) <= 1e-5 * np.linalg.norm(xd[:, j]), j


def test_vcycle_is_a_complex_symmetric_operator():
    """With R = P^T, a diagonal smoother and as many sweeps after the coarse
    correction as before, the V-cycle of a complex-symmetric A is itself complex
    symmetric (B = B^T, not B^H): a restriction by P^H or unequal sweep counts
    break it."""
    op = fe_like(14, seed=13)
    A = op.shifted(0.3 + 2j)
    h = sa_hierarchy(A, strength0(op.K, op.M), max_coarse=8)
    assert len(h.levels) >= 3
    I = np.eye(op.n, dtype=complex)
    for nu in (1, 2):
        B = np.stack([vcycle(h, I[:, j], 0, nu) for j in range(op.n)], axis=1)
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()
        assert np.abs(B - B.conj().T).max() > 1e-3 * np.abs(B).max()


@pytest.mark.parametrize("steps", [1, 2, 4])
def test_amg_bicgstab_cycle_equals_scipy_bicgstab(steps):
    """A cycle of AMG-preconditioned BiCGSTAB steps equals SciPy's own bicgstab
    with the V-cycle as its preconditioner M (zero start, the same number of
    steps): the composition of the Krylov method and the V-cycle is pinned by a
    second implementation."""
    op = fe_like(24, seed=14)
    A = op.shifted(0.4 + 3j)
    h = sa_hierarchy(A, strength0(op.K, op.M), max_coarse=16)
    assert len(h.levels) >= 3
    rng = np.random.default_rng(5)
    f = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    e = bicgstab_cycle(A, lambda x: vcycle(h, x), f, steps)
    Mop = spla.LinearOperator(A.shape, matvec=lambda x: vcycle(h, np.asarray(x).ravel()), dtype=complex)
    e_ref, _ = spla.bicgstab(A, f, x0=np.zeros_like(f), rtol=1e-300, atol=0.0, maxiter=steps, M=Mop)
    assert np.linalg.norm(e - e_ref) <= 1e-10 * np.linalg.norm(e_ref)
