"""Pins of the oracle's multigrid inner solve (the inexact preconditioner of Section 4).

Independent routes: re-discretisation of a homogeneous medium on the coarse
grid (the coarse-face rule must reproduce it exactly), exactness of the
interpolation on linear fields, sparse LU for the solve, and measured
contraction rates.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle.gmg import Hierarchy, GMGInner


@pytest.mark.parametrize("shape,expect", [
    ((512, 512), [(512, 512), (256, 256), (128, 128), (64, 64), (32, 32), (16, 16), (8, 8), (4, 4)]),
    ((12, 20), [(12, 20), (6, 10), (3, 5)]),
    ((10, 10, 10), [(10, 10, 10), (5, 5, 5)]),
    ((16, 8, 4), [(16, 8, 4), (8, 4, 4), (4, 4, 4)]),
])
def test_level_shapes(shape, expect):
    op = oracle.assemble(shape, (1.0,) * len(shape), np.ones(shape), np.ones(shape), (1 << (2 * len(shape))) - 1)
    hier = Hierarchy(op, [1j])
    assert [L.shape for L in hier.levels] == expect


@pytest.mark.parametrize("shape,mask", [((16, 24), 0b1111), ((8, 8, 12), 0b111111), ((16, 16), 0b1001)])
def test_coarse_operator_is_rediscretisation_for_homogeneous_media(shape, mask):
    h = (2.0, 1.0, 0.5)[:len(shape)]
    op = oracle.assemble(shape, h, np.full(shape, 2e-4), np.full(shape, 3e-5), mask)
    hier = Hierarchy(op, [0.1j])
    for L in hier.levels[1:]:
        ref = oracle.assemble(L.shape, L.h, np.full(L.shape, 2e-4), np.full(L.shape, 3e-5), mask)
        assert abs(L.K - ref.K).max() <= 1e-13 * abs(ref.K).max()
        assert np.allclose(L.m, ref.m_diag, rtol=1e-14)


def test_prolongation_exact_on_linear_fields_and_restriction_sums():
    shape = (8, 12)
    op = oracle.assemble(shape, (1.0, 1.0), np.ones(shape), np.ones(shape), 0b1111)
    hier = Hierarchy(op, [1j])
    L0, L1 = hier.levels[0], hier.levels[1]
    # coarse cell centres at 2I+0.5 (fine-index units); fine centres at i
    J, I = np.meshgrid(np.arange(L1.shape[0]), np.arange(L1.shape[1]), indexing="ij")
    coarse = 0.3 * (2 * I + 0.5) - 0.7 * (2 * J + 0.5) + 5.0
    fine = L0.P @ coarse.ravel()
    j, i = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
    exact = 0.3 * i - 0.7 * j + 5.0
    inner = (i > 0) & (i < shape[1] - 1) & (j > 0) & (j < shape[0] - 1)
    assert np.allclose(fine.reshape(shape)[inner], exact[inner], rtol=0, atol=1e-13)
    # next to a zero-head face the coarse ghost is minus the boundary cell:
    # weight 3/4 - 1/4 = 1/2 per such axis
    c = coarse
    fr = fine.reshape(shape)
    assert np.isclose(fr[0, 0], 0.25 * c[0, 0], rtol=1e-14)
    assert np.isclose(fr[0, 1], 0.5 * (0.75 * c[0, 0] + 0.25 * c[0, 1]), rtol=1e-14)
    assert np.isclose(fr[1, 1], 0.75 * (0.75 * c[0, 0] + 0.25 * c[0, 1]) + 0.25 * (0.75 * c[1, 0] + 0.25 * c[1, 1]),
                      rtol=1e-14)
    # restriction sums children
    f = np.arange(op.n, dtype=float)
    rc = L0.R @ f
    assert np.isclose(rc.sum(), f.sum())
    assert np.isclose(rc[0], f[0] + f[1] + f[12] + f[13])


@pytest.mark.parametrize("shape,bound", [((64, 64), 0.2), ((16, 16, 16), 0.2)])
def test_vcycle_contraction_homogeneous(shape, bound):
    d = len(shape)
    op = oracle.assemble(shape, (500.0 / shape[0],) * d, np.full(shape, 1e-4), np.full(shape, 1e-5), (1 << 2 * d) - 1)
    hier = Hierarchy(op, [2j * np.pi / 100])
    v = np.random.default_rng(1).standard_normal(op.n) + 0j
    _, _, p1 = hier.solve(v, 0, 0.0, cycles=2)
    _, _, p2 = hier.solve(v, 0, 0.0, cycles=6)
    rate = (p2 / p1) ** (1.0 / 4.0)
    assert rate <= bound, rate


def test_gmg_solution_matches_sparse_lu_to_eps():
    from paper_1212_3660_gb300 import synth
    pr = synth.make_problem((32, 32), n_f=3, periods=(10.0, 1000.0), n_p=1, seed=9)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    tau = pr.tau_bar[0]
    hier = Hierarchy(op, [tau])
    v = np.random.default_rng(2).standard_normal(op.n) + 1j * np.random.default_rng(3).standard_normal(op.n)
    v /= np.linalg.norm(v)
    for eps in (1e-6, 1e-10):
        z, c, pn = hier.solve(v, 0, eps)
        assert pn <= eps and c < 50
        z_lu = spla.spsolve(op.shifted(tau).tocsc(), v)
        # A (z - z_lu) = -p, so the error is within ||A^{-1}|| * ||p||
        sv_min = np.linalg.svd(op.shifted(tau).toarray(), compute_uv=False).min()
        assert np.linalg.norm(z - z_lu) <= 1.01 * pn / sv_min + 1e-14 * np.linalg.norm(z_lu)


def test_inner_replay_runs_given_cycles():
    shape = (16, 16)
    op = oracle.assemble(shape, (1.0, 1.0), np.ones(shape), np.ones(shape), 0b1111)
    hier = Hierarchy(op, [0.5j])
    inner = GMGInner(hier, 1e-3, replay_cycles=[4, 1])
    v = np.ones(op.n, dtype=complex)
    assert inner(v, 0, 1)[1] == 4
    assert inner(v, 0, 2)[1] == 1
