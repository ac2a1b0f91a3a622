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


@pytest.mark.parametrize("shape,expect", [
    # even halving would stop at 125^2, 25^3 and 35 x 45 (> 1024 cells): odd
    # sides then halve too, rounding up, while a level has more than 1024 cells
    ((250, 250), [(250, 250), (125, 125), (63, 63), (32, 32), (16, 16), (8, 8), (4, 4)]),
    ((100, 100, 100), [(100, 100, 100), (50, 50, 50), (25, 25, 25), (13, 13, 13), (7, 7, 7)]),
    ((70, 90), [(70, 90), (35, 45), (18, 23), (9, 23)]),
    # an even-halving hierarchy that ends at <= 1024 cells is kept as it is
    ((2048, 5), [(2048, 5), (1024, 5), (512, 5), (256, 5), (128, 5), (64, 5), (32, 5), (16, 5), (8, 5), (4, 5)]),
])
def test_level_shapes_ragged(shape, expect):
    op = oracle.assemble(shape, (1.0,) * len(shape), np.ones(shape), np.ones(shape), (1 << (2 * len(shape))) - 1)
    hier = Hierarchy(op, [1j])
    assert [L.shape for L in hier.levels] == expect
    assert hier.levels[-1].n <= 1024


@pytest.mark.parametrize("shape", [(70, 90), (30, 50, 50), (289, 40)])
def test_ragged_levels_homogeneous_geometry(shape):
    """Coarse levels of a homogeneous medium on ragged hierarchies are the
    two-point flux discretisation on the coarse cells, whose widths are the
    numbers of finest cells they cover (1D: children summed; the one-child cell
    of an odd axis keeps its child's width): a face along axis q joins cells of
    widths W1, W2 over the distance (W1 + W2) h_q / 2 and has the area of the
    other axes' widths; a zero-head face sits half a width away; storage is
    S_s times the cell volume. R sums each fine cell into exactly one coarse
    cell, and with no-flow faces every row of P sums to 1."""
    d = len(shape)
    h = (2.0, 1.0, 0.5)[:d]          # per grid axis a (x first)
    K0, S0 = 2e-4, 3e-5
    for mask in (0, (1 << 2 * d) - 1):
        op = oracle.assemble(shape, h, np.full(shape, K0), np.full(shape, S0), mask)
        hier = Hierarchy(op, [0.1j])
        widths = [np.ones(n) for n in shape]   # per numpy axis q, in finest cells
        ragged_seen = False
        for F, L in zip(hier.levels[:-1], hier.levels[1:]):
            for q in range(d):
                if L.shape[q] < F.shape[q]:
                    w = widths[q]
                    ragged_seen |= len(w) % 2 == 1
                    widths[q] = np.array([w[2 * I:2 * I + 2].sum() for I in range(L.shape[q])])
            hq = [h[d - 1 - q] for q in range(d)]     # spacing of numpy axis q
            grids = np.meshgrid(*[widths[q] * hq[q] for q in range(d)], indexing="ij")
            vol = np.prod(grids, axis=0)
            for a in range(d):
                q = d - 1 - a
                area = vol / grids[q]
                W = widths[q] * hq[q]
                shp = [1] * d
                shp[q] = L.shape[q]
                Wl = np.concatenate([[np.nan], W[:-1]]).reshape(shp)   # low neighbour's width
                Wh = np.concatenate([W[1:], [np.nan]]).reshape(shp)    # high neighbour's width
                Wc = W.reshape(shp)
                lo = K0 * area / ((Wl + Wc) / 2)
                hi = K0 * area / ((Wc + Wh) / 2)
                first = [slice(None)] * d
                first[q] = 0
                last = [slice(None)] * d
                last[q] = L.shape[q] - 1
                lo[tuple(first)] = (K0 * area / (Wc / 2))[tuple(first)] if (mask >> (2 * a)) & 1 else 0.0
                hi[tuple(last)] = (K0 * area / (Wc / 2))[tuple(last)] if (mask >> (2 * a + 1)) & 1 else 0.0
                assert np.allclose(L.t_lo[a], lo, rtol=1e-13, atol=0), (L.shape, a)
                assert np.allclose(L.t_hi[a], hi, rtol=1e-13, atol=0), (L.shape, a)
            assert np.allclose(L.m.reshape(L.shape), S0 * vol, rtol=1e-13)
            assert np.array_equal(np.asarray(F.R.sum(axis=0)).ravel(), np.ones(F.n))
            if mask == 0:
                assert np.allclose(np.asarray(F.P.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-15)
        assert ragged_seen


@pytest.mark.parametrize("shape", [(66, 70), (18, 22, 26), (289, 289)])
def test_ragged_hierarchy_contracts_and_solves(shape):
    """Measured V-cycle contraction on ragged hierarchies for every tau of a
    synthetic log-normal aquifer (a wrong child, face or weight at the one-child
    cells shows as a slow or divergent cycle; 289^2 keeps one-cell-wide edge
    cells through four levels), and the solve against sparse LU."""
    from paper_1212_3660_gb300 import synth
    d = len(shape)
    pr = synth.make_problem(shape, n_f=10, periods=(5.0, 3600.0), n_p=3, seed=20000)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    hier = Hierarchy(op, pr.tau_bar)
    v = np.random.default_rng(1).standard_normal(op.n) + 0j
    for p in range(len(pr.tau_bar)):
        _, _, p1 = hier.solve(v, p, 0.0, cycles=2)
        _, _, p2 = hier.solve(v, p, 0.0, cycles=6)
        assert (p2 / p1) ** 0.25 <= 0.25, p
    tau = pr.tau_bar[0]
    v /= np.linalg.norm(v)
    z, c, pn = hier.solve(v, 0, 1e-10)
    assert pn <= 1e-10
    A = op.shifted(tau).tocsc()
    assert [L.n for L in hier.levels][-1] <= 1024 and any(
        F.shape[q] % 2 == 1 and L.shape[q] < F.shape[q]
        for F, L in zip(hier.levels[:-1], hier.levels[1:]) for q in range(d))
    z_lu = spla.spsolve(A, v)
    assert np.linalg.norm(z - z_lu) <= 1e-6 * np.linalg.norm(z_lu)


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
