"""Pins of the oracle's finite-volume operator (Section 5.1, Eq. phasor1).

Independent routes: Kronecker-product assembly of the homogeneous operator,
the discrete-sine-transform (DST-II) eigenbasis of the mirrored-ghost Dirichlet
Laplacian (closed form), and hand-computed two-cell transmissibilities.
"""
import math

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle


def tridiag_end3(n, lo_dirichlet=True, hi_dirichlet=True):
    """tridiag(-1, 2, -1) with first/last diagonal 3 (zero head, mirrored ghost) or 1 (no flow)."""
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    T[0, 0] = 3.0 if lo_dirichlet else 1.0
    T[n - 1, n - 1] = 3.0 if hi_dirichlet else 1.0
    return T.tocsr()


def kron_operator(shape, h, k0, mask):
    d = len(shape)
    n = int(np.prod(shape))
    out = sp.csr_matrix((n, n))
    for a in range(d):
        q = d - 1 - a
        geo = float(np.prod([h[b] for b in range(d) if b != a])) / h[a]
        mats = [sp.identity(s) for s in shape]
        mats[q] = tridiag_end3(shape[q], mask >> (2 * a) & 1, mask >> (2 * a + 1) & 1)
        term = mats[0]
        for m in mats[1:]:
            term = sp.kron(term, m)
        out = out + k0 * geo * term
    return out.tocsr()


@pytest.mark.parametrize("shape,h,mask", [
    ((6, 9), (2.0, 3.0), 0b1111),
    ((5, 4, 7), (1.0, 0.5, 2.0), 0b111111),
    ((8, 8), (1.0, 1.0), 0b0110),
    ((3, 4, 5), (1.0, 1.0, 1.0), 0b100101),
])
def test_homogeneous_matches_kronecker_form(shape, h, mask):
    k0, s0 = 3e-4, 2e-5
    op = oracle.assemble(shape, h, np.full(shape, k0), np.full(shape, s0), mask)
    ref = kron_operator(shape, h, k0, mask)
    assert abs(op.K - ref).max() <= 1e-13 * abs(ref).max()
    assert np.allclose(op.m_diag, s0 * np.prod(h), rtol=1e-15)


def test_symmetric_and_row_sums_are_boundary_faces():
    rng = np.random.default_rng(3)
    shape, h = (7, 5, 6), (1.0, 2.0, 0.5)
    cond = np.exp(rng.standard_normal(shape))
    op = oracle.assemble(shape, h, cond, np.ones(shape), 0b111111)
    assert abs(op.K - op.K.T).max() == 0.0
    rs = op.K @ np.ones(op.n)
    # interior faces cancel in a row sum; only the cell's boundary faces remain
    bnd = np.zeros(shape)
    d = len(shape)
    for a in range(d):
        q = d - 1 - a
        sl = [slice(None)] * d
        sl[q] = 0
        bnd[tuple(sl)] += op.t_lo[a][tuple(sl)]
        sl[q] = shape[q] - 1
        bnd[tuple(sl)] += op.t_hi[a][tuple(sl)]
    assert np.abs(rs - bnd.ravel()).max() <= 1e-13 * np.abs(rs).max()
    assert np.count_nonzero(bnd) == op.n - 5 * 3 * 4
    # all faces no-flow: constants are in the kernel of K
    op2 = oracle.assemble(shape, h, cond, np.ones(shape), 0)
    assert np.abs(op2.K @ np.ones(op2.n)).max() <= 1e-14 * abs(op2.K).max()


def test_two_cell_transmissibilities_by_hand():
    # grid 1 x 2 (one row, two cells in x), hx = 2, hy = 3, K = (1, 3), all zero-head
    op = oracle.assemble((1, 2), (2.0, 3.0), np.array([[1.0, 3.0]]), np.ones((1, 2)), 0b1111)
    t_int = (3.0 / 2.0) * 2 * 1 * 3 / (1 + 3)            # A_x / h_x * harmonic mean = 2.25
    bx0, bx1 = 2 * 1.0 * 3.0 / 2.0, 2 * 3.0 * 3.0 / 2.0    # x faces: 2 K A_x / h_x
    by0, by1 = 2 * 1.0 * 2.0 / 3.0, 2 * 3.0 * 2.0 / 3.0    # y faces (low and high): 2 K A_y / h_y
    expect = np.array([[t_int + bx0 + 2 * by0, -t_int], [-t_int, t_int + bx1 + 2 * by1]])
    assert np.allclose(op.K.toarray(), expect, rtol=1e-15)
    assert np.allclose(op.m_diag, 6.0)


def dst_eigs(n):
    k = np.arange(1, n + 1)
    return 4.0 * np.sin(math.pi * k / (2.0 * n)) ** 2


def dst_solve(shape, h, k0, s0, sigma, b):
    """(K + sigma M)^{-1} b for a homogeneous medium with zero head on every face, by DST-II."""
    d = len(shape)
    lam = np.zeros(shape)
    for a in range(d):
        q = d - 1 - a
        geo = float(np.prod([h[c] for c in range(d) if c != a])) / h[a]
        e = dst_eigs(shape[q]) * k0 * geo
        bshape = [1] * d
        bshape[q] = shape[q]
        lam = lam + e.reshape(bshape)
    lam = lam + sigma * s0 * float(np.prod(h))
    bh = sfft.dstn(b.reshape(shape), type=2, norm="ortho")
    return sfft.idstn(bh / lam, type=2, norm="ortho").ravel()


@pytest.mark.parametrize("shape,h", [((16, 12), (1.0, 1.5)), ((6, 8, 5), (1.0, 1.0, 2.0))])
def test_dst_closed_form_solve(shape, h):
    k0, s0, sigma = 1e-4, 1e-5, 0.3j
    op = oracle.assemble(shape, h, np.full(shape, k0), np.full(shape, s0), (1 << (2 * len(shape))) - 1)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    x_dst = dst_solve(shape, h, k0, s0, sigma, b)
    r = b - op.shifted(sigma) @ x_dst
    assert np.linalg.norm(r) <= 1e-13 * np.linalg.norm(b)
    x_lu = spla.spsolve(op.shifted(sigma).tocsc(), b)
    assert np.linalg.norm(x_lu - x_dst) <= 1e-12 * np.linalg.norm(x_dst)
