"""The library's host AMG setup (the C++ that fks_op_amg runs, reached through
fks_amg_host_shape without a GPU) against the oracle's hierarchy: level sizes
and every level's aggregates bit for bit, Jacobi weights to rounding, entry
counts of A_l and P_l, and the argument checks."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle.amg import sa_hierarchy, strength0
from paper_1212_3660_gb300 import fks, synth

from csr_util import fe_like


def level0(K, M, tau):
    """K + tau M on the entries where K or M is nonzero (and the diagonal), sorted columns."""
    S = strength0(K, M).tocsr()
    S.sort_indices()
    A = (sp.csr_matrix(K) + tau * sp.csr_matrix(M)).tocsr()
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    vals = np.asarray(A[rows, S.indices]).ravel().astype(np.complex128)
    return sp.csr_matrix((vals, S.indices.copy(), S.indptr.copy()), shape=S.shape)


def lib_or_skip():
    try:
        fks.lib()
    except Exception as e:  # the library is built by __graft_entry__.build()
        pytest.skip(f"libfks.so not available: {e}")


def grid_op():
    pr = synth.make_problem(shape=(12, 20, 10), n_f=2, periods=(5.0, 3600.0), n_p=2, seed=10)
    g = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    return oracle.CSROperator(g.K.tocsr(), g.M.tocsr())


CASES = [
    ("fe40", lambda: fe_like(40, seed=1), 0.1j, {}),
    ("fe40_high", lambda: fe_like(40, seed=1), 100j, {}),
    ("fe64_coarse32", lambda: fe_like(64, seed=2), 3 - 2j, dict(max_coarse=32)),
    ("fe64_two_levels", lambda: fe_like(64, seed=2), 0.05j, dict(max_levels=2, max_coarse=1)),
    ("grid3d", grid_op, 0.5j, {}),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_host_setup_matches_the_oracle(case):
    lib_or_skip()
    _, make, tau, kw = case
    op = make()
    A0 = level0(op.K, op.M, tau)
    got = fks.fks_amg_host_shape(A0, **kw)
    h = sa_hierarchy(op.shifted(tau), strength0(op.K, op.M), **kw)
    assert list(got["sizes"]) == h.sizes
    assert len(got["agg"]) == len(h.levels) - 1
    for l, a in enumerate(got["agg"]):
        assert np.array_equal(a, h.levels[l].agg), l
    assert np.allclose(got["omega"], [lv.omega for lv in h.levels], rtol=1e-14, atol=0)
    assert got["nnz_a"][0] == A0.nnz
    for l in range(len(h.levels) - 1):
        # structural products: at least the oracle's entries (SciPy drops exact zeros)
        assert got["nnz_p"][l] >= h.levels[l].P.nnz
        assert got["nnz_a"][l + 1] >= h.levels[l + 1].A.nnz
    assert got["nnz_p"][-1] == 0


def test_host_setup_rejects_bad_input():
    lib_or_skip()
    op = fe_like(6, seed=0)
    A0 = level0(op.K, op.M, 1j)
    with pytest.raises(fks.FksError):
        fks.fks_amg_host_shape(A0, max_levels=17)
    bad = A0.copy()
    bad.data[0] = np.nan
    with pytest.raises(fks.FksError):
        fks.fks_amg_host_shape(bad)
    z = A0.tolil()
    z[3, 3] = 0.0                      # a stored zero on the diagonal
    z = z.tocsr()
    z.sort_indices()
    with pytest.raises(fks.FksError) as e:
        fks.fks_amg_host_shape(sp.csr_matrix((z.data, z.indices, z.indptr), shape=z.shape))
    assert "diagonal" in str(e.value)
    unsorted = A0.copy()
    r = unsorted.indptr[5]
    unsorted.indices[r], unsorted.indices[r + 1] = unsorted.indices[r + 1], unsorted.indices[r]
    with pytest.raises(fks.FksError):
        fks.fks_amg_host_shape(unsorted)
