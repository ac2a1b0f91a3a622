"""Assembly x_j = Z_{m_j} y_j (Algorithm 4) on the tensor cores against the FP64
kernel on the same solve. The Arnoldi iteration is the same in both runs (the
assembly comes after it), so the two X differ only by how the products are
rounded: both errors are of order K' 2^-53 max|Z_i.| max|Y_.j| per entry
(K' = 2 x steps), which for these solves is below 1e-12 ||x_j||."""
import numpy as np
import pytest

import oracle
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, rel_err, oracle_op

pytestmark = pytest.mark.gpu

CASES = [
    dict(shape=(16, 16), n_f=3, periods=(10.0, 1000.0), n_p=1, seed=3),                 # 2 row tiles, 1 column tile
    dict(shape=(40, 24), n_f=7, periods=(5.0, 3600.0), n_p=3, seed=8),                  # ragged rows, odd n_f
    dict(shape=(64, 64), n_f=40, periods=(5.0, 3600.0), n_p=3, seed=5, n_src=3),        # 3 column tiles, 3 sources
    dict(shape=(12, 20, 10), n_f=17, periods=(5.0, 3600.0), n_p=2, seed=10, ss_var=0.25),  # 3D
    # 424 row tiles x 2 sources: more (source, row tile) items than CTAs, so
    # each persistent CTA runs several items through its ring and both TMEM sets
    dict(shape=(256, 212), n_f=23, periods=(5.0, 3600.0), n_p=3, seed=6, n_src=2),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["shape"])))
@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_tensor_core_assembly_matches_fp64_kernel(case, precision):
    need_gpu()
    pr = synth.make_problem(m_max=60, **case)
    s = Solver(pr)
    a = s.solve(inner_tol=1e-10, precision=precision, assembly=1)
    b = s.solve(inner_tol=1e-10, precision=precision, assembly=0)
    assert a.status == b.status == fks.FKS_OK
    assert np.array_equal(a.m_j, b.m_j) and np.array_equal(a.steps, b.steps)
    assert np.array_equal(a.inner_cycles, b.inner_cycles)
    for r in range(a.X.shape[0]):
        for j in range(a.X.shape[1]):
            assert rel_err(b.X[r, j], a.X[r, j]) <= 1e-12, (r, j)
    # the true residuals of the tensor-core x_j, recomputed by the oracle's operator
    op = oracle_op(pr)
    rhs = pr.rhs()
    for r in range(b.X.shape[0]):
        tr = oracle.true_residuals(op, rhs[:, r], pr.sigma, b.X[r].T)
        assert np.all(tr <= pr.tol * 1.0001)
        assert np.allclose(b.res_true[r], tr, rtol=1e-6, atol=1e-15)
    s.close()


def test_tensor_core_assembly_is_deterministic_and_graph_equals_host():
    need_gpu()
    pr = synth.make_problem((48, 48), n_f=12, periods=(5.0, 3600.0), n_p=3, seed=16, n_src=2, m_max=60)
    s = Solver(pr)
    g = s.solve(inner_tol=1e-10, launch_mode=0)
    h = s.solve(inner_tol=1e-10, launch_mode=1)
    g2 = s.solve(inner_tol=1e-10, launch_mode=0)
    assert np.array_equal(g.X, h.X) and np.array_equal(g.X, g2.X)
    s.close()


def test_bad_assembly_option_rejected():
    need_gpu()
    pr = synth.make_problem((16, 16), n_f=3, periods=(10.0, 1000.0), n_p=1, seed=2)
    s = Solver(pr)
    with pytest.raises(fks.FksError) as e:
        s.solve(assembly=2)
    assert e.value.status == fks.FKS_ERR_ARG
    s.close()
