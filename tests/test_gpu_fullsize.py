"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark times (CUDA graph, autotuned thresholds, relaxed
inner tolerance l = 0.003): every shift certified, and sampled outputs checked
one by one against the oracle (true residuals with the oracle's own sparse K and
M; for 512 x 512 also the sparse-LU solution of sampled shifts)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, residual_floor

pytestmark = pytest.mark.gpu

RELAX = 0.003
EPS = 1e-10


def _solve_like_bench(pr, precision, device_out=False):
    s = Solver(pr)
    fks.fks_op_autotune(s.op, precision, complex(pr.tau_bar[len(pr.tau_bar) // 2]))
    out = s.solve(precision=precision, inner_tol=EPS, inner_relax=RELAX, launch_mode=0, device_out=device_out)
    return s, out


def _check_certified(pr, out):
    assert out.status == fks.FKS_OK
    assert np.all(out.shift_status == 0)
    assert np.all(out.res_bound <= pr.tol) and np.all(out.res_true <= pr.tol * 1.0001)


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_2d_512x512_200_shifts(precision):
    need_gpu()
    pr = synth.workload(2, m_max=100)
    s, out = _solve_like_bench(pr, precision)
    _check_certified(pr, out)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    sample = list(range(0, 200, 20)) + [199]
    X = out.X[0]
    tr = oracle.true_residuals(op, b, pr.sigma[sample], X[sample].T)
    assert np.all(tr <= pr.tol * 1.0001)
    assert np.allclose(tr, out.res_true[0, sample], rtol=1e-6, atol=1e-14)
    floor = residual_floor(op, b, pr.sigma[sample], X[sample].T)
    assert np.all(tr <= out.res_bound[0, sample] * (1 + 1e-6) + floor)
    for j in (0, 199):   # highest and lowest frequency
        xd = spla.splu(op.shifted(pr.sigma[j]).tocsc()).solve(b)
        assert np.linalg.norm(X[j] - xd) <= 1e-6 * np.linalg.norm(xd), j
    s.close()


def test_3d_128_cubed_mixed_sampled():
    """128^3 (2.1M cells), anisotropic field, lognormal storage, 200 shifts, four
    tau, complex64 cycles: sampled true residuals by the oracle."""
    need_gpu()
    pr = synth.workload(3, m_max=100)
    s, out = _solve_like_bench(pr, fks.FKS_PREC_MIXED, device_out=True)
    _check_certified(pr, out)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    sample = [0, 67, 133, 199]
    Xs = out.X[0, sample].cpu().numpy()
    tr = oracle.true_residuals(op, b, pr.sigma[sample], Xs.T)
    assert np.all(tr <= pr.tol * 1.0001)
    assert np.allclose(tr, out.res_true[0, sample], rtol=1e-6, atol=1e-14)
    s.close()


def test_3d_96_cubed_batched_sources_sampled():
    """The batched configuration's grid (96^3, 100 shifts, four tau) with 8 of
    its 64 wells in one lockstep batch, complex64 cycles: sampled (source, shift)
    true residuals by the oracle."""
    need_gpu()
    pr = synth.workload(4, m_max=100)
    pr.src_cells = pr.src_cells[:8].copy()
    s, out = _solve_like_bench(pr, fks.FKS_PREC_MIXED, device_out=True)
    _check_certified(pr, out)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    rhs = pr.rhs()
    for r in (0, 3, 7):
        sample = [0, 50, 99]
        Xs = out.X[r, sample].cpu().numpy()
        tr = oracle.true_residuals(op, rhs[:, r], pr.sigma[sample], Xs.T)
        assert np.all(tr <= pr.tol * 1.0001), r
        assert np.allclose(tr, out.res_true[r, sample], rtol=1e-6, atol=1e-14), r
    s.close()
