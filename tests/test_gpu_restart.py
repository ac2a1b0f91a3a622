"""Restarted flexible FOM on the GPU (options.restart_len, Section 2.2.2)
against the oracle's restarted solve (oracle/restart.py) and the unrestarted
solve."""
import numpy as np
import pytest

import oracle
from oracle.gmg import Hierarchy, GMGInner
from oracle.restart import restarted_ffom
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, residual_floor

pytestmark = pytest.mark.gpu
EPS = 1e-10


def _problem(shape=(48, 40), n_f=10, seed=71, n_src=1, m_max=60):
    return synth.make_problem(shape, n_f=n_f, periods=(5.0, 3600.0), n_p=3, seed=seed, n_src=n_src, m_max=m_max)


def test_one_cycle_is_the_unrestarted_solve():
    need_gpu()
    pr = _problem()
    s = Solver(pr)
    a = s.solve(variant=fks.FKS_FFOM, inner_tol=EPS)
    assert int(a.steps[0]) < pr.m_max
    b = s.solve(variant=fks.FKS_FFOM, inner_tol=EPS, restart_len=pr.m_max)
    assert a.status == b.status == fks.FKS_OK
    assert np.array_equal(a.X, b.X) and np.array_equal(a.m_j, b.m_j)
    assert np.array_equal(a.res_est, b.res_est) and np.array_equal(a.res_bound, b.res_bound)
    assert np.allclose(a.res_true, b.res_true, rtol=1e-12, atol=1e-18)
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
@pytest.mark.parametrize("cycle", [6, 11])
def test_restarts_match_the_oracle(precision, cycle):
    """Several cycles (multigrid inner solves): every shift certified, the true
    residuals recomputed by the oracle within tol and within the carried
    bound, and x within 1e-6 of the oracle's restarted solution (both solve to
    1e-8 with their own rounding: kappa * tol)."""
    need_gpu()
    pr = _problem(seed=72)
    s = Solver(pr)
    out = s.solve(variant=fks.FKS_FFOM, inner_tol=EPS, restart_len=cycle, precision=precision)
    assert out.status == fks.FKS_OK and np.all(out.shift_status == 0)
    assert int(out.steps[0]) > cycle                 # restarts happened
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    x = out.X[0].T
    tr = oracle.true_residuals(op, b, pr.sigma, x)
    assert np.all(tr <= pr.tol * 1.0001)
    assert np.allclose(tr, out.res_true[0], rtol=1e-6, atol=1e-14)
    assert np.all(out.res_bound[0] <= pr.tol)
    assert np.all(tr <= out.res_bound[0] * (1 + 1e-6) + residual_floor(op, b, pr.sigma, x))
    ref = restarted_ffom(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, cycle, 40,
                         GMGInner(Hierarchy(op, pr.tau_bar), EPS))
    assert np.all(ref.status == 0)
    for j in range(len(pr.sigma)):
        assert np.linalg.norm(x[:, j] - ref.x[:, j]) <= 1e-6 * np.linalg.norm(ref.x[:, j]), j
    assert abs(int(out.steps[0]) - ref.steps) <= cycle
    s.close()


def test_sources_are_independent_and_cycles_can_run_out():
    need_gpu()
    pr = _problem(seed=73, n_src=3)
    s = Solver(pr)
    full = s.solve(variant=fks.FKS_FFOM, inner_tol=EPS, restart_len=8)
    assert full.status == fks.FKS_OK
    solo = s.solve(pr.rhs().T[[1]].copy(), variant=fks.FKS_FFOM, inner_tol=EPS, restart_len=8)
    assert np.array_equal(full.X[1], solo.X[0]) and np.array_equal(full.m_j[1], solo.m_j[0])
    short = s.solve(variant=fks.FKS_FFOM, inner_tol=EPS, restart_len=4, max_restarts=1)
    assert short.status == fks.FKS_NOT_CONVERGED
    assert np.any(short.shift_status == fks.FKS_NOT_CONVERGED)
    assert np.all(short.m_j <= 8)
    s.close()


def test_restart_arguments_rejected():
    need_gpu()
    pr = _problem(shape=(16, 16), n_f=3, seed=74)
    s = Solver(pr)
    with pytest.raises(fks.FksError):
        s.solve(variant=fks.FKS_FGMRES, restart_len=5)
    with pytest.raises(fks.FksError):
        s.solve(variant=fks.FKS_FFOM, restart_len=pr.m_max + 1)
    s.close()
