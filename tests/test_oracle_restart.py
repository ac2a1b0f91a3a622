"""Pins of the restarted flexible FOM (oracle/restart.py): the unrestarted
solve when one cycle suffices, collinearity of the shifted residuals at a
restart (Eq. fomresidualsimplified), convergence to the direct solutions
across several restarts with exact inner solves, and the certified bound with
inexact (multigrid) inner solves."""
import numpy as np
import pytest

import oracle
from oracle.fgmres import OK
from oracle.gmg import Hierarchy, GMGInner
from oracle.restart import restarted_ffom
from paper_1212_3660_gb300 import synth

from gpu_util import residual_floor


def _problem(shape=(20, 24), n_f=6, seed=61, n_p=3):
    pr = synth.make_problem(shape, n_f=n_f, periods=(5.0, 3600.0), n_p=n_p, seed=seed)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    return pr, op, pr.rhs()[:, 0]


def test_one_long_cycle_is_the_unrestarted_solve():
    pr, op, b = _problem()
    ex = oracle.ExactInner(op, pr.tau_bar)
    ref = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-9, 80, ex, variant="ffom")
    res = restarted_ffom(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-9, 80, 3, ex)
    assert res.cycles == 1 and res.steps == ref.steps
    assert np.array_equal(res.m_j, ref.m_j) and np.array_equal(res.status, ref.status)
    assert np.max(np.abs(res.x - ref.x)) <= 1e-12 * np.max(np.abs(ref.x))


def test_residuals_are_collinear_at_a_restart():
    """After one cycle of m steps (exact inner solves) the true residual of every
    shift not yet converged is C_j v_{m+1}."""
    pr, op, b = _problem(seed=62)
    ex = oracle.ExactInner(op, pr.tau_bar)
    m = 6
    res = restarted_ffom(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-12, m, 1, ex)
    one = oracle.shifted_solve(op, b / np.linalg.norm(b), pr.sigma, pr.tau_bar, pr.schedule, 1e-12, m, ex,
                               variant="ffom", keep_basis=True)
    v = one.V[:, m]
    open_ = [j for j in range(len(pr.sigma)) if res.status[j] != OK]
    assert len(open_) >= 3
    for j in open_:
        s = pr.sigma[j]
        r = b - op.shifted(s) @ res.x[:, j]
        c = np.vdot(v, r)
        assert np.linalg.norm(r - c * v) <= 1e-9 * np.linalg.norm(r), j
        assert abs(abs(c) / np.linalg.norm(b) - res.res_est[j]) <= 1e-8 * res.res_est[j], j


@pytest.mark.parametrize("cycle_len", [4, 7, 12])
def test_restarts_converge_to_direct_solutions(cycle_len):
    pr, op, b = _problem(seed=63)
    ex = oracle.ExactInner(op, pr.tau_bar)
    res = restarted_ffom(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-9, cycle_len, 60, ex)
    assert res.cycles > 1 and np.all(res.status == OK)
    tr = oracle.true_residuals(op, b, pr.sigma, res.x)
    assert np.all(tr <= 1e-9 * 1.0001)
    assert np.all(np.abs(tr - res.res_est) <= 1e-6 * np.maximum(tr, 1e-14) + 1e-15)
    xd = oracle.direct_solve(op, b, pr.sigma)
    for j in range(len(pr.sigma)):
        assert np.linalg.norm(res.x[:, j] - xd[:, j]) <= 1e-6 * np.linalg.norm(xd[:, j])
    # the step at which a shift is certified is a step of the whole run
    assert np.all(res.m_j <= res.steps)


def test_inexact_inner_solves_stay_certified():
    """With multigrid inner solves the unseen errors of every cycle are carried:
    the true residual stays within the accumulated bound, itself within tol."""
    pr, op, b = _problem(shape=(32, 32), seed=64)
    inner = GMGInner(Hierarchy(op, pr.tau_bar), 1e-10)
    res = restarted_ffom(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-8, 6, 60, inner)
    assert res.cycles > 1 and np.all(res.status == OK)
    tr = oracle.true_residuals(op, b, pr.sigma, res.x)
    assert np.all(res.res_bound <= 1e-8)
    assert np.all(tr <= res.res_bound * (1 + 1e-6) + residual_floor(op, b, pr.sigma, res.x))
