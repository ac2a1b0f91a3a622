"""Serving: requests of different grids, shift counts and source counts go
through the request loop (memory admission, merging of compatible requests,
concurrent lanes); every result must be bitwise what fks_solve gives the same
request alone."""
import numpy as np
import pytest

from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def make_requests():
    probs = [synth.make_problem((64, 64), n_f=6, periods=(5.0, 3600.0), n_p=3, seed=40, n_src=3, m_max=60),
             synth.make_problem((48, 40), n_f=4, periods=(10.0, 1000.0), n_p=2, seed=41, m_max=60),
             synth.make_problem((12, 16, 16), n_f=5, periods=(5.0, 3600.0), n_p=2, seed=42, m_max=60)]
    solvers = [Solver(p) for p in probs]
    # (problem index, precision, shift subset): requests 0, 3, 5 and 6 share
    # operator, shifts and options and can be merged into one batch
    plan = [(0, fks.FKS_PREC_FP64, None), (1, fks.FKS_PREC_MIXED, None), (2, fks.FKS_PREC_MIXED, None),
            (0, fks.FKS_PREC_FP64, None), (0, fks.FKS_PREC_FP64, 3), (0, fks.FKS_PREC_FP64, None),
            (0, fks.FKS_PREC_FP64, None), (1, fks.FKS_PREC_FP64, None)]
    reqs = []
    for i, (pi, prec, sub) in enumerate(plan):
        p, s = probs[pi], solvers[pi]
        rng = np.random.default_rng(100 + i)
        nr = int(rng.integers(1, 4))
        b = np.zeros((nr, p.n), np.complex128)
        for r in range(nr):
            b[r, rng.integers(0, p.n)] = 1.0 + 0.5j * r
        sigma = p.sigma if sub is None else p.sigma[:sub]
        opts, keep = fks.make_options(tol=p.tol, m_max=p.m_max, precision=prec, inner_tol=1e-10, schedule=p.schedule)
        reqs.append((p, s, fks.ServerRequest(s.op, b, sigma, p.tau_bar, opts, keep, p.n), prec))
    return solvers, reqs


def test_results_alone_and_in_the_mix_are_identical():
    need_gpu()
    solvers, reqs = make_requests()
    srv = fks.fks_server_create(solvers[0].ctx, 4 << 30, lanes=3)
    for _, _, r, _ in reqs:
        fks.fks_server_submit(srv, r)
    for _, _, r, _ in reqs:
        assert fks.fks_server_wait(srv, r.ticket) == fks.FKS_OK
        t0, t1, t2 = fks.fks_server_times(srv, r.ticket)
        assert t0 <= t1 <= t2
    for p, s, r, prec in reqs:
        alone = s.solve(b=r.b, sigma=r.sigma, precision=prec, inner_tol=1e-10)
        assert np.array_equal(alone.X, r.X)
        assert np.array_equal(alone.m_j, r.m_j)
        assert np.array_equal(alone.res_true, r.res_true)
        assert np.all(r.res_true <= p.tol * 1.0001)
    fks.fks_server_destroy(srv)
    for s in solvers:
        s.close()


def test_cancel_a_queued_request():
    need_gpu()
    solvers, reqs = make_requests()
    srv = fks.fks_server_create(solvers[0].ctx, 4 << 30, lanes=1)
    for _, _, r, _ in reqs:
        fks.fks_server_submit(srv, r)
    last = reqs[-1][2]
    try:
        fks.fks_server_cancel(srv, last.ticket)
        cancelled = True
    except fks.FksError:
        cancelled = False                          # already started: nothing to check
    for _, _, r, _ in reqs:
        res = fks.fks_server_wait(srv, r.ticket)
        if cancelled and r is last:
            assert res == fks.FKS_ERR_CANCELLED
        else:
            assert res == fks.FKS_OK
    fks.fks_server_destroy(srv)
    for s in solvers:
        s.close()
