"""Serving: requests of different grids, shift counts and source counts go
through the request loop (memory admission, continuous batching, concurrent
lanes); every result must be bitwise what fks_solve gives the same request
alone. Requests that arrive while a batch runs join it at an Arnoldi-step
boundary; running requests can be cancelled or time out; a workspace that
cannot be allocated fails its requests and leaks nothing."""
import time

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
    # operator, shifts and options and can share one batch
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


def _alone_equal(s, r, prec, tol, inner_tol=1e-10):
    alone = s.solve(b=r.b, sigma=r.sigma, precision=prec, inner_tol=inner_tol)
    assert np.array_equal(alone.X, r.X)
    assert np.array_equal(alone.m_j, r.m_j)
    assert np.array_equal(alone.res_true, r.res_true)
    assert np.all(r.res_true <= tol * 1.0001)


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
        _alone_equal(s, r, prec, p.tol)
    assert fks.fks_server_launches(srv) > 0
    fks.fks_server_destroy(srv)
    for s in solvers:
        s.close()


def test_page_locked_output_arrays_reused_across_requests():
    """Requests on two operators whose x_j go into the caller's page-locked
    arrays (out=), submitted twice with the same arrays, as the mixed 2D batch
    of the bench does: both rounds give the bits of each request alone."""
    need_gpu()
    import torch
    probs = [synth.make_problem((64, 64), n_f=6, periods=(5.0, 3600.0), n_p=3, seed=46, m_max=60),
             synth.make_problem((96, 96), n_f=5, periods=(5.0, 3600.0), n_p=4, seed=47, m_max=60)]
    solvers = [Solver(p) for p in probs]
    keep_t = [torch.empty((1, len(p.sigma), p.n), dtype=torch.complex128, pin_memory=True) for p in probs]
    outs = [t.numpy() for t in keep_t]
    srv = fks.fks_server_create(solvers[0].ctx, 2 << 30, lanes=2)
    for rnd in range(2):
        reqs = []
        for p, s, out in zip(probs, solvers, outs):
            out.fill(np.nan)
            opts, keep = fks.make_options(tol=p.tol, m_max=p.m_max, precision=fks.FKS_PREC_MIXED, inner_tol=1e-10,
                                          schedule=p.schedule)
            r = fks.ServerRequest(s.op, p.rhs().T.copy(), p.sigma, p.tau_bar, opts, keep, p.n, out=out)
            fks.fks_server_submit(srv, r)
            reqs.append(r)
        for g, (p, s, r) in enumerate(zip(probs, solvers, reqs)):
            assert fks.fks_server_wait(srv, r.ticket) == fks.FKS_OK, rnd
            assert r.X is outs[g]
            _alone_equal(s, r, fks.FKS_PREC_MIXED, p.tol)
    fks.fks_server_destroy(srv)
    for s in solvers:
        s.close()


def _long_problem():
    # 256^2, 200 shifts, tolerance 1e-10: tens of Arnoldi steps
    return synth.make_problem((256, 256), n_f=200, periods=(5.0, 3600.0), n_p=3, seed=44, m_max=100, tol=1e-10)


def _request(p, s, src_cells, prec=fks.FKS_PREC_MIXED, **kw):
    b = np.zeros((len(src_cells), p.n), np.complex128)
    for r, c in enumerate(src_cells):
        b[r, c] = 1.0
    opts, keep = fks.make_options(tol=p.tol, m_max=p.m_max, precision=prec, inner_tol=1e-12, schedule=p.schedule)
    return fks.ServerRequest(s.op, b, p.sigma, p.tau_bar, opts, keep, p.n, **kw)


def _wait_started(srv, r, limit=60.0):
    t_end = time.time() + limit
    while time.time() < t_end:
        if fks.fks_server_times(srv, r.ticket)[1] > 0:
            return
        time.sleep(0.0005)
    raise AssertionError("request did not start")


def test_late_request_joins_a_running_batch():
    """One lane: a compatible request submitted while another runs is admitted
    into the running batch's free slots at a step boundary (it starts before the
    first one ends, which one lane could not do otherwise), and its results are
    bitwise those of its solve alone."""
    need_gpu()
    p = _long_problem()
    s = Solver(p)
    srv = fks.fks_server_create(s.ctx, 8 << 30, lanes=1)
    a = _request(p, s, [p.n // 2 + 128])
    b = _request(p, s, [1000, 40000])
    fks.fks_server_submit(srv, a)
    _wait_started(srv, a)
    fks.fks_server_submit(srv, b)
    assert fks.fks_server_wait(srv, a.ticket) == fks.FKS_OK
    assert fks.fks_server_wait(srv, b.ticket) == fks.FKS_OK
    ta, tb = fks.fks_server_times(srv, a.ticket), fks.fks_server_times(srv, b.ticket)
    assert tb[1] < ta[2], (ta, tb)           # admitted while the first request was running
    _alone_equal(s, b, fks.FKS_PREC_MIXED, p.tol, 1e-12)
    _alone_equal(s, a, fks.FKS_PREC_MIXED, p.tol, 1e-12)
    fks.fks_server_destroy(srv)
    s.close()


def test_cancel_and_timeout_of_running_requests():
    """A running request stops at the next step boundary when cancelled
    (FKS_ERR_CANCELLED) or when its time limit passes (FKS_ERR_TIMEOUT); the
    lane and its budget stay usable: a later request completes normally."""
    need_gpu()
    p = _long_problem()
    s = Solver(p)
    srv = fks.fks_server_create(s.ctx, 8 << 30, lanes=1)
    r1 = _request(p, s, [p.n // 2 + 128])
    fks.fks_server_submit(srv, r1)
    _wait_started(srv, r1)
    fks.fks_server_cancel(srv, r1.ticket)
    assert fks.fks_server_wait(srv, r1.ticket) == fks.FKS_ERR_CANCELLED
    with pytest.raises(fks.FksError):
        fks.fks_server_cancel(srv, r1.ticket)     # already finished
    r2 = _request(p, s, [5000], timeout_s=1e-4)
    fks.fks_server_submit(srv, r2)
    assert fks.fks_server_wait(srv, r2.ticket) == fks.FKS_ERR_TIMEOUT
    r3 = _request(p, s, [7000], with_x=False)
    fks.fks_server_submit(srv, r3)
    assert fks.fks_server_wait(srv, r3.ticket) == fks.FKS_OK
    assert r3.X is None and np.all(r3.res_true <= p.tol * 1.0001)
    fks.fks_server_destroy(srv)
    s.close()


def test_injected_allocation_failure_fails_the_batch_and_leaks_nothing():
    """A workspace reservation that fails as cudaMalloc does when the device is
    out of memory (an injected failure, on the host) ends the batch's request
    with FKS_ERR_OOM; the budget it held is released, so the next request, which
    is larger than the whole budget, runs (it may only while nothing else holds
    any: a leak would leave it queued)."""
    need_gpu()
    p = synth.make_problem((96, 96), n_f=8, periods=(5.0, 3600.0), n_p=2, seed=45, m_max=60)
    s = Solver(p)
    r1 = _request(p, s, [100])
    # a one-byte budget: a request runs only while nothing else holds any of it
    srv = fks.fks_server_create(s.ctx, 1, lanes=1)
    fks.fks_debug_fail_allocs(1)
    try:
        fks.fks_server_submit(srv, r1)
        assert fks.fks_server_wait(srv, r1.ticket) == fks.FKS_ERR_OOM
    finally:
        fks.fks_debug_fail_allocs(0)
    r2 = _request(p, s, [200, 300])
    fks.fks_server_submit(srv, r2)
    t_end = time.time() + 60
    done = False
    while time.time() < t_end and not done:
        done, res = fks.fks_server_poll(srv, r2.ticket)
        time.sleep(0.001)
    assert done and res == fks.FKS_OK
    fks.fks_server_destroy(srv)
    s.close()


def test_request_larger_than_the_budget_runs_source_by_source():
    """With room for one source at a time (a one-byte budget: a batch gets one
    slot), a request's sources are admitted in turn as slots free up; each is
    delivered as it finishes and the results equal the solve alone."""
    need_gpu()
    p = synth.make_problem((80, 64), n_f=12, periods=(5.0, 3600.0), n_p=3, seed=46, m_max=60)
    s = Solver(p)
    srv = fks.fks_server_create(s.ctx, 1, lanes=2)
    r = _request(p, s, [10, 2000, 4000])
    fks.fks_server_submit(srv, r)
    assert fks.fks_server_wait(srv, r.ticket) == fks.FKS_OK
    _alone_equal(s, r, fks.FKS_PREC_MIXED, p.tol, 1e-12)
    fks.fks_server_destroy(srv)
    s.close()
