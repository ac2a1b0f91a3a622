"""GPU parity of the AMG-preconditioned BiCGSTAB inner solve of CSR operators
(Section 6's smoothed-aggregation AMG + BiCGSTAB) against the oracle: the
aggregates of every level bit for bit, the inner solve with a fixed number of
cycles value by value, whole shifted solves under the replay protocol, complex64
cycles free-running, graph = host loop and batch = solo bit for bit, and the
finite-element workload at full size with sampled true residuals."""
import numpy as np
import pytest

import oracle
from oracle.amg import AMGBiCGStabInner, sa_hierarchy, strength0
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from csr_util import csr_arrays, fe_like, sparse_problem
from gpu_util import need_gpu, rel_err, replay_arrays, residual_floor

pytestmark = pytest.mark.gpu


def grid_csr(pr):
    g = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    return oracle.CSROperator(g.K.tocsr(), g.M.tocsr())


def _solver(op, pr, **amg):
    return Solver(pr, csr=csr_arrays(op.K, op.M), amg=amg or True)


@pytest.mark.parametrize("which", ["fe40", "fe64_coarse32", "grid3d"])
def test_aggregates_match_the_oracle_bitwise(which):
    need_gpu()
    kw = {}
    if which == "fe40":
        op = fe_like(40, seed=1)
    elif which == "fe64_coarse32":
        op = fe_like(64, seed=2)
        kw = dict(max_coarse=32)
    else:
        op = grid_csr(synth.make_problem(shape=(12, 20, 10), n_f=2, periods=(5.0, 3600.0), n_p=2, seed=10))
    pr = sparse_problem(op.n)
    s = _solver(op, pr, **kw)
    taus = [0.1j, 10j]
    fks.fks_op_amg_setup(s.op, taus, fks.FKS_PREC_FP64)
    sizes, aggs = fks.fks_op_amg_info(s.op)
    h = sa_hierarchy(op.shifted(taus[0]), strength0(op.K, op.M), **({"max_coarse": kw["max_coarse"]} if kw else {}))
    assert list(sizes) == h.sizes
    assert len(aggs) == len(h.levels) - 1
    for l, a in enumerate(aggs):
        assert np.array_equal(a, h.levels[l].agg.astype(np.int32)), l
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
@pytest.mark.parametrize("cycles", [1, 3])
def test_amg_inner_cycles_match_the_oracle(precision, cycles):
    need_gpu()
    op = fe_like(48, seed=3)
    pr = sparse_problem(op.n)
    s = _solver(op, pr)
    for tau in (0.05j, 5.0 + 20j):
        v = np.random.default_rng(4).standard_normal(op.n) + 1j * np.random.default_rng(5).standard_normal(op.n)
        v /= np.linalg.norm(v)
        z = np.zeros_like(v)
        st, c, pn = fks.fks_precond_apply(s.op, tau, v, z, 1e-10, cycles=cycles, precision=precision)
        zr, cr, pr_ = AMGBiCGStabInner(op, [tau], 1e-10).solve(v, 0, cycles)
        assert c == cr == cycles
        if precision == fks.FKS_PREC_FP64:
            assert rel_err(z, zr) <= 1e-10
            assert abs(pn - pr_) <= 1e-9 * pr_ + 1e-15
        else:
            assert rel_err(z, zr) <= 1e-4
    s.close()


def test_amg_inner_reaches_eps_in_few_cycles():
    need_gpu()
    op = fe_like(64, seed=6)
    pr = sparse_problem(op.n)
    s = _solver(op, pr)
    v = np.random.default_rng(6).standard_normal(op.n) + 0j
    for tau in (0.01j, 1j, 100j):
        for precision in (fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED):
            z = np.zeros_like(v)
            st, c, pn = fks.fks_precond_apply(s.op, tau, v, z, 1e-10, precision=precision)
            assert st == fks.FKS_OK and c <= (6 if precision == fks.FKS_PREC_FP64 else 12), (tau, precision, c)
            r = np.linalg.norm(v - op.shifted(tau) @ z)
            assert pn <= 1e-10 * np.linalg.norm(v) and abs(r - pn) <= 1e-14 * np.linalg.norm(v)
    s.close()


def _replay_check(op, pr, steps=4):
    """Complex128 path under the replay protocol (as for the Jacobi cycles):
    x_j to 1e-8, steps, freeze steps and inner cycle counts exactly."""
    eps = 1e-10
    b = pr.rhs()[:, 0]
    ref = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max,
                               AMGBiCGStabInner(op, pr.tau_bar, eps, steps=steps))
    rc, mj = replay_arrays(pr, [ref])
    s = _solver(op, pr)
    out = s.solve(inner_tol=eps, precision=fks.FKS_PREC_FP64, replay_cycles=rc, replay_mj=mj, inner_steps=steps)
    assert out.status in (fks.FKS_OK, fks.FKS_NOT_CONVERGED, fks.FKS_INNER_NOT_CONVERGED)
    assert np.array_equal(out.m_j[0], ref.m_j)
    assert int(out.steps[0]) == ref.steps
    assert np.array_equal(out.inner_cycles[0, :ref.steps], ref.cycles)
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= 1e-8, j
    tr = oracle.true_residuals(op, b, pr.sigma, out.X[0].T)
    assert np.allclose(out.res_true[0], tr, rtol=1e-6, atol=1e-15)
    assert np.all(out.pnorm[0, :ref.steps] <= 10 * eps) and np.all(ref.pnorm <= eps)
    # the bound holds for the exact Arnoldi relation; the computed one carries
    # rounding of about one residual evaluation per step
    floor = residual_floor(op, b, pr.sigma, out.X[0].T) * ref.steps
    assert np.all(tr <= out.res_bound[0] * (1 + 1e-6) + floor)
    s.close()


@pytest.mark.parametrize("case", ["fe24", "fe40"])
def test_amg_replay_parity_fe(case):
    need_gpu()
    if case == "fe24":
        op = fe_like(24, seed=7)
        pr = sparse_problem(op.n, n_f=8, omega=(1e-2, 1e2), taus=(0.1, 10.0), seed=1, m_max=80)
    else:
        op = fe_like(40, seed=8)
        pr = sparse_problem(op.n, n_f=6, omega=(3e-2, 3e1), taus=(0.3,), seed=2, m_max=80)
    _replay_check(op, pr)


@pytest.mark.parametrize("shape", [(40, 24), (12, 20, 10)])
def test_amg_replay_parity_grid_operators(shape):
    need_gpu()
    kw = dict(shape=shape, n_f=6, periods=(5.0, 3600.0), n_p=2, seed=8)
    if len(shape) == 3:
        kw.update(corr_frac=(0.2, 0.2, 0.05), ss_var=0.25)
    pr = synth.make_problem(m_max=80, **kw)
    _replay_check(grid_csr(pr), pr)


def test_amg_mixed_precision_converges():
    need_gpu()
    op = fe_like(48, seed=9)
    pr = sparse_problem(op.n, n_f=8, seed=1)
    s = _solver(op, pr)
    out = s.solve(inner_tol=1e-10, precision=fks.FKS_PREC_MIXED)
    assert out.status in (fks.FKS_OK, fks.FKS_INNER_NOT_CONVERGED)
    b = pr.rhs()[:, 0]
    tr = oracle.true_residuals(op, b, pr.sigma, out.X[0].T)
    assert np.all(tr <= pr.tol * 1.0001)
    floor = residual_floor(op, b, pr.sigma, out.X[0].T) * int(out.steps[0])
    assert np.all(tr <= out.res_bound[0] * (1 + 1e-6) + floor)
    xd = oracle.direct_solve(op, b, pr.sigma)
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], xd[:, j]) <= 1e-5, j
    s.close()


def test_amg_graph_equals_host_loop_and_batch_equals_solo():
    need_gpu()
    op = fe_like(32, seed=11)
    pr = sparse_problem(op.n, n_f=10, n_src=2, seed=3)
    s = _solver(op, pr)
    g = s.solve(inner_tol=1e-10, launch_mode=0)
    h = s.solve(inner_tol=1e-10, launch_mode=1)
    assert g.status == fks.FKS_OK
    assert np.array_equal(g.X, h.X) and np.array_equal(g.inner_cycles, h.inner_cycles)
    b = pr.rhs()
    for r in range(2):
        tr = oracle.true_residuals(op, b[:, r], pr.sigma, g.X[r].T)
        assert np.all(tr <= pr.tol * 1.0001)
    solo = s.solve(b=np.ascontiguousarray(b[:, 1:2].T), inner_tol=1e-10)
    assert np.array_equal(solo.X[0], g.X[1])
    s.close()


def test_amg_restarted_ffom_is_certified():
    need_gpu()
    op = fe_like(40, seed=12)
    pr = sparse_problem(op.n, n_f=8, seed=5)
    s = _solver(op, pr)
    out = s.solve(inner_tol=1e-10, variant=fks.FKS_FFOM, restart_len=8, max_restarts=40)
    assert out.status == fks.FKS_OK
    b = pr.rhs()[:, 0]
    tr = oracle.true_residuals(op, b, pr.sigma, out.X[0].T)
    assert np.all(tr <= pr.tol * 1.0001)
    s.close()


def test_amg_arguments_and_errors():
    need_gpu()
    op = fe_like(8, seed=0)
    pr = sparse_problem(op.n)
    s = Solver(pr, csr=csr_arrays(op.K, op.M))
    with pytest.raises(fks.FksError):
        fks.fks_op_amg_info(s.op)                         # nothing built yet
    for bad in (dict(max_levels=17), dict(max_coarse=5000), dict(nu=9), dict(max_levels=-1)):
        with pytest.raises(fks.FksError):
            fks.fks_op_amg(s.op, True, **bad)
    with pytest.raises(fks.FksError):
        fks.fks_op_amg_setup(s.op, [1j])                  # AMG not enabled
    fks.fks_op_amg(s.op, True, max_levels=1)
    fks.fks_op_amg_setup(s.op, [1j])
    sizes, aggs = fks.fks_op_amg_info(s.op)
    assert list(sizes) == [op.n] and aggs == []          # one level: the dense inverse
    out = s.solve(inner_tol=1e-10)
    assert out.status == fks.FKS_OK
    # a single-level V-cycle is the exact inverse: one BiCGSTAB step per solve
    assert np.all(out.inner_cycles[0, :int(out.steps[0])] == 1)
    g = synth.make_problem(shape=(8, 8), n_f=2, periods=(5.0, 3600.0), n_p=1, seed=1)
    sg = Solver(g)
    with pytest.raises(fks.FksError):
        fks.fks_op_amg(sg.op, True)
    sg.close()
    s.close()


def test_fe_workload_full_size_sampled():
    """The finite-element workload (256 x 256 nodes, 50 shifts, three taus) with
    AMG cycles in both precisions, in the launch configuration the benchmark
    times: every shift certified; sampled true residuals by the oracle and two
    shifts against a sparse direct solve."""
    need_gpu()
    import scipy.sparse.linalg as spla
    pr = synth.fe_workload()
    op = oracle.CSROperator(pr.K, pr.M)
    b = pr.rhs()[:, 0]
    for precision in (fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED):
        s = Solver(pr, csr=pr.csr_arrays(), amg=True)
        out = s.solve(precision=precision, inner_tol=1e-10, inner_relax=0.003)
        assert out.status == fks.FKS_OK and np.all(out.shift_status == 0)
        assert np.all(out.res_bound <= pr.tol) and np.all(out.res_true <= pr.tol * 1.0001)
        sample = [0, 12, 25, 37, 49]
        X = out.X[0]
        tr = oracle.true_residuals(op, b, pr.sigma[sample], X[sample].T)
        assert np.all(tr <= pr.tol * 1.0001)
        assert np.allclose(tr, out.res_true[0, sample], rtol=1e-6, atol=1e-14)
        for j in (0, 49):
            xd = spla.splu(op.shifted(pr.sigma[j]).tocsc()).solve(b)
            assert np.linalg.norm(X[j] - xd) <= 1e-6 * np.linalg.norm(xd), j
        s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_cooperative_and_stage_amg_cycles_agree_bitwise(precision):
    """One source at 65,536 unknowns runs each AMG-preconditioned cycle as one
    cooperative launch; three sources exceed the resident blocks and run the
    stage kernels. Same rows, same per-row arithmetic: every source of the batch
    is bitwise its solo solve."""
    need_gpu()
    op = fe_like(256, seed=9)
    pr = sparse_problem(op.n, n_f=4, n_src=3, seed=9, m_max=100)
    s = _solver(op, pr)
    batch = s.solve(precision=precision, inner_tol=1e-10, inner_relax=0.003)
    b = pr.rhs().T.copy()
    for r in range(3):
        solo = s.solve(b[[r]], precision=precision, inner_tol=1e-10, inner_relax=0.003)
        assert np.array_equal(batch.X[r], solo.X[0]), r
        assert np.array_equal(batch.inner_cycles[r], solo.inner_cycles[0]), r
        assert np.array_equal(batch.shift_status[r], solo.shift_status[0]), r
        assert np.array_equal(batch.m_j[r], solo.m_j[0]), r
    s.close()
