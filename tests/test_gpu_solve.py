"""GPU parity of the whole flexible shifted solve against the oracle.

Replay protocol: the oracle's inner-cycle counts and freeze steps m_j are fed
to the GPU (replay mode), so both sides execute the same sequence of
operations and differ only by rounding; every x_j must then agree to 1e-8
relative (complex128 path). Free-running solves are checked by the true
residual, recomputed on the CPU with the oracle's operator.
"""
import numpy as np
import pytest

import oracle
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, oracle_run, replay_arrays, rel_err, residual_floor

pytestmark = pytest.mark.gpu

CASES = [
    dict(shape=(64, 64), n_f=10, periods=(10.0, 1000.0), n_p=1, seed=1),            # 64x64 workload
    dict(shape=(40, 24), n_f=7, periods=(5.0, 3600.0), n_p=3, seed=8),               # ragged, 3 taus
    dict(shape=(16, 16, 16), n_f=6, periods=(5.0, 3600.0), n_p=2, seed=9),           # 3D
    dict(shape=(12, 20, 10), n_f=5, periods=(5.0, 3600.0), n_p=4, seed=10, corr_frac=(0.2, 0.2, 0.05),
         ss_var=0.25),                                                               # aniso + lognormal S_s
    dict(shape=(30, 18), n_f=4, periods=(10.0, 1000.0), n_p=2, seed=12, dirichlet_mask=0b0011),  # no-flow y
    # even halving would end at 33 x 35 and 9 x 11 x 13 (> 1024 cells): ragged halving of odd sides
    dict(shape=(66, 70), n_f=5, periods=(5.0, 3600.0), n_p=2, seed=14),
    dict(shape=(18, 22, 26), n_f=4, periods=(5.0, 3600.0), n_p=2, seed=15),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["shape"])))
@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_replay_parity(case, precision):
    need_gpu()
    pr = synth.make_problem(m_max=80, **case)
    eps = 1e-10
    op, ref = oracle_run(pr, eps)
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    out = s.solve(inner_tol=eps, precision=precision, replay_cycles=rc, replay_mj=mj)
    assert out.status in (fks.FKS_OK, fks.FKS_NOT_CONVERGED)
    assert np.array_equal(out.m_j[0], ref.m_j)
    assert int(out.steps[0]) == ref.steps
    tol = 1e-8 if precision == fks.FKS_PREC_FP64 else 1e-6
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= tol, j
    # the GPU's own true residual equals the oracle's recomputation
    tr = oracle.true_residuals(op, pr.rhs()[:, 0], pr.sigma, out.X[0].T)
    assert np.allclose(out.res_true[0], tr, rtol=1e-6, atol=1e-15)
    assert np.allclose(out.res_bound[0], ref.res_bound, rtol=1e-5, atol=1e-4 * pr.tol)
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_free_running_reaches_tolerance(precision):
    need_gpu()
    pr = synth.workload(1)
    s = Solver(pr)
    out = s.solve(precision=precision, inner_tol=1e-10)
    assert out.status == fks.FKS_OK
    op, ref = oracle_run(pr, 1e-10)
    tr = oracle.true_residuals(op, pr.rhs()[:, 0], pr.sigma, out.X[0].T)
    assert np.all(tr <= pr.tol * 1.0001)
    assert np.all(out.res_bound[0] <= pr.tol)
    floor = residual_floor(op, pr.rhs()[:, 0], pr.sigma, out.X[0].T)
    assert np.all(tr <= out.res_bound[0] * (1 + 1e-6) + floor)      # Eq. trueresidual holds
    # free-running vs oracle: within kappa * tol, reported not gated at 1e-8
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= 1e-5
    s.close()


def test_multiple_sources_are_independent_processes():
    need_gpu()
    pr = synth.make_problem((32, 32), n_f=5, periods=(5.0, 3600.0), n_p=2, seed=14, n_src=3, m_max=60)
    eps = 1e-10
    refs = [oracle_run(pr, eps, src=r)[1] for r in range(3)]
    rc, mj = replay_arrays(pr, refs)
    s = Solver(pr)
    out = s.solve(inner_tol=eps, replay_cycles=rc, replay_mj=mj)
    for r in range(3):
        for j in range(len(pr.sigma)):
            assert rel_err(out.X[r, j], refs[r].x[:, j]) <= 1e-8
    # solo solve of source 1 gives the same result as inside the batch
    b1 = pr.rhs().T[1:2].copy()
    solo = s.solve(b=b1, inner_tol=eps, replay_cycles=rc[1:2], replay_mj=mj[1:2])
    assert np.array_equal(solo.X[0], out.X[1])
    s.close()


def test_ffom_variant_replay():
    need_gpu()
    pr = synth.make_problem((24, 24), n_f=5, periods=(10.0, 1000.0), n_p=2, seed=15, m_max=60)
    eps = 1e-10
    op, ref = oracle_run(pr, eps, variant="ffom")
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    out = s.solve(inner_tol=eps, variant=fks.FKS_FFOM, replay_cycles=rc, replay_mj=mj)
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= 1e-8
    s.close()


def test_zero_rhs_gives_zero_solution():
    need_gpu()
    pr = synth.make_problem((16, 16), n_f=3, periods=(10.0, 1000.0), n_p=1, seed=2)
    s = Solver(pr)
    out = s.solve(b=np.zeros((1, pr.n), np.complex128))
    assert out.status == fks.FKS_OK
    assert np.all(out.X == 0) and np.all(out.m_j == 0)
    s.close()


def test_sigma_equal_tau_and_single_mode_converge_in_one_step():
    need_gpu()
    pr = synth.make_problem((20, 20), n_f=2, periods=(10.0, 1000.0), n_p=1, seed=2, homogeneous=True)
    s = Solver(pr)
    tau = pr.tau_bar
    out = s.solve(sigma=np.array([tau[0], 0.5 * tau[0]]), inner_tol=1e-12)
    assert out.m_j[0, 0] == 1
    # one sine mode of the homogeneous box is an eigenvector of K and M: every
    # shift is solved exactly from the first basis vector (Section 3, breakdown)
    ii, jj = np.meshgrid(np.arange(1, 21), np.arange(1, 21), indexing="xy")
    kx, ky = 3, 2
    mode = (np.sin(np.pi * kx * (ii - 0.5) / 20) * np.sin(np.pi * ky * (jj - 0.5) / 20)).ravel()
    k0, s0 = float(pr.cond.flat[0]), float(pr.ss.flat[0])
    lam = k0 * (4 * np.sin(np.pi * kx / 40) ** 2 + 4 * np.sin(np.pi * ky / 40) ** 2)
    out = s.solve(b=mode.astype(np.complex128)[None, :], inner_tol=1e-13)
    assert np.all(out.m_j[0] == 1)
    for j, sg in enumerate(pr.sigma):
        x = mode / (lam + sg * s0 * np.prod(pr.h))
        assert rel_err(out.X[0, j], x) <= 1e-9
    s.close()


def test_m_max_reached_reports_not_converged():
    need_gpu()
    pr = synth.make_problem((32, 32), n_f=4, periods=(5.0, 3600.0), n_p=2, seed=3)
    s = Solver(pr)
    out = s.solve(m_max=3, tol=1e-12)
    assert out.status == fks.FKS_NOT_CONVERGED
    assert np.all(out.m_j <= 3) and np.any(out.shift_status == 1)
    s.close()


def test_invalid_arguments_rejected_before_device_work():
    need_gpu()
    pr = synth.make_problem((16, 16), n_f=3, periods=(10.0, 1000.0), n_p=1, seed=2)
    s = Solver(pr)
    with pytest.raises(fks.FksError) as e:
        s.solve(tol=-1.0)
    assert e.value.status == fks.FKS_ERR_ARG
    with pytest.raises(fks.FksError):
        s.solve(schedule=[3])
    with pytest.raises(fks.FksError):
        s.solve(sigma=np.array([np.nan + 0j]))
    with pytest.raises(fks.FksError):
        fks.fks_op_grid(s.ctx, 2, (16, 16), (1.0, 1.0), -np.ones(256), np.ones(256), 0xF)
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_graph_and_host_driven_loops_agree_bitwise(precision):
    """The step loop as one CUDA graph (conditional WHILE nodes) runs the same
    kernels in the same order as the host-driven loop."""
    need_gpu()
    pr = synth.make_problem((48, 48), n_f=6, periods=(5.0, 3600.0), n_p=3, seed=16, n_src=2, m_max=60)
    s = Solver(pr)
    g = s.solve(precision=precision, inner_tol=1e-10, launch_mode=0)
    h = s.solve(precision=precision, inner_tol=1e-10, launch_mode=1)
    g2 = s.solve(precision=precision, inner_tol=1e-10, launch_mode=0)     # cached graph, second launch
    assert np.array_equal(g.X, h.X) and np.array_equal(g2.X, h.X)
    assert np.array_equal(g.m_j, h.m_j) and np.array_equal(g.inner_cycles, h.inner_cycles)
    assert np.array_equal(g.steps, h.steps)
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED, fks.FKS_PREC_MIXED_BF16])
def test_fused_and_per_sweep_kernels_agree_bitwise(precision):
    """Fused 2D tile kernels and per-half-sweep kernels perform the same
    operations in the same order; the autotuner's choice cannot change results."""
    need_gpu()
    pr = synth.make_problem((192, 160), n_f=5, periods=(5.0, 3600.0), n_p=3, seed=17, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, 0)
    a = s.solve(precision=precision, inner_tol=1e-10)
    fks.fks_op_set_fusion(s.op, precision, -1)
    b = s.solve(precision=precision, inner_tol=1e-10)
    picked = fks.fks_op_autotune(s.op, precision, pr.tau_bar[1])
    c = s.solve(precision=precision, inner_tol=1e-10)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.X, c.X), picked
    assert np.array_equal(a.inner_cycles, b.inner_cycles)
    # the tile shape of the fused kernels does not change any cell's update
    fks.fks_op_set_fusion(s.op, precision, -1)
    for t16 in (0, -1):
        fks.fks_op_set_tiles(s.op, precision, t16)
        d = s.solve(precision=precision, inner_tol=1e-10)
        assert np.array_equal(a.X, d.X), t16
    for t8 in (-1, 7680, 0):
        fks.fks_op_set_tiles8(s.op, precision, t8)
        d = s.solve(precision=precision, inner_tol=1e-10)
        assert np.array_equal(a.X, d.X), t8
    # nor does moving small levels into the single-block tail kernel
    for tail in (1024, 4096, 256):
        fks.fks_op_set_tail(s.op, precision, tail)
        d = s.solve(precision=precision, inner_tol=1e-10)
        assert np.array_equal(a.X, d.X), tail
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED, fks.FKS_PREC_MIXED_BF16])
@pytest.mark.parametrize("shape,n_src", [((20, 24, 40), 1), ((32, 48, 32), 2)])
def test_fused_3d_levels_agree_bitwise(precision, shape, n_src):
    """The 3D z-march kernels (four half sweeps, residual and restriction, or
    interpolation and four half sweeps, per launch) repeat the per-level
    kernels' operations in the same order: the same bits for every tile shape
    and z-chunk, including ragged tiles (40 x 24 cells in x-y against 16 x 16
    and 32 x 16 tiles) and ragged chunks (20 planes in chunks of 6 or 8), a
    level that is not coarsened in z (10 x 6 x 5 below 20 x 12 x 10) and the
    host-driven loop."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=5, periods=(5.0, 3600.0), n_p=3, seed=37, n_src=n_src, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, 0)
    a = s.solve(precision=precision, inner_tol=1e-10)
    fks.fks_op_set_fusion(s.op, precision, -1)
    nl = len(fks.fks_op_zchunks(s.op, precision))
    for t16, t8 in ((0, 0), (-1, 0), (-1, -1)):        # 32 x 16, 16 x 16, 8 x 8 tiles
        fks.fks_op_set_tiles(s.op, precision, t16)
        fks.fks_op_set_tiles8(s.op, precision, t8)
        for zc in (2, 6, 8, 0):
            for lv in range(nl):
                fks.fks_op_set_zchunk(s.op, precision, lv, zc)
            d = s.solve(precision=precision, inner_tol=1e-10)
            assert np.array_equal(a.X, d.X), (t16, t8, zc)
            assert np.array_equal(a.inner_cycles, d.inner_cycles) and np.array_equal(a.m_j, d.m_j)
    h = s.solve(precision=precision, inner_tol=1e-10, launch_mode=1)
    assert np.array_equal(a.X, h.X)
    fks.fks_op_autotune(s.op, precision, pr.tau_bar[1])
    c = s.solve(precision=precision, inner_tol=1e-10)
    assert np.array_equal(a.X, c.X), (fks.fks_op_tiling(s.op, precision), fks.fks_op_zchunks(s.op, precision))
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_fused_3d_replay_parity(precision):
    """Replay parity with the oracle on a 3D grid whose levels all run in the
    z-march kernels (chunks of 4 planes, 8 x 8 tiles), every x_j to 1e-8
    (complex128) or 1e-6 (complex64 cycles)."""
    need_gpu()
    pr = synth.make_problem((24, 16, 32), n_f=6, periods=(5.0, 3600.0), n_p=3, seed=39, m_max=80,
                            corr_frac=(0.2, 0.2, 0.05), ss_var=0.25)
    eps = 1e-10
    op, ref = oracle_run(pr, eps)
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, -1)
    fks.fks_op_set_tiles8(s.op, precision, -1)
    for lv in range(len(fks.fks_op_zchunks(s.op, precision))):
        fks.fks_op_set_zchunk(s.op, precision, lv, 4)
    out = s.solve(inner_tol=eps, precision=precision, replay_cycles=rc, replay_mj=mj)
    assert np.array_equal(out.m_j[0], ref.m_j)
    tol = 1e-8 if precision == fks.FKS_PREC_FP64 else 1e-6
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= tol, j
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
@pytest.mark.parametrize("shape,n_src", [((64, 80), 1), ((256, 256), 3)])
def test_cluster_vcycle_agrees_bitwise(precision, shape, n_src):
    """The cluster kernel (lower levels as bands of rows in the shared memory of
    an 8-CTA cluster) updates every cell with the operations of the per-level
    kernels in the same order: the same bits from every starting level. 64 x 80
    ends on a 4 x 5 coarsest level (odd rows on the last banded level, a single
    banded level when started there); 256 x 256 with three sources."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=5, periods=(5.0, 3600.0), n_p=3, seed=31, n_src=n_src, m_max=60)
    s = Solver(pr)
    a = s.solve(precision=precision, inner_tol=1e-10)
    assert fks.fks_op_tiling(s.op, precision)[3] == 0
    starts = set()
    for cmax in (1 << 40, 4096, 1024, 256, 80, 64):
        try:
            fks.fks_op_set_cluster(s.op, precision, cmax)
        except fks.FksError:
            continue
        assert fks.fks_op_tiling(s.op, precision)[3] == cmax
        d = s.solve(precision=precision, inner_tol=1e-10)
        assert np.array_equal(a.X, d.X), cmax
        assert np.array_equal(a.inner_cycles, d.inner_cycles) and np.array_equal(a.m_j, d.m_j)
        starts.add(cmax)
    assert len(starts) >= 3, starts
    # host-driven loop, and the tuner's pick
    fks.fks_op_set_cluster(s.op, precision, 1024)
    h = s.solve(precision=precision, inner_tol=1e-10, launch_mode=1)
    assert np.array_equal(a.X, h.X)
    fks.fks_op_autotune(s.op, precision, pr.tau_bar[1])
    c = s.solve(precision=precision, inner_tol=1e-10)
    assert np.array_equal(a.X, c.X), fks.fks_op_tiling(s.op, precision)
    fks.fks_op_set_cluster(s.op, precision, 0)
    assert fks.fks_op_tiling(s.op, precision)[3] == 0
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
@pytest.mark.parametrize("shape,n_src", [((64, 80), 2), ((128, 128), 3)])
def test_tail_kernels_agree_bitwise(precision, shape, n_src):
    """The single-block tail in its register-resident 2D form (levels of at
    most 1024 cells, cells owned in pairs), in its general form (a 4096-cell
    level) and the per-level kernels with only the coarsest level in the tail
    give the same bits."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=5, periods=(5.0, 3600.0), n_p=3, seed=33, n_src=n_src, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, -1)
    fks.fks_op_set_tail(s.op, precision, 1)       # the coarsest level alone
    a = s.solve(precision=precision, inner_tol=1e-10)
    for tail in (80, 320, 1024, 4096):
        fks.fks_op_set_tail(s.op, precision, tail)
        d = s.solve(precision=precision, inner_tol=1e-10)
        assert np.array_equal(a.X, d.X), tail
        assert np.array_equal(a.inner_cycles, d.inner_cycles), tail
    fks.fks_op_set_fusion(s.op, precision, 0)     # per-sweep kernels above the tail
    fks.fks_op_set_tail(s.op, precision, 1024)
    d = s.solve(precision=precision, inner_tol=1e-10)
    assert np.array_equal(a.X, d.X)
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_ragged_hierarchy_paths_agree_bitwise(precision):
    """126 x 130 halves to 63 x 65, which even halving cannot coarsen further, so
    odd sides halve too: 32 x 33, 16 x 17, 8 x 17, 4 x 17. The fused tile kernels
    and the 2D tail keep to levels with two children per coarse cell; every
    choice of fusion and tail (the general tail over the ragged levels included)
    and the autotuner's give the bits of the per-level kernels."""
    need_gpu()
    pr = synth.make_problem((126, 130), n_f=5, periods=(5.0, 3600.0), n_p=3, seed=34, n_src=2, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, 0)
    fks.fks_op_set_tail(s.op, precision, 1)
    a = s.solve(precision=precision, inner_tol=1e-10)
    assert a.status == fks.FKS_OK
    for fuse in (0, -1):
        fks.fks_op_set_fusion(s.op, precision, fuse)
        for tail in (64, 320, 1100, 4096):
            fks.fks_op_set_tail(s.op, precision, tail)
            d = s.solve(precision=precision, inner_tol=1e-10)
            assert np.array_equal(a.X, d.X), (fuse, tail)
    fks.fks_op_autotune(s.op, precision, pr.tau_bar[1])
    d = s.solve(precision=precision, inner_tol=1e-10)
    assert np.array_equal(a.X, d.X), fks.fks_op_tiling(s.op, precision)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    for r in range(2):
        tr = oracle.true_residuals(op, pr.rhs()[:, r], pr.sigma, a.X[r].T)
        assert (tr <= pr.tol).all()
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED, fks.FKS_PREC_MIXED_BF16])
def test_one_source_restriction_agrees_with_batched_form(precision):
    """A lone source restricts 3D levels in 32 x 8 x 2 tiles (fine residuals
    first, then the sum over children); a batch of sources uses one thread per
    coarse cell for all of its sources. On 18 x 22 x 26, whose hierarchy
    continues ragged below 9 x 11 x 13 (children past the odd sides skipped),
    each source alone gives the bits it gets inside the batch."""
    need_gpu()
    pr = synth.make_problem((18, 22, 26), n_f=5, periods=(5.0, 3600.0), n_p=3, seed=41, n_src=2, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, 0)
    fks.fks_op_set_tail(s.op, precision, 1)
    both = s.solve(precision=precision, inner_tol=1e-10)
    assert both.status == fks.FKS_OK
    for r in range(2):
        alone = s.solve(b=pr.rhs().T[r:r + 1].copy(), precision=precision, inner_tol=1e-10)
        assert np.array_equal(alone.X[0], both.X[r]), r
        assert np.array_equal(alone.inner_cycles[0], both.inner_cycles[r]), r
    s.close()


@pytest.mark.parametrize("shape", [(289, 289), (45, 45, 45)])
def test_odd_aquifers_certify_every_shift(shape):
    """Odd-sided aquifers whose hierarchies are ragged from the finest level
    (289^2 keeps one-cell-wide edge cells through four levels): free-running
    mixed-precision solves certify every shift, and the GPU's true residuals
    equal the oracle's recomputation."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=8, periods=(5.0, 3600.0), n_p=3, seed=20000, m_max=80)
    s = Solver(pr)
    out = s.solve(precision=fks.FKS_PREC_MIXED, inner_tol=1e-10, inner_relax=0.003)
    assert out.status == fks.FKS_OK
    assert int(out.inner_cycles.max()) < 50
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    tr = oracle.true_residuals(op, pr.rhs()[:, 0], pr.sigma, out.X[0].T)
    assert (tr <= pr.tol).all()
    assert np.allclose(out.res_true[0], tr, rtol=1e-6, atol=1e-15)
    s.close()


@pytest.mark.parametrize("shape", [(32, 32, 32), (96, 80)])
def test_launch_overlap_changes_no_bits(shape):
    """Programmatic dependent launch of the multigrid and defect kernels (the
    default) and plain launches, each in the graph and host-driven loops, give
    the same bits; the graph capture keeps the overlap on."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=6, periods=(5.0, 3600.0), n_p=3, seed=36, n_src=2, m_max=60)
    s = Solver(pr)
    prev = fks.fks_set_pdl(1)
    try:
        outs = []
        for on in (1, 0):
            fks.fks_set_pdl(on)
            for mode in (0, 1):
                outs.append(s.solve(precision=fks.FKS_PREC_MIXED, inner_tol=1e-10, launch_mode=mode))
                if on:
                    assert fks.fks_set_pdl(-1) == 1
        assert outs[0].status == fks.FKS_OK
        for o in outs[1:]:
            assert np.array_equal(outs[0].X, o.X)
            assert np.array_equal(outs[0].inner_cycles, o.inner_cycles)
    finally:
        fks.fks_set_pdl(prev)
        s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED, fks.FKS_PREC_MIXED_BF16])
@pytest.mark.parametrize("shape,n_src", [((32, 48, 40), 2), ((160, 128), 1), ((45, 45, 45), 1)])
def test_cooperative_lower_cycle_agrees_bitwise(precision, shape, n_src):
    """The lower levels' V-cycle in one cooperative launch (from every level
    above the tail, down to the coarsest, on even and ragged hierarchies, in
    the graph and host-driven loops) gives the bits of the separate kernels."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=5, periods=(5.0, 3600.0), n_p=3, seed=37, n_src=n_src, m_max=60)
    s = Solver(pr)
    fks.fks_op_set_fusion(s.op, precision, 0)
    fks.fks_op_set_tail(s.op, precision, 64)
    fks.fks_op_set_coop(s.op, precision, 0)
    a = s.solve(precision=precision, inner_tol=1e-10)
    assert a.status == fks.FKS_OK
    sizes = sorted({int(np.prod(L)) for L in _level_shapes(shape)[1:] if int(np.prod(L)) > 64}, reverse=True)
    assert sizes
    for cm in sizes:
        fks.fks_op_set_coop(s.op, precision, cm)
        assert fks.fks_op_coop_max(s.op, precision) == cm
        for mode in (0, 1):
            d = s.solve(precision=precision, inner_tol=1e-10, launch_mode=mode)
            assert np.array_equal(a.X, d.X), (cm, mode)
            assert np.array_equal(a.inner_cycles, d.inner_cycles), (cm, mode)
    fks.fks_op_set_coop(s.op, precision, 0)
    s.close()


def _level_shapes(shape):
    """The multigrid level shapes of a grid (numpy axis order), as the oracle forms them."""
    op = oracle.assemble(shape, (1.0,) * len(shape), np.ones(shape), np.ones(shape), (1 << (2 * len(shape))) - 1)
    from oracle.gmg import Hierarchy
    return [L.shape for L in Hierarchy(op, [1j]).levels]


def test_cluster_vcycle_rejects_inapplicable_levels():
    """48 x 48 coarsens to 24 x 24 (3 rows per band, followed by a 12-row level
    that does not split into 8 bands): no starting level qualifies."""
    need_gpu()
    pr = synth.make_problem((48, 48), n_f=3, periods=(5.0, 3600.0), n_p=2, seed=32, m_max=40)
    s = Solver(pr)
    for prec in (fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED):
        with pytest.raises(fks.FksError):
            fks.fks_op_set_cluster(s.op, prec, 1 << 40)
        assert fks.fks_op_tiling(s.op, prec)[3] == 0
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_relaxed_inner_tolerance(precision):
    """Relaxed inner tolerances: every shift is still certified (the true
    residual, recomputed by the oracle, within the bound and tol), the inner
    work drops against a fixed eps, and the step and cycle counts follow the
    oracle's relaxed solve (the tolerance of a step depends on estimates that
    both sides compute with their own rounding, so a cycle count may differ
    where a residual sits on its threshold)."""
    need_gpu()
    from oracle.gmg import Hierarchy, GMGInner
    pr = synth.make_problem((96, 80), n_f=24, periods=(5.0, 3600.0), n_p=3, seed=21, m_max=100)
    s = Solver(pr)
    fixed = s.solve(precision=precision, inner_tol=1e-10)
    rel = s.solve(precision=precision, inner_tol=1e-10, inner_relax=0.01)
    assert rel.status == fks.FKS_OK
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    tr = oracle.true_residuals(op, b, pr.sigma, rel.X[0].T)
    assert np.all(tr <= pr.tol * 1.0001) and np.all(rel.res_bound[0] <= pr.tol)
    assert np.all(tr <= rel.res_bound[0] * (1 + 1e-6) + residual_floor(op, b, pr.sigma, rel.X[0].T))
    assert rel.inner_cycles.sum() < 0.85 * fixed.inner_cycles.sum()
    ref = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max,
                               GMGInner(Hierarchy(op, pr.tau_bar), 1e-10), inner_relax=0.01, eps=1e-10)
    assert abs(int(rel.steps[0]) - ref.steps) <= 1
    assert abs(int(rel.inner_cycles.sum()) - int(ref.cycles.sum())) <= 0.05 * ref.cycles.sum()
    s.close()


def test_relaxed_inner_tolerance_replay_parity():
    """The oracle's relaxed solve replayed on the GPU: x_j to 1e-8."""
    need_gpu()
    from oracle.gmg import Hierarchy, GMGInner
    pr = synth.make_problem((64, 48), n_f=12, periods=(5.0, 3600.0), n_p=3, seed=22, m_max=80)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    ref = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max,
                               GMGInner(Hierarchy(op, pr.tau_bar), 1e-10), inner_relax=0.01, eps=1e-10)
    assert ref.eps_k.max() > 1e-9
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    out = s.solve(inner_tol=1e-10, inner_relax=0.01, replay_cycles=rc, replay_mj=mj)
    assert np.array_equal(out.m_j[0], ref.m_j) and int(out.steps[0]) == ref.steps
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.x[:, j]) <= 1e-8, j
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_replay_parity_beyond_64_steps(precision):
    """A solve of 82 Arnoldi steps (tolerance 1e-10, one tau at the geometric
    mean of a 1 s to 10 h period range): more steps than one exact tensor-core
    accumulation covers (64), so the tensor-core assembly runs two chunks and
    adds them in 64-bit integers. Every x_j to 1e-8 (complex128 cycles) or 1e-6
    (complex64 cycles) of the oracle's, from the tensor cores and from the FP64
    assembly kernel, and the two within 1e-12 of each other."""
    need_gpu()
    pr = synth.make_problem((32, 32), n_f=12, periods=(1.0, 36000.0), n_p=1, seed=51, m_max=100, tol=1e-10)
    eps = 1e-12
    op, ref = oracle_run(pr, eps)
    assert ref.steps > 64
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    tol = 1e-8 if precision == fks.FKS_PREC_FP64 else 1e-6
    outs = []
    for assembly in (0, 1):
        out = s.solve(inner_tol=eps, precision=precision, replay_cycles=rc, replay_mj=mj, assembly=assembly)
        assert np.array_equal(out.m_j[0], ref.m_j) and int(out.steps[0]) == ref.steps
        for j in range(len(pr.sigma)):
            assert rel_err(out.X[0, j], ref.x[:, j]) <= tol, (assembly, j)
        outs.append(out)
    for j in range(len(pr.sigma)):
        assert rel_err(outs[0].X[0, j], outs[1].X[0, j]) <= 1e-12, j
    s.close()


@pytest.mark.parametrize("shape", [(128, 96), (24, 32, 40)])
def test_bf16_smoother_option_certifies_every_shift(shape):
    """The bf16-smoother option (multigrid coefficients rounded to bf16 inside
    the complex64 cycle, complex128 defect correction with the exact operator):
    free-running solves reach the 1e-8 true residual for every shift, checked
    with the oracle's own operator, and x_j agree with the complex128 solve
    within what the tolerance allows."""
    need_gpu()
    pr = synth.make_problem(shape, n_f=12, periods=(5.0, 3600.0), n_p=3, seed=48, m_max=100,
                            corr_frac=(0.2, 0.2, 0.05) if len(shape) == 3 else (0.2, 0.2, 0.2))
    s = Solver(pr)
    out = s.solve(precision=fks.FKS_PREC_MIXED_BF16, inner_tol=1e-10, inner_relax=0.003)
    assert out.status == fks.FKS_OK
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    tr = oracle.true_residuals(op, pr.rhs()[:, 0], pr.sigma, out.X[0].T)
    assert np.all(tr <= pr.tol * 1.0001), tr.max()
    assert np.allclose(tr, out.res_true[0], rtol=1e-6, atol=1e-15)
    ref = s.solve(precision=fks.FKS_PREC_FP64, inner_tol=1e-10)
    for j in range(len(pr.sigma)):
        assert rel_err(out.X[0, j], ref.X[0, j]) <= 1e-5, j
    s.close()
