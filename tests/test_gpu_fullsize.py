"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark times (CUDA graph, autotuned thresholds, relaxed
inner tolerance l = 0.003): every shift certified, and sampled outputs checked
one by one against the oracle (true residuals with the oracle's own sparse K and
M; for 512 x 512 also the sparse-LU solution of sampled shifts). Replay parity
at full size: the oracle's inner-cycle counts and freeze steps replayed on the
GPU in the bench's launch configuration, every x_j compared with the oracle's
(512 x 512: all 200 shifts, every element; 128^3: 8 shifts, 1025 sampled cells
and the norm, from the record tests/golden/make_replay_3d.py wrote)."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle.gmg import GMGInner, Hierarchy
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, rel_err, replay_arrays, residual_floor

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


@pytest.fixture(scope="module")
def oracle_512():
    """The oracle's solve of the 512 x 512 workload with the bench's inner rule."""
    pr = synth.workload(2, m_max=100)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    ref = oracle.shifted_solve(op, pr.rhs()[:, 0], pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max,
                               GMGInner(Hierarchy(op, pr.tau_bar), EPS), inner_relax=RELAX, eps=EPS)
    return pr, ref


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_2d_512x512_replay_parity_every_shift(precision, oracle_512):
    """All 200 shifts of the 512 x 512 workload in the bench's launch
    configuration (autotuned tiles, cluster and tail kernels, CUDA graph,
    tensor-core assembly), replaying the oracle's cycles and freeze steps:
    every element of every x_j to 1e-8 relative (complex128 cycles) or 1e-6
    (complex64 cycles)."""
    need_gpu()
    pr, ref = oracle_512
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    fks.fks_op_autotune(s.op, precision, complex(pr.tau_bar[len(pr.tau_bar) // 2]))
    out = s.solve(precision=precision, inner_tol=EPS, replay_cycles=rc, replay_mj=mj, launch_mode=0)
    assert np.array_equal(out.m_j[0], ref.m_j) and int(out.steps[0]) == ref.steps
    tol = 1e-8 if precision == fks.FKS_PREC_FP64 else 1e-6
    errs = [rel_err(out.X[0, j], ref.x[:, j]) for j in range(len(pr.sigma))]
    assert max(errs) <= tol, (int(np.argmax(errs)), max(errs))
    s.close()


def _replay_record(path):
    rec = {}
    for line in open(path):
        if line.startswith("#"):
            continue
        key, *vals = line.split()
        rec[key] = vals
    return rec


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_3d_128_cubed_replay_parity_sampled(precision):
    """128^3 (2.1M cells) with 8 of the workload's shifts, in the bench's launch
    configuration, replaying the oracle's recorded cycles and freeze steps:
    each x_j's norm, and x_j at 1025 sampled cells element by element, within
    1e-8 (complex128 cycles) or 1e-6 (complex64 cycles) of ||x_j||."""
    need_gpu()
    here = os.path.dirname(os.path.abspath(__file__))
    rec = _replay_record(os.path.join(here, "golden", "replay_3d_128cube_f8.txt"))
    idx = np.linspace(0, 199, 8).round().astype(int)
    pr = synth.workload(3, m_max=100)
    pr.sigma = pr.sigma[idx].copy()
    steps = int(rec["steps"][0])
    rc = np.zeros((1, pr.m_max), np.int32)
    rc[0, :steps] = [int(c) for c in rec["cycles"]]
    mj = np.array([[int(m) for m in rec["m_j"]]], np.int32)
    s = Solver(pr)
    fks.fks_op_autotune(s.op, precision, complex(pr.tau_bar[len(pr.tau_bar) // 2]))
    out = s.solve(precision=precision, inner_tol=EPS, replay_cycles=rc, replay_mj=mj, launch_mode=0, device_out=True)
    assert np.array_equal(out.m_j, mj) and int(out.steps[0]) == steps
    tol = 1e-8 if precision == fks.FKS_PREC_FP64 else 1e-6
    cells = np.array([int(c) for c in rec["cells"]])
    import torch
    X = out.X[0]
    for j in range(len(pr.sigma)):
        xnorm = float(rec["xnorm"][j])
        assert abs(float(torch.linalg.vector_norm(X[j])) - xnorm) <= tol * xnorm, j
        v = np.array([float(t) for t in rec[f"x{j}"]])
        ref = v[0::2] + 1j * v[1::2]
        got = X[j, torch.from_numpy(cells).cuda()].cpu().numpy()
        assert np.max(np.abs(got - ref)) <= tol * xnorm, (j, float(np.max(np.abs(got - ref)) / xnorm))
    assert np.all(out.res_true[0] <= pr.tol * 1.01)
    s.close()
