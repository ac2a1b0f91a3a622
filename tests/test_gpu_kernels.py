"""GPU parity of the operator apply and the multigrid inner solve against the
oracle (same seeded inputs, through the C ABI)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.gmg import Hierarchy
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, oracle_op, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [((64, 64), None), ((20, 24), None), ((1, 7), None), ((16, 12, 10), None), ((9, 5, 6), 0b010110),
          ((24, 24), 0b0110), ((33, 17), None)]


@pytest.mark.parametrize("shape,mask", SHAPES)
def test_operator_apply_matches_oracle(shape, mask):
    need_gpu()
    pr = synth.make_problem(shape, n_f=2, periods=(10, 1000), n_p=1, seed=3, dirichlet_mask=mask)
    s = Solver(pr)
    op = oracle_op(pr)
    rng = np.random.default_rng(7)
    nvec = 3
    x = rng.standard_normal((nvec, pr.n)) + 1j * rng.standard_normal((nvec, pr.n))
    for sh in (0.0, 0.37j, 1.5 - 2j):
        y = np.zeros_like(x)
        fks.fks_op_apply(s.op, sh, x, y, nvec)
        for v in range(nvec):
            ref = op.K @ x[v] + sh * (op.M @ x[v])
            assert rel_err(y[v], ref) <= 1e-14
    s.close()


@pytest.mark.parametrize("shape", [(64, 64), (24, 20), (16, 16, 16), (12, 10, 8), (96, 80), (200, 136), (40, 40, 24)])
@pytest.mark.parametrize("cycles", [1, 3])
def test_fixed_cycles_match_oracle_vcycle(shape, cycles):
    need_gpu()
    pr = synth.make_problem(shape, n_f=2, periods=(10, 1000), n_p=1, seed=5)
    s = Solver(pr)
    op = oracle_op(pr)
    tau = pr.tau_bar[0]
    hier = Hierarchy(op, [tau])
    rng = np.random.default_rng(11)
    v = rng.standard_normal(pr.n) + 1j * rng.standard_normal(pr.n)
    v /= np.linalg.norm(v)
    z_ref, c_ref, p_ref = hier.solve(v, 0, 0.0, cycles=cycles)
    z = np.zeros_like(v)
    st, c, pn = fks.fks_precond_apply(s.op, tau, v, z, 1e-30, cycles=cycles)
    assert c == cycles
    assert rel_err(z, z_ref) <= 1e-12
    assert abs(pn - p_ref) <= 1e-9 * p_ref + 1e-15
    # complex64 cycles with complex128 defect correction: same iterate to fp32 accuracy
    z32 = np.zeros_like(v)
    st, c, pn32 = fks.fks_precond_apply(s.op, tau, v, z32, 1e-30, cycles=cycles, precision=fks.FKS_PREC_MIXED)
    assert rel_err(z32, z_ref) <= 1e-4
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_inner_solve_reaches_eps(precision, eps):
    need_gpu()
    pr = synth.make_problem((48, 40), n_f=2, periods=(5, 3600), n_p=1, seed=6)
    s = Solver(pr)
    op = oracle_op(pr)
    tau = pr.tau_bar[0]
    rng = np.random.default_rng(2)
    v = rng.standard_normal(pr.n) + 1j * rng.standard_normal(pr.n)
    v /= np.linalg.norm(v)
    z = np.zeros_like(v)
    st, c, pn = fks.fks_precond_apply(s.op, tau, v, z, eps, precision=precision)
    p_true = np.linalg.norm(v - op.shifted(tau) @ z)
    assert pn <= eps and c <= 50
    assert abs(p_true - pn) <= 1e-3 * eps                 # reported ||p|| is the true residual
    z_lu = spla.spsolve(op.shifted(tau).tocsc(), v)
    sv_min = np.linalg.svd(op.shifted(tau).toarray(), compute_uv=False).min()
    assert np.linalg.norm(z - z_lu) <= 1.01 * pn / sv_min
    s.close()
