"""GPU convergence monitors (Section 3) against the oracle: the exported flexible
Hessenberg matrix and preconditioner shifts of a replayed solve, and Prop. 3's
alpha recorded by the Givens update at each shift's freeze step."""
import numpy as np
import pytest

from oracle.monitors import gmres_alpha
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, oracle_run, replay_arrays

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [fks.FKS_FGMRES, fks.FKS_FFOM])
def test_hessenberg_export_and_alpha_match_oracle(variant):
    need_gpu()
    pr = synth.make_problem((40, 36), n_f=12, periods=(5.0, 3600.0), n_p=3, seed=51, m_max=60)
    eps = 1e-10
    op, ref = oracle_run(pr, eps, variant="ffom" if variant == fks.FKS_FFOM else "fgmres")
    rc, mj = replay_arrays(pr, [ref])
    s = Solver(pr)
    out = s.solve(inner_tol=eps, variant=variant, replay_cycles=rc, replay_mj=mj)
    k = int(out.steps[0])
    assert k == ref.steps
    # H_bar column-major per step: hbar[0, c] is column c + 1 (rows 1..m_max + 1)
    Hg = out.hbar[0, :k, :k + 1].T
    assert np.max(np.abs(Hg - ref.H)) <= 1e-9 * np.max(np.abs(ref.H))
    assert np.all(out.hbar[0, k:] == 0) and np.all(out.hbar[0, :k, k + 1:] == 0)
    assert np.array_equal(out.tau_k[0, :k], ref.taus) and np.all(out.tau_k[0, k:] == 0)
    for j, sg in enumerate(pr.sigma):
        m = int(out.m_j[0, j])
        a_ref = gmres_alpha(ref.H, ref.taus, sg, m)
        assert out.gmres_alpha[0, j] == pytest.approx(a_ref, rel=1e-7, abs=1e-13), (j, m)
    s.close()


def test_alpha_of_zero_rhs_source_and_multi_source_slices():
    """A zero right-hand side leaves its monitors at zero; a batch reports each
    source's own alpha (bitwise what the source gets alone)."""
    need_gpu()
    pr = synth.make_problem((32, 32), n_f=5, periods=(5.0, 3600.0), n_p=2, seed=52, n_src=3, m_max=50)
    s = Solver(pr)
    b = pr.rhs().T.copy()
    b[1] = 0
    out = s.solve(b, inner_tol=1e-10)
    assert np.all(out.gmres_alpha[1] == 0) and np.all(out.hbar[1] == 0)
    solo = s.solve(b[[2]], inner_tol=1e-10)
    assert np.array_equal(out.gmres_alpha[2], solo.gmres_alpha[0])
    assert np.array_equal(out.hbar[2], solo.hbar[0]) and np.array_equal(out.tau_k[2], solo.tau_k[0])
    s.close()
