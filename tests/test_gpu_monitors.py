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


def _match(a, b):
    """max distance of a greedy nearest pairing of two multisets of complex values"""
    b = list(b)
    worst = 0.0
    for x in sorted(a, key=lambda z: -abs(z)):
        d = [abs(x - y) for y in b]
        i = int(np.argmin(d))
        worst = max(worst, d[i])
        b.pop(i)
    return worst


def test_ritz_values_of_a_solve_match_oracle():
    """fks_ritz on a solve's exported H_bar and tau_k (two sources, one with a zero
    right-hand side) against the oracle's Ritz values of the same matrices."""
    need_gpu()
    from oracle.monitors import ritz_pairs
    pr = synth.make_problem((40, 36), n_f=8, periods=(5.0, 3600.0), n_p=3, seed=53, n_src=2, m_max=60)
    s = Solver(pr)
    b = pr.rhs().T.copy()
    b[1] = 0
    out = s.solve(b, inner_tol=1e-10)
    theta, status = s.ritz(out)
    k = int(out.steps[0])
    assert k > 5 and np.all(status == 0)
    H = out.hbar[0, :k, :k + 1].T
    ref = ritz_pairs(H, out.tau_k[0], 0.0, k)[0]
    assert _match(theta[0, :k], ref) <= 1e-9 * np.max(np.abs(ref))
    assert np.all(theta[0, k:] == 0) and np.all(theta[1] == 0) and int(out.steps[1]) == 0
    s.close()


@pytest.mark.parametrize("m", [1, 2, 17, 64, 128])
def test_ritz_values_of_random_hessenberg_matrices(m):
    """The GPU eigenvalue solver against NumPy on random upper Hessenberg H_bar
    (positive subdiagonal, as Arnoldi produces; eigenvalues that a relative
    perturbation of 1e-14 moves by at most 1e-13) and random tau, up to m_max."""
    need_gpu()
    from paper_1212_3660_gb300 import fks as F
    rng = np.random.default_rng(m)
    n_rhs, m_max = 3, max(m, 2)
    hbar = np.zeros((n_rhs, m_max, m_max + 1), np.complex128)
    tau = np.zeros((n_rhs, m_max), np.complex128)
    steps = np.array([m, max(1, m // 2), m], np.int32)
    ctx = F.fks_create(0)
    refs = []
    for r in range(n_rhs):
        k = int(steps[r])
        Hm = np.triu(rng.standard_normal((k + 1, k)) + 1j * rng.standard_normal((k + 1, k)), -1)
        for c in range(k):
            Hm[c + 1, c] = abs(Hm[c + 1, c]) + 0.1
        # a dominant diagonal keeps H_m and the eigenvalues well conditioned
        # (random Hessenberg matrices of order 64 reach cond 1e10)
        Hm[:k, :k] += (2.0 + 1.0j) * np.sqrt(k) * np.eye(k)
        hbar[r, :k, :k + 1] = Hm.T
        tau[r, :k] = 1j * np.exp(rng.uniform(-3, 0, k))
        G = np.linalg.inv(Hm[:k, :k]) - np.diag(tau[r, :k])
        refs.append(np.linalg.eigvals(G))
    theta = np.zeros((n_rhs, m_max), np.complex128)
    status = np.zeros(n_rhs, np.int32)
    F.fks_ritz(ctx, hbar, tau, steps, n_rhs, m_max, theta, status)
    assert np.all(status == 0), status
    for r in range(n_rhs):
        k = int(steps[r])
        assert _match(theta[r, :k], refs[r]) <= 1e-8 * np.max(np.abs(refs[r])), r
    F.fks_destroy(ctx)


def test_ritz_rejects_bad_arguments():
    need_gpu()
    from paper_1212_3660_gb300 import fks as F
    ctx = F.fks_create(0)
    h = np.zeros((1, 4, 5), np.complex128)
    t = np.zeros((1, 4), np.complex128)
    th = np.zeros((1, 4), np.complex128)
    stt = np.zeros(1, np.int32)
    with pytest.raises(F.FksError):
        F.fks_ritz(ctx, h, t, np.array([5], np.int32), 1, 4, th, stt)
    with pytest.raises(F.FksError):
        F.fks_ritz(ctx, h, t, np.array([2], np.int32), 1, 129, th, stt)
    F.fks_destroy(ctx)
