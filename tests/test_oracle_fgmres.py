"""Pins of the oracle's flexible shifted solver (Algorithms 3 and 4, Section 4 bounds).

Independent routes: dense numpy solves on tiny grids, the DST-II closed form for
a homogeneous box, SciPy's textbook GMRES on the right-preconditioned operator
(K + sigma M)(K + tau M)^{-1} (single tau, Eq. shiftinvariant), special cases
with known answers (sigma = tau, one DST mode), and the identities/inequalities
of Eq. arnoldimod, Eq. zmvmrelation, Eq. fomgmresresidual, Eq. resdiff,
Eq. fomresidualsimplified and Prop. 3.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle.fgmres import shifted_hessenberg, OK, BREAKDOWN
from oracle.gmg import Hierarchy, GMGInner
from paper_1212_3660_gb300 import synth

from test_oracle_operator import dst_solve, dst_eigs


def small_problem(shape=(24, 24), n_f=6, n_p=2, seed=4, **kw):
    pr = synth.make_problem(shape, n_f=n_f, periods=(10.0, 1000.0), n_p=n_p, seed=seed, **kw)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    return pr, op, pr.rhs()[:, 0]


def test_arnoldi_relations_exact_inner():
    pr, op, b = small_problem()
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-10, 60, oracle.ExactInner(op, pr.tau_bar),
                               keep_basis=True)
    k = res.steps
    V, Z, H = res.V, res.Z, res.H
    assert np.linalg.norm(V.conj().T @ V - np.eye(k + 1)) <= 1e-12
    MZ = op.M @ Z
    assert np.linalg.norm(MZ - V @ H) <= 1e-12 * np.linalg.norm(MZ)               # Eq. arnoldimod
    KZ = op.K @ Z + MZ * res.taus[None, :]
    assert np.linalg.norm(KZ - V[:, :k]) <= 1e-10 * np.linalg.norm(V[:, :k])        # Eq. zmvmrelation
    for j, s in enumerate(pr.sigma):                                                 # Eq. shiftedarnoldimod
        lhs = op.shifted(s) @ Z
        rhs = V @ shifted_hessenberg(H, res.taus, s, k)
        assert np.linalg.norm(lhs - rhs) <= 1e-9 * np.linalg.norm(rhs)
    tr = oracle.true_residuals(op, b, pr.sigma, res.x)                               # Eq. fomgmresresidual
    assert np.all(np.abs(tr - res.res_est) <= 1e-9 * np.maximum(tr, 1e-12) + 1e-13)
    assert np.all(tr <= 1e-10 * 1.0001)


def test_arnoldi_relations_inexact_inner():
    pr, op, b = small_problem(seed=7)
    hier = Hierarchy(op, pr.tau_bar)
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-8, 60, GMGInner(hier, 1e-6),
                               keep_basis=True)
    k = res.steps
    V, Z, H = res.V, res.Z, res.H
    assert np.linalg.norm(V.conj().T @ V - np.eye(k + 1)) <= 1e-12
    MZ = op.M @ Z
    assert np.linalg.norm(MZ - V @ H) <= 1e-12 * np.linalg.norm(MZ)  # holds with inexact inner solves too
    P = V[:, :k] - (op.K @ Z + MZ * res.taus[None, :])                   # p_k of Eq. zmmoditer
    assert np.allclose(np.linalg.norm(P, axis=0), res.pnorm, rtol=1e-6)
    assert np.all(res.pnorm <= 1e-6 * (1 + 1e-12))


@pytest.mark.parametrize("shape", [(4, 4), (8, 8), (16, 16), (4, 4, 4)])
def test_tiny_grids_match_dense_solve(shape):
    pr = synth.make_problem(shape, n_f=5, periods=(10.0, 1000.0), n_p=2, seed=11)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-13, op.n,
                               oracle.ExactInner(op, pr.tau_bar))
    for j, s in enumerate(pr.sigma):
        A = op.shifted(s).toarray()
        xd = np.linalg.solve(A, b)
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(res.x[:, j] - xd) <= max(kappa * 1e-13, 1e-12) * np.linalg.norm(xd)


def test_homogeneous_box_matches_dst_closed_form():
    shape = (32, 32)
    pr = synth.make_problem(shape, n_f=8, periods=(5.0, 3600.0), n_p=3, seed=1, homogeneous=True)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    tol = 1e-9
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, tol, 100, oracle.ExactInner(op, pr.tau_bar))
    assert np.all(res.status == OK)
    k0, s0 = float(pr.cond.flat[0]), float(pr.ss.flat[0])
    for j, s in enumerate(pr.sigma):
        x = dst_solve(shape, pr.h, k0, s0, s, b)
        A = op.shifted(s)
        # ||x - x*|| <= ||A^{-1}|| ||r|| <= ||A^{-1}|| tol ||b||
        lam_min = np.min(np.abs(k0 * (dst_eigs(32)[:, None] + dst_eigs(32)[None, :]) + s * s0 * np.prod(pr.h)))
        assert np.linalg.norm(res.x[:, j] - x) <= 1.01 * tol * np.linalg.norm(b) / lam_min
        assert np.linalg.norm(b - A @ res.x[:, j]) <= tol * np.linalg.norm(b) * 1.0001


def test_sigma_equal_tau_converges_in_one_step():
    pr, op, b = small_problem(n_p=1)
    tau = pr.tau_bar[0]
    sig = np.array([tau, 0.3 * tau])
    ex = oracle.ExactInner(op, [tau])
    res = oracle.shifted_solve(op, b, sig, [tau], [0], 1e-12, 50, ex, keep_basis=True)
    assert res.m_j[0] == 1
    x_exact = spla.spsolve(op.shifted(tau).tocsc(), b)
    assert np.linalg.norm(res.x[:, 0] - x_exact) <= 1e-13 * np.linalg.norm(x_exact)
    assert np.allclose(res.x[:, 0], res.beta * res.Z[:, 0], rtol=1e-14)


def test_single_dst_mode_breaks_down_at_step_one():
    shape = (12, 10)
    k0, s0 = 2e-4, 1e-5
    h = (1.0, 1.0)
    op = oracle.assemble(shape, h, np.full(shape, k0), np.full(shape, s0), 0b1111)
    jj, ii = np.meshgrid(np.arange(1, 13), np.arange(1, 11), indexing="ij")
    kx, ky = 3, 2
    mode = np.sin(math.pi * kx * (ii - 0.5) / 10) * np.sin(math.pi * ky * (jj - 0.5) / 12)
    b = mode.ravel().astype(complex)
    lam = k0 * (4 * math.sin(math.pi * kx / 20) ** 2 + 4 * math.sin(math.pi * ky / 24) ** 2)
    sig = np.array([0.01j, 0.5j, 3.0j])
    res = oracle.shifted_solve(op, b, sig, [0.1j], [0], 1e-12, 20, oracle.ExactInner(op, [0.1j]))
    assert res.steps == 1 and res.breakdown
    for j, s in enumerate(sig):
        assert np.allclose(res.x[:, j], b / (lam + s * s0), rtol=1e-12)


def test_single_tau_residual_history_equals_scipy_gmres():
    pr, op, b = small_problem(shape=(20, 20), n_p=1)
    tau = pr.tau_bar[0]
    sigma = 0.37 * tau + 0.0
    A_s = op.shifted(sigma).tocsc()
    lu = spla.splu(op.shifted(tau).tocsc())
    Aprec = spla.LinearOperator((op.n, op.n), matvec=lambda v: A_s @ lu.solve(v.astype(complex)), dtype=complex)
    m = 15
    hist_scipy = []
    spla.gmres(Aprec, b, restart=m, maxiter=1, rtol=1e-300, atol=0.0, callback=hist_scipy.append,
               callback_type="pr_norm")
    res = oracle.shifted_solve(op, b, [sigma], [tau], [0], 0.0, m, oracle.ExactInner(op, [tau]), history=True)
    ours = np.array([h[0] for h in res.hist])
    n = min(len(hist_scipy), len(ours))
    assert n >= 10
    assert np.allclose(ours[:n], np.array(hist_scipy[:n]), rtol=1e-8, atol=1e-14)


@pytest.mark.parametrize("eps", [1e-6, 1e-9, 1e-11])
def test_inexact_residual_gap_bound(eps):
    """Eq. resdiff: | ||r|| - ||r_tilde|| | <= ||r - r_tilde|| <= sum |y_i| ||p_i|| <= eps ||y||_1."""
    pr, op, b = small_problem(shape=(32, 32), n_f=8, n_p=3, seed=12)
    hier = Hierarchy(op, pr.tau_bar)
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-8, 80, GMGInner(hier, eps),
                               keep_basis=True)
    tr = oracle.true_residuals(op, b, pr.sigma, res.x) * res.beta
    for j in range(len(pr.sigma)):
        y = res.y[j]
        mj = res.m_j[j]
        gap_bound = float(np.sum(np.abs(y) * res.pnorm[:mj]))
        assert abs(tr[j] - res.res_est[j] * res.beta) <= gap_bound * (1 + 1e-8) + 1e-15
        assert gap_bound <= eps * np.sum(np.abs(y)) * (1 + 1e-12)
        assert tr[j] <= res.res_bound[j] * res.beta * (1 + 1e-8)


def test_ffom_residual_closed_form_and_prop3():
    pr, op, b = small_problem(shape=(16, 16), n_f=5, n_p=2, seed=13)
    ex = oracle.ExactInner(op, pr.tau_bar)
    m = 6
    fom = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 0.0, m, ex, variant="ffom", keep_basis=True)
    gm = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 0.0, m, ex, variant="fgmres", keep_basis=True)
    H, taus = fom.H, fom.taus
    for j, s in enumerate(pr.sigma):
        y = fom.y[j]
        # Eq. fomresidualsimplified: ||r^fom|| = |(sigma - tau_m) h_{m+1,m} e_m^T y|
        closed = abs((s - taus[m - 1]) * H[m, m - 1] * y[m - 1])
        tr = oracle.true_residuals(op, b, [s], fom.x[:, [j]])[0] * fom.beta
        assert abs(closed - tr) <= 1e-8 * tr + 1e-14
        # Prop. 3
        Hs = shifted_hessenberg(H, taus, s, m)
        eta = H[m, m - 1] * (s - taus[m - 1])
        em = np.zeros(m); em[-1] = 1
        alpha = np.linalg.norm(eta * np.linalg.solve(Hs[:m, :m].conj().T, em))
        r_f = b - op.shifted(s) @ fom.x[:, j]
        r_g = b - op.shifted(s) @ gm.x[:, j]
        assert np.linalg.norm(r_f - r_g) <= alpha * (1 + alpha) / (1 + alpha ** 2) * np.linalg.norm(r_f) * (1 + 1e-8) + 1e-13
        # GMRES minimises the residual over the same space
        assert np.linalg.norm(r_g) <= np.linalg.norm(r_f) * (1 + 1e-10) + 1e-13


def test_zero_rhs_and_schedule_cycling():
    pr, op, b = small_problem()
    res = oracle.shifted_solve(op, np.zeros(op.n), pr.sigma, pr.tau_bar, pr.schedule, 1e-8, 10,
                               oracle.ExactInner(op, pr.tau_bar))
    assert np.all(res.x == 0) and np.all(res.status == OK)
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, [1, 0, 0], 0.0, 7, oracle.ExactInner(op, pr.tau_bar))
    idx = [1, 0, 0, 1, 0, 0, 1]
    assert np.array_equal(res.taus, pr.tau_bar[idx])
    assert np.array_equal(synth.schedule(3, "cycled"), [0, 1, 2])
    assert np.array_equal(synth.schedule(2, "blocks", 6), [0, 0, 0, 1, 1, 1])


def test_planted_conjugation_mistake_is_caught(monkeypatch):
    """A plausible slip (v_i^T w instead of v_i^* w) must break a pin above."""
    import oracle.fgmres as fg
    pr, op, b = small_problem(shape=(12, 12), n_f=3)
    monkeypatch.setattr(fg.np, "vdot", lambda a, c: np.dot(a, c))
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 1e-10, 60, oracle.ExactInner(op, pr.tau_bar),
                               keep_basis=True)
    k = res.steps
    assert np.linalg.norm(res.V.conj().T @ res.V - np.eye(k + 1)) > 1e-6


def test_relaxed_inner_tolerance_is_certified_and_saves_cycles():
    """Relaxed inner tolerances (Section 4, last paragraph): every step's inner
    residual meets its own eps_k; eps_k follows the largest residual estimate of
    the shifts still iterating, which FGMRES never increases, so eps_k does not
    decrease; the solve still certifies every shift by Eq. trueresidual (the
    true residual, recomputed, is within the bound and tol); and the inner work
    is smaller than with a fixed eps."""
    pr = synth.make_problem((48, 40), n_f=24, periods=(5.0, 3600.0), n_p=3, seed=21, m_max=100)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    hier = Hierarchy(op, pr.tau_bar)
    b = pr.rhs()[:, 0]
    tol, eps, ell = 1e-8, 1e-10, 0.01
    fixed = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, tol, 100, GMGInner(hier, eps))
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, tol, 100, GMGInner(hier, eps),
                               history=True, inner_relax=ell, eps=eps)
    assert np.all(res.status == OK)
    assert res.cycles.sum() < 0.85 * fixed.cycles.sum()
    assert np.all(res.pnorm <= res.eps_k * (1 + 1e-12))          # ||v_k|| = 1
    assert res.eps_k[0] == eps and np.all(np.diff(res.eps_k) >= 0)
    for k in range(2, res.steps + 1):
        live_after = res.m_j > k - 1
        r_prev = np.max(res.hist[k - 2][live_after])
        assert res.eps_k[k - 1] == min(1e-3, max(eps, ell * tol / r_prev))
    assert res.eps_k.max() > 100 * eps
    tr = oracle.true_residuals(op, b, pr.sigma, res.x)
    assert np.all(res.res_bound <= tol)
    assert np.all(tr <= res.res_bound * (1 + 1e-9) + 1e-15)
