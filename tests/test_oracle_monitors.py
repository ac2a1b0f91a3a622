"""Pins of the convergence monitors (oracle/monitors.py; Section 3, Props. 1-3)
against things other than their formulas: explicit products with K and M on
the basis of an exact-inner run, the spectrum of (K, M) when the Krylov space is
the whole space, the true FFOM residual, and a QR factorisation (the route the
GPU takes for Prop. 3's alpha)."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from oracle.monitors import (fom_residual_bound, gmres_alpha, ritz_pairs, ritz_residual_norms,
                             square_shifted)
from paper_1212_3660_gb300 import synth


def _run(shape, n_f, seed, m, variant="fgmres", tol=0.0):
    pr = synth.make_problem(shape, n_f=n_f, periods=(10.0, 1000.0), n_p=2, seed=seed)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, tol, m, oracle.ExactInner(op, pr.tau_bar),
                               variant=variant, keep_basis=True)
    return pr, op, b, res


def test_ritz_residuals_and_petrov_galerkin_explicit():
    """Eq. residualritzeigen against (K + sigma M) M^{-1} u - theta u formed with
    the sparse K and M, u = V_{m+1} H_bar f; and that residual is orthogonal to
    V_m (Eq. petrovgalerkin)."""
    pr, op, b, res = _run((12, 14), 3, 21, 9)
    m = res.steps
    V, H, taus = res.V, res.H, res.taus
    Minv = 1.0 / op.m_diag
    for s in pr.sigma:
        theta, F = ritz_pairs(H, taus, s, m)
        rho = ritz_residual_norms(H, taus, s, m, theta, F)
        for k in range(m):
            u = V @ (H @ F[:, k])
            r = op.shifted(s) @ (Minv * u) - theta[k] * u
            assert abs(np.linalg.norm(r) - rho[k]) <= 1e-7 * max(np.linalg.norm(u) * abs(theta[k]), 1e-300)
            assert np.linalg.norm(V[:, :m].conj().T @ r) <= 1e-7 * max(np.linalg.norm(r), 1e-12 * np.linalg.norm(u))


def test_ritz_values_move_with_the_shift():
    """H_m^{-1} H_m(sigma; T) = H_m^{-1} + sigma I - T: the Ritz values at sigma are
    those at sigma' plus (sigma - sigma')."""
    pr, op, b, res = _run((10, 10), 4, 22, 8)
    m = res.steps
    t0 = np.sort_complex(ritz_pairs(res.H, res.taus, 0.0, m)[0])
    for s in pr.sigma:
        ts = np.sort_complex(ritz_pairs(res.H, res.taus, s, m)[0] - s)
        assert np.max(np.abs(ts - t0)) <= 1e-9 * np.max(np.abs(t0))


def test_full_space_ritz_values_are_the_spectrum_of_K_M():
    """With the Krylov space the whole space (m = n, exact inner solves), the Ritz
    values of (K + sigma M) M^{-1} are lambda + sigma, lambda the eigenvalues of
    K x = lambda M x."""
    pr = synth.make_problem((3, 4), n_f=2, periods=(10.0, 1000.0), n_p=2, seed=23)
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(op.n) + 1j * rng.standard_normal(op.n)
    res = oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, 0.0, op.n, oracle.ExactInner(op, pr.tau_bar),
                               keep_basis=True)
    m = res.steps
    assert m == op.n
    lam = sla.eigh(op.K.toarray(), op.M.toarray(), eigvals_only=True)
    s = pr.sigma[1]
    theta = np.sort_complex(ritz_pairs(res.H, res.taus, s, m)[0] - s)
    assert np.max(np.abs(theta.imag)) <= 1e-8 * np.max(lam)
    assert np.max(np.abs(np.sort(theta.real) - np.sort(lam))) <= 1e-8 * np.max(lam)


@pytest.mark.parametrize("m", [3, 6, 10])
def test_prop2_bounds_the_true_ffom_residual(m):
    pr, op, b, res = _run((14, 12), 5, 24, m, variant="ffom")
    for j, s in enumerate(pr.sigma):
        tr = oracle.true_residuals(op, b, [s], res.x[:, [j]])[0] * res.beta
        assert tr <= fom_residual_bound(res.H, res.taus, s, res.steps, res.beta) * (1 + 1e-8) + 1e-14


def test_prop3_alpha_is_the_tangent_of_the_last_rotation():
    """alpha = |eta| / |R_mm| with H_m(sigma; T) = Q R (the last row of R^{-1} is
    e_m^T / R_mm and Q is unitary): the form the GPU's Givens update records."""
    pr, op, b, res = _run((12, 12), 6, 25, 7)
    m = res.steps
    for s in pr.sigma:
        R = np.linalg.qr(square_shifted(res.H, res.taus, s, m))[1]
        eta = res.H[m, m - 1] * (s - res.taus[m - 1])
        assert gmres_alpha(res.H, res.taus, s, m) == pytest.approx(abs(eta) / abs(R[m - 1, m - 1]), rel=1e-10)
