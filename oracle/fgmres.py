"""Flexible Arnoldi + per-shift FGMRES / FFOM for (K + sigma_j M) x_j = b (oracle).

Followed passages:
  Algorithm 3 (flexible Arnoldi, Section 2.2): for k = 1..m solve
      (K + tau_k M) z_k = v_k, w = M z_k, orthogonalise w against v_1..v_k giving
      h_{1:k,k}, h_{k+1,k} = ||w||, v_{k+1} = w / h_{k+1,k}; stop if h_{k+1,k} = 0.
      Reading of the printed loop: the coefficient is h_{i,k} = v_i^* w and the
      update subtracts h_{i,k} v_i (the printed w^* v_i and v_k are typos; only this
      reading makes w orthogonal to v_i). Orthogonalisation here is modified
      Gram-Schmidt followed by one full second pass (MGS2); the coefficients of
      both passes are summed.
  Eq. shiftedarnoldimod: H_bar(sigma; T_k) = [I; 0] + H_bar_k (sigma I - T_k),
      T_k = diag(tau_1..tau_k).
  Algorithm 4: for every shift not yet converged, FGMRES takes
      y = argmin ||beta e_1 - H_bar(sigma_j; T_k) y|| (here numpy.linalg.lstsq on the
      explicit (k+1) x k matrix), FFOM solves H_k(sigma_j; T_k) y = beta e_1;
      x_j = Z_k y.
  Section 4, Eq. resdiff / Eq. trueresidual: with inexact inner solves,
      ||r_true|| <= ||beta e_1 - H_bar(sigma_j) y|| + sum_i |y_i| ||p_i||; shift j is
      declared converged when this bound is <= tol * beta (relative to
      ||r_0|| = beta, x_0 = 0, as in Section 6.1), and is then frozen with (m_j, y_j).
  Section 3 (after Prop. 3): h_{k+1,k} = 0 means the iterate is exact; the solve
      stops there (status "breakdown").
  Section 4 (last paragraph) points to inner tolerances that grow as the outer
      residual falls (Simoncini and Szyld); the paper does not pursue them. The
      optional relaxation here (relaxed_eps) follows that idea; the stopping test
      is unchanged, so a relaxed solve is certified by the same bound.

Everything is complex128 and runs one shift and one step at a time.
"""
from __future__ import annotations

import dataclasses

import numpy as np

OK, NOT_CONVERGED, BREAKDOWN = 0, 1, 2
BREAKDOWN_RTOL = 1e-13
RELAX_EPS_MAX = 1e-3      # cap on a relaxed inner tolerance


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray            # n x n_f
    m_j: np.ndarray          # steps used by each shift
    status: np.ndarray       # OK / NOT_CONVERGED / BREAKDOWN per shift
    res_est: np.ndarray      # ||beta e1 - H_bar y|| / beta
    res_bound: np.ndarray    # (||beta e1 - H_bar y|| + sum |y_i| ||p_i||) / beta
    steps: int               # Arnoldi steps taken
    breakdown: bool
    beta: float
    pnorm: np.ndarray        # ||p_k|| per step
    cycles: np.ndarray       # inner cycles per step
    taus: np.ndarray         # tau_k per step
    H: np.ndarray            # (steps+1) x steps Hessenberg
    V: np.ndarray | None = None
    Z: np.ndarray | None = None
    y: list | None = None
    hist: list | None = None     # per step: r_est / beta of every shift still live
    eps_k: np.ndarray | None = None  # per step: the relaxed inner tolerance used


def shifted_hessenberg(H, taus, sigma, k):
    """[I; 0] + H_bar_k (sigma I - T_k) as a (k+1) x k matrix (Eq. shiftedarnoldimod)."""
    E = np.zeros((k + 1, k), dtype=np.complex128)
    E[:k, :k] = np.eye(k)
    return E + H[:k + 1, :k] * (sigma - taus[:k])[None, :]


def small_solve(Hs, beta, k, variant):
    rhs = np.zeros(k + 1, dtype=np.complex128)
    rhs[0] = beta
    if variant == "fgmres":
        y = np.linalg.lstsq(Hs, rhs, rcond=None)[0]
    else:
        y = np.linalg.solve(Hs[:k, :k], rhs[:k])
    return y, float(np.linalg.norm(rhs - Hs @ y))


def relaxed_eps(eps, relax, tol, r_prev):
    """Inner tolerance of a step under relaxation (after Simoncini and Szyld, the
    theory Section 4 refers to): the inner residual may grow as the outer
    residual falls, eps_k = min(RELAX_EPS_MAX, max(eps, relax * tol / R_{k-1})),
    R_{k-1} the largest relative residual estimate of the shifts still
    iterating after step k-1 (1 before the first step). relax <= 0: eps."""
    if relax <= 0:
        return eps
    return min(RELAX_EPS_MAX, max(eps, relax * tol / r_prev))


def shifted_solve(op, b, sigmas, taus_bar, sched, tol, m_max, inner, variant="fgmres",
                  replay_mj=None, keep_basis=False, history=False, inner_relax=0.0, eps=0.0) -> SolveResult:
    """Solve (K + sigma_j M) x_j = b for all shifts from one flexible Arnoldi basis.

    op: object with .M (sparse) and .n; inner(v, tau_index, k) -> (z, cycles, ||p||);
    taus_bar: distinct preconditioner shifts; sched: tau_bar index per step, cycled.
    replay_mj: optional per-shift step at which to freeze (otherwise the bound decides).
    inner_relax > 0: the inner tolerance of step k is relaxed_eps(eps, inner_relax,
    tol, R_{k-1}) and is passed as inner(v, tau_index, k, eps_k); the stopping
    test stays the bound of Eq. trueresidual with the measured ||p_i||.
    tol may be one value or one per shift (a restarted solve gives each shift
    its own share of the tolerance); the relaxed rule uses the smallest.
    """
    n = op.n
    sigmas = np.asarray(sigmas, dtype=np.complex128)
    nf = len(sigmas)
    tols = np.broadcast_to(np.asarray(tol, dtype=np.float64), (nf,))
    tol = float(tols.min()) if nf else 0.0
    b = np.asarray(b, dtype=np.complex128).reshape(n)
    beta = float(np.linalg.norm(b))
    x = np.zeros((n, nf), dtype=np.complex128)
    m_j = np.zeros(nf, dtype=np.int64)
    status = np.full(nf, NOT_CONVERGED, dtype=np.int64)
    res_est = np.zeros(nf)
    res_bound = np.zeros(nf)
    if beta == 0.0:
        status[:] = OK
        return SolveResult(x, m_j, status, res_est, res_bound, 0, False, 0.0, np.zeros(0), np.zeros(0, int),
                           np.zeros(0, complex), np.zeros((1, 0), complex))
    V = np.zeros((n, m_max + 1), dtype=np.complex128)
    Z = np.zeros((n, m_max), dtype=np.complex128)
    H = np.zeros((m_max + 1, m_max), dtype=np.complex128)
    taus = np.zeros(m_max, dtype=np.complex128)
    pnorm = np.zeros(m_max)
    cycles = np.zeros(m_max, dtype=np.int64)
    eps_k = np.zeros(m_max)
    r_prev = 1.0
    ys = [None] * nf
    V[:, 0] = b / beta
    live = np.ones(nf, dtype=bool)
    stop_at = m_max if replay_mj is None else int(np.max(replay_mj))
    k = 0
    breakdown = False
    hist = [] if history else None
    while k < stop_at:
        k += 1
        p = int(sched[(k - 1) % len(sched)])
        taus[k - 1] = taus_bar[p]
        if inner_relax > 0:
            eps_k[k - 1] = relaxed_eps(eps, inner_relax, tol, r_prev)
            z, c, pn = inner(V[:, k - 1], p, k, eps_k[k - 1])
        else:
            z, c, pn = inner(V[:, k - 1], p, k)
        Z[:, k - 1] = z
        pnorm[k - 1] = pn
        cycles[k - 1] = c
        w = op.M @ z
        w0 = float(np.linalg.norm(w))
        for _ in range(2):                       # MGS, then one more full pass
            for i in range(k):
                hik = np.vdot(V[:, i], w)        # v_i^* w
                w = w - hik * V[:, i]
                H[i, k - 1] += hik
        hn = float(np.linalg.norm(w))
        H[k, k - 1] = hn
        breakdown = hn <= BREAKDOWN_RTOL * w0
        if not breakdown:
            V[:, k] = w / hn
        if history:
            hist.append(np.full(nf, np.nan))
        r_prev = 0.0
        for j in np.nonzero(live)[0]:
            Hs = shifted_hessenberg(H, taus, sigmas[j], k)
            y, rt = small_solve(Hs, beta, k, variant)
            if history:
                hist[-1][j] = rt / beta
            bound = rt + float(np.sum(np.abs(y) * pnorm[:k]))
            if replay_mj is not None:
                done = k == int(replay_mj[j]) or breakdown
                conv = bound <= tols[j] * beta
            else:
                conv = bound <= tols[j] * beta
                done = conv or breakdown or k == m_max
            if done:
                live[j] = False
                m_j[j] = k
                ys[j] = y
                res_est[j] = rt / beta
                res_bound[j] = bound / beta
                status[j] = OK if conv else (BREAKDOWN if breakdown else NOT_CONVERGED)
            else:
                r_prev = max(r_prev, rt / beta)
        if breakdown or not live.any():
            break
    for j in range(nf):
        if ys[j] is not None:
            x[:, j] = Z[:, :m_j[j]] @ ys[j]
    res = SolveResult(x, m_j, status, res_est, res_bound, k, bool(breakdown), beta, pnorm[:k], cycles[:k],
                      taus[:k], H[:k + 1, :k].copy())
    res.hist = hist
    res.eps_k = eps_k[:k].copy() if inner_relax > 0 else None
    if keep_basis:
        res.V = V[:, :k + 1].copy()
        res.Z = Z[:, :k].copy()
        res.y = ys
    return res


def true_residuals(op, b, sigmas, x):
    """||b - (K + sigma_j M) x_j|| / ||b|| for every shift (Eq. fomgmresresidual, first line)."""
    b = np.asarray(b, dtype=np.complex128).reshape(-1)
    beta = float(np.linalg.norm(b))
    out = np.zeros(len(sigmas))
    for j, s in enumerate(sigmas):
        r = b - (op.K @ x[:, j] + s * (op.M @ x[:, j]))
        out[j] = np.linalg.norm(r) / (beta if beta > 0 else 1.0)
    return out
