"""Restarted flexible FOM for shifted systems (oracle).

Test infrastructure: imported by the tests only, never by the product path.

Followed passages:
  Section 2.2.2 (Restarting): for FOM the residuals of all shifts are collinear,
      so the Arnoldi process restarts on the common residual direction with each
      shift's right-hand side scaled by its own scalar (the paper points to
      Simoncini 2003 and Gu et al. 2007 and does not explore it further).
  Eq. fomresidualsimplified: after m steps the FFOM residual of shift j is
      -v_{m+1} (sigma_j - tau_m) h_{m+1,m} e_m^* y_j, i.e. c_j v_{m+1} with
      c_j = -(sigma_j - tau_m) h_{m+1,m} y_{j,m}.
  Section 6 (experiments): beyond m steps the same sequence of preconditioners
      is recycled; here step k of the whole run takes tau from the schedule at
      (k - 1) mod len, across restarts.
  Eq. trueresidual with inexact inner solves: a cycle leaves on x_j an error
      that its estimate does not see, bounded by sum_i |y_i| ||p_i|| of that
      cycle. The restart carries it: with the residual estimate of the current
      iterate C_j v (v of unit norm) and the accumulated unseen part A_j
      (absolute), the next cycle solves (K + sigma_j M) d = v, x_j += C_j d, and
      a shift is certified when |C_j| bound_cycle + A_j <= tol ||b||, i.e. when the
      cycle's own bound reaches tol_j = (tol ||b|| - A_j) / |C_j|.

Each cycle is one call of oracle.fgmres.shifted_solve (FFOM) on the shifts not
yet certified, with per-shift tolerances.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .fgmres import OK, NOT_CONVERGED, BREAKDOWN, shifted_solve


@dataclasses.dataclass
class RestartResult:
    x: np.ndarray           # n x n_f
    status: np.ndarray      # OK / NOT_CONVERGED / BREAKDOWN per shift
    res_est: np.ndarray     # |C_j| est_cycle / ||b|| at the end
    res_bound: np.ndarray   # (|C_j| bound_cycle + A_j) / ||b||
    m_j: np.ndarray         # steps of the whole run at which shift j was certified
    cycles: int             # cycles run
    steps: int              # Arnoldi steps of the whole run


def restarted_ffom(op, b, sigmas, taus_bar, sched, tol, cycle_len, max_cycles, inner):
    sigmas = np.asarray(sigmas, dtype=np.complex128)
    nf = len(sigmas)
    b = np.asarray(b, dtype=np.complex128).reshape(op.n)
    beta0 = float(np.linalg.norm(b))
    x = np.zeros((op.n, nf), dtype=np.complex128)
    status = np.full(nf, NOT_CONVERGED, dtype=np.int64)
    est = np.zeros(nf)
    bnd = np.zeros(nf)
    mj = np.zeros(nf, dtype=np.int64)
    if beta0 == 0.0:
        status[:] = OK
        return RestartResult(x, status, est, bnd, mj, 0, 0)
    sched = np.asarray(sched)
    C = np.full(nf, beta0, dtype=np.complex128)   # residual estimate of x_j: C_j v
    A = np.zeros(nf)                              # accumulated unseen part
    v = b / beta0
    live = np.arange(nf)
    done_steps = 0
    cycles = 0
    for c in range(max_cycles):
        if live.size == 0:
            break
        cycles += 1
        tol_j = (tol * beta0 - A[live]) / np.abs(C[live])
        if np.any(tol_j <= 0):
            # the unseen part alone exceeds the tolerance: not certifiable
            bad = live[tol_j <= 0]
            status[bad] = NOT_CONVERGED
            keep = tol_j > 0
            live, tol_j = live[keep], tol_j[keep]
            if live.size == 0:
                break
        sched_c = np.roll(sched, -(done_steps % len(sched)))
        res = shifted_solve(op, v, sigmas[live], taus_bar, sched_c, tol_j, cycle_len, inner, variant="ffom",
                            keep_basis=True)
        k = res.steps
        next_live = []
        for i, j in enumerate(live):
            x[:, j] += C[j] * res.x[:, i]
            if res.status[i] in (OK, BREAKDOWN):
                status[j] = OK if res.status[i] == OK else BREAKDOWN
                est[j] = abs(C[j]) * res.res_est[i] / beta0
                bnd[j] = (abs(C[j]) * res.res_bound[i] + A[j]) / beta0
                mj[j] = done_steps + int(res.m_j[i])
            else:
                y = res.y[i]
                m = int(res.m_j[i])
                coef = -(sigmas[j] - res.taus[m - 1]) * res.H[m, m - 1] * y[m - 1]
                A[j] += abs(C[j]) * (res.res_bound[i] - res.res_est[i])
                C[j] = C[j] * coef
                est[j] = abs(C[j]) / beta0
                bnd[j] = (abs(C[j]) + A[j]) / beta0
                mj[j] = done_steps + m
                next_live.append(j)
        done_steps += k
        if res.breakdown:
            break
        v = res.V[:, k].copy()       # v_{m+1}, the common residual direction
        live = np.asarray(next_live, dtype=np.int64)
    return RestartResult(x, status, est, bnd, mj, cycles, done_steps)
