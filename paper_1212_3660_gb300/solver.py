"""Convenience layer over the C ABI for synthetic problems (marshalling only).

`Solver` owns a context and an operator and calls fks_solve with numpy (host)
or torch (device) buffers. The operator is the grid operator of a
synth.Problem, or, when `csr` is given, a general sparse K and M in CSR form
(the problem then only supplies shifts, schedule, tolerance and sources). It
contains no arithmetic of the method: every step runs in libfks.so.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import fks


@dataclasses.dataclass
class SolveOutput:
    status: int
    X: object            # n_rhs x n_f x n (numpy or torch)
    res_est: np.ndarray  # n_rhs x n_f
    res_bound: np.ndarray
    res_true: np.ndarray
    m_j: np.ndarray
    shift_status: np.ndarray
    steps: np.ndarray
    inner_cycles: np.ndarray  # n_rhs x m_max
    pnorm: np.ndarray
    breakdown: np.ndarray
    gmres_alpha: np.ndarray = None  # n_rhs x n_f: Prop. 3's alpha at each shift's freeze step
    hbar: np.ndarray = None         # n_rhs x m_max x (m_max + 1): column k-1 of H_bar is hbar[r, k-1]
    tau_k: np.ndarray = None        # n_rhs x m_max


class Solver:
    def __init__(self, problem, device: int = 0, csr=None, amg=None):
        """csr: optional (k_rowptr, k_col, k_val, m_rowptr, m_col, m_val) of an n x n K and M.
        amg: for a CSR operator, True or a dict of fks_op_amg's max_levels, max_coarse, nu:
        the BiCGSTAB steps of the inner solve are then preconditioned by an AMG V-cycle."""
        self.p = problem
        self.op = None
        self.ctx = fks.fks_create(device)
        if csr is not None:
            self.op = fks.fks_op_csr(self.ctx, problem.n, *csr)
            if amg:
                fks.fks_op_amg(self.op, True, **(amg if isinstance(amg, dict) else {}))
            return
        d = problem.dim
        ncell = [problem.shape[d - 1 - a] for a in range(d)]
        self.op = fks.fks_op_grid(self.ctx, d, ncell, problem.h, problem.cond, problem.ss, problem.dirichlet_mask)

    def close(self):
        if self.op is not None:
            fks.fks_op_destroy(self.op)
            self.op = None
        if self.ctx is not None:
            fks.fks_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b=None, *, precision=fks.FKS_PREC_FP64, variant=fks.FKS_FGMRES, tol=None, m_max=None,
              inner_tol=0.0, inner_max_cycles=50, replay_cycles=None, replay_mj=None, device_out=False,
              stream=None, sigma=None, tau=None, schedule=None, launch_mode=0, inner_steps=0, assembly=0,
              inner_relax=0.0, restart_len=0, max_restarts=0):
        p = self.p
        b = p.rhs().T.copy() if b is None else b            # n_rhs x n
        n_rhs = b.shape[0]
        sigma = np.ascontiguousarray(p.sigma if sigma is None else sigma, dtype=np.complex128)
        tau = np.ascontiguousarray(p.tau_bar if tau is None else tau, dtype=np.complex128)
        sched = p.schedule if schedule is None else schedule
        m_max = p.m_max if m_max is None else m_max
        n_f = len(sigma)
        opts, keep = fks.make_options(tol=p.tol if tol is None else tol, m_max=m_max, variant=variant,
                                      precision=precision, inner_tol=inner_tol, inner_max_cycles=inner_max_cycles,
                                      schedule=sched, replay_cycles=replay_cycles, replay_mj=replay_mj,
                                      launch_mode=launch_mode, inner_steps=inner_steps,
                                      assembly=assembly, inner_relax=inner_relax, restart_len=restart_len,
                                      max_restarts=max_restarts)
        if device_out:
            import torch
            X = torch.empty((n_rhs, n_f, p.n), dtype=torch.complex128, device="cuda")
        else:
            X = np.zeros((n_rhs, n_f, p.n), dtype=np.complex128)
        est = np.zeros((n_rhs, n_f))
        bnd = np.zeros((n_rhs, n_f))
        tru = np.zeros((n_rhs, n_f))
        mj = np.zeros((n_rhs, n_f), np.int32)
        sst = np.zeros((n_rhs, n_f), np.int32)
        info, arr = fks.make_info(n_rhs, m_max, n_f)
        st = fks.fks_solve(self.op, b, n_rhs, sigma, n_f, tau, len(tau), opts, X, est, bnd, tru, mj, sst, info,
                           stream)
        return SolveOutput(st, X, est, bnd, tru, mj, sst, arr["steps"], arr["inner_cycles"].reshape(n_rhs, m_max),
                           arr["pnorm"].reshape(n_rhs, m_max), arr["breakdown"], arr["gmres_alpha"], arr["hbar"],
                           arr["tau_k"])

    def sensitivity(self, phi, psi, sigma=None, stream=None):
        """(dh/dlnK, dh/dlnS), each n_m x n_f x n complex128, from forward phasors
        phi (n_f x n) and adjoint phasors psi (n_m x n_f x n); numpy in, numpy
        out (torch tensors on the device are used in place)."""
        sigma = np.ascontiguousarray(self.p.sigma if sigma is None else sigma, dtype=np.complex128)
        n_f = len(sigma)
        if hasattr(psi, "is_cuda") and psi.is_cuda:
            import torch
            n_m = psi.shape[0]
            jk = torch.empty_like(psi)
            js = torch.empty_like(psi)
        else:
            phi = np.ascontiguousarray(phi, dtype=np.complex128)
            psi = np.ascontiguousarray(psi, dtype=np.complex128)
            n_m = psi.shape[0]
            jk = np.zeros_like(psi)
            js = np.zeros_like(psi)
        fks.fks_sensitivity(self.op, phi, psi, n_m, sigma, n_f, jk, js, stream)
        return jk, js

    def ritz(self, out):
        """(theta, status) of Prop. 1 for every source of a SolveOutput: theta
        n_rhs x m_max at sigma = 0 (the first steps[r] entries of row r are its
        Ritz values; add sigma for another shift), status per source."""
        n_rhs, m_max = out.hbar.shape[0], out.hbar.shape[1]
        theta = np.zeros((n_rhs, m_max), np.complex128)
        status = np.zeros(n_rhs, np.int32)
        steps = np.ascontiguousarray(out.steps, dtype=np.int32)
        fks.fks_ritz(self.ctx, np.ascontiguousarray(out.hbar), np.ascontiguousarray(out.tau_k), steps, n_rhs, m_max,
                     theta, status)
        return theta, status
