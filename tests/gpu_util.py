"""Helpers shared by the GPU tests: build the library once, run the oracle and
the CUDA path on the same seeded problem."""
import numpy as np
import pytest

import oracle
from oracle.gmg import Hierarchy, GMGInner
from paper_1212_3660_gb300 import build, fks, synth
from paper_1212_3660_gb300.solver import Solver


def need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    build.build()


def oracle_op(pr):
    return oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)


def oracle_run(pr, eps, variant="fgmres", src=0, exact=False):
    op = oracle_op(pr)
    b = pr.rhs()[:, src]
    inner = oracle.ExactInner(op, pr.tau_bar) if exact else GMGInner(Hierarchy(op, pr.tau_bar), eps)
    return op, oracle.shifted_solve(op, b, pr.sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max, inner,
                                    variant=variant)


def replay_arrays(pr, refs):
    """Per-source replay arrays (cycles per step, freeze step per shift) from oracle runs."""
    n_rhs = len(refs)
    rc = np.zeros((n_rhs, pr.m_max), np.int32)
    mj = np.zeros((n_rhs, len(pr.sigma)), np.int32)
    for r, ref in enumerate(refs):
        rc[r, :ref.steps] = ref.cycles
        mj[r] = ref.m_j
    return rc, mj


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def residual_floor(op, b, sigmas, X):
    """Rounding floor of a computed relative residual ||b - (K + s M) x|| / ||b||:
    8 u || |K| |x| + |s| |M| |x| || / ||b|| per shift (X: n x n_f). Residuals
    below it are not resolved by floating point on either side."""
    b = np.asarray(b).reshape(-1)
    nb = float(np.linalg.norm(b)) or 1.0
    aK, aM = abs(op.K), abs(op.M)
    out = np.zeros(len(sigmas))
    for j, s in enumerate(sigmas):
        ax = np.abs(X[:, j])
        out[j] = 8 * 2.0 ** -53 * np.linalg.norm(aK @ ax + abs(s) * (aM @ ax)) / nb
    return out
