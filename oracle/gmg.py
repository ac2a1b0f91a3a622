"""Geometric-multigrid inner solve (oracle).

The paper applies the preconditioners (K + tau_k M)^{-1} inexactly by an inner
iterative solver (Section 4, Eq. zmmoditer): z_k ~ (K + tau_k M)^{-1} v_k with
p_k = v_k - (K + tau_k M) z_k and ||p_k|| <= eps ||v_k||. Its own inner solver was
smoothed-aggregation AMG + BiCGSTAB (Section 6); this build uses geometric
multigrid on the structured grid instead. The multigrid specification below is
this build's own (the paper gives none); the GPU path implements the same
specification independently:

  levels   coarsen grid axis a by 2 while n_a is even and n_a > 4 (per axis);
           stop when no axis coarsens. If the coarsest level so formed has more
           than MAX_COARSE cells (too large for the exact solve), the hierarchy
           is formed again with "ragged" halving: while a level has more than
           MAX_COARSE cells, an odd axis with n_a > 4 also coarsens, to
           (n_a + 1) / 2 cells, children 2I and 2I + 1 except the last coarse
           cell, whose only child is the last fine cell.
  coarse   face transmissibility = (sum of the fine faces on the coarse face)
           x (fine centre distance across it) / (coarse centre distance), the
           distances from the cell widths in fine cells (a zero-head boundary face:
           the half widths); on evenly halved axes this is the sum / r_a. A ragged
           axis's last coarse cell keeps its lone child's width, so its faces are
           those of a two-point flux discretisation on the non-uniform coarse
           cells (a plain / r_a there made V-cycles diverge on grids like 289^2,
           whose one-cell-wide edge cells persist through several levels).
           Coarse storage = sum of the children.
  R        restriction = sum of the children.
  P        prolongation = cell-centred (bi/tri)linear interpolation, weights 3/4
           and 1/4 per coarsened axis; beyond a zero-head face the coarse ghost
           is minus the boundary cell, beyond a no-flow face it equals it.
  smoother red-black Gauss-Seidel (red: sum of grid indices even); pre-smoothing
           nu1 = 2 sweeps red then black, post-smoothing nu2 = 2 sweeps black then red.
  coarsest exact solve (dense LU).
  cycle    V-cycle from a zero initial guess on every level.
  outer    stationary iteration z <- z + V(v - A z) from z = 0, stopping when
           ||v - A z|| <= eps ||v|| or after max_cycles cycles; ||p|| = final
           ||v - A z|| is returned (computed exactly).

Everything here uses scipy sparse matrices built by Kronecker products and a
general sparse matrix-vector product; the red-black sweep updates all cells of
one colour from the full residual, which equals Gauss-Seidel over that colour
because cells of one colour are not coupled by the 2d+1-point operator.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .operator import matrix_from_faces

NU1 = 2
NU2 = 2
MAX_COARSE = 1024   # largest coarsest level (cells) solved exactly


def _ratios(shape, ragged=False):
    # numpy axis order; grid axis a = d-1-q. Ragged: odd axes > 4 also halve
    # (rounding up) while the level has more than MAX_COARSE cells.
    big = ragged and int(np.prod(shape)) > MAX_COARSE
    return tuple(2 if (s > 4 and (s % 2 == 0 or big)) else 1 for s in shape)


def _coarsen_sum(arr, r, sel_q=None, sel_off=None):
    """Sum over the children of each coarse cell (children 2I, 2I + 1 per
    coarsened axis; an odd axis's last coarse cell has the one child 2I). With
    sel_q, only the child at offset sel_off along numpy axis sel_q is taken: 0
    is the first child, r - 1 the last one (the lone child of a ragged cell)."""
    d = arr.ndim
    for q in range(d):
        if r[q] == 2 and arr.shape[q] % 2 == 1:
            # pad the odd axis to even: with zeros (no second child), or, where
            # the last child is selected, with a copy of the lone child
            pad = [(0, 0)] * d
            pad[q] = (0, 1)
            mode = "edge" if (q == sel_q and sel_off == r[q] - 1) else "constant"
            arr = np.pad(arr, pad, mode=mode)
    new = []
    for n, rq in zip(arr.shape, r):
        new += [n // rq, rq]
    x = arr.reshape(new)
    if sel_q is not None:
        x = np.take(x, [sel_off], axis=2 * sel_q + 1)
    return x.sum(axis=tuple(2 * q + 1 for q in range(d)))


def _face_factors(w, r):
    """Per coarse cell along one axis, the factors of its low and high faces
    (fine centre distance / coarse centre distance, or half widths at the
    boundary), and the coarse widths; w = fine cell widths in finest cells."""
    n = len(w)
    if r == 1:
        return np.ones(n), np.ones(n), w.copy()
    nc = (n + 1) // 2
    W = np.array([w[2 * I:2 * I + 2].sum() for I in range(nc)])
    lo = np.empty(nc)
    hi = np.empty(nc)
    for I in range(nc):
        first, last = 2 * I, min(2 * I + 1, n - 1)
        lo[I] = w[first] / W[I] if I == 0 else (w[first - 1] + w[first]) / (W[I - 1] + W[I])
        hi[I] = w[last] / W[I] if I == nc - 1 else (w[last] + w[last + 1]) / (W[I] + W[I + 1])
    return lo, hi, W


def _prolong_1d(n_f, n_c, r, dirichlet_lo, dirichlet_hi):
    if r == 1:
        return sp.identity(n_c, format="csr")
    rows, cols, vals = [], [], []
    for i in range(n_f):
        parent = i // 2
        nb = parent - 1 if i % 2 == 0 else parent + 1
        rows.append(i); cols.append(parent); vals.append(0.75)
        if 0 <= nb < n_c:
            rows.append(i); cols.append(nb); vals.append(0.25)
        else:
            dir_face = dirichlet_lo if nb < 0 else dirichlet_hi
            rows.append(i); cols.append(parent); vals.append(-0.25 if dir_face else 0.25)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_f, n_c))


def _restrict_1d(n_f, n_c, r):
    if r == 1:
        return sp.identity(n_c, format="csr")
    cols = np.arange(n_f)
    return sp.csr_matrix((np.ones(n_f), (cols // 2, cols)), shape=(n_c, n_f))


def _kron_all(mats):
    out = mats[0]
    for m in mats[1:]:
        out = sp.kron(out, m, format="csr")
    return out.tocsr()


class Level:
    def __init__(self, shape, h, t_lo, t_hi, m_diag, mask):
        self.shape = tuple(shape)
        self.h = tuple(h)
        self.t_lo = t_lo
        self.t_hi = t_hi
        self.m = m_diag.reshape(-1)
        self.mask = mask
        self.K = matrix_from_faces(self.shape, t_lo, t_hi)
        self.M = sp.diags(self.m).tocsr()
        d = len(shape)
        coords = np.indices(self.shape).sum(axis=0)
        self.red = (coords % 2 == 0).ravel()
        self.black = ~self.red
        self.P = None   # prolongation from the next coarser level
        self.R = None   # restriction to the next coarser level

    @property
    def n(self):
        return int(np.prod(self.shape))


class Hierarchy:
    """Multigrid levels of K, M and, per distinct tau, the shifted matrices."""

    def __init__(self, op, taus, max_coarse=None):
        self._build(op, ragged=False)
        if self.levels[-1].n > MAX_COARSE:
            self._build(op, ragged=True)
        self.taus = np.asarray(taus, dtype=np.complex128)
        self.A = [[(L.K + t * L.M).tocsr() for L in self.levels] for t in self.taus]
        self.D = [[A.diagonal() for A in As] for As in self.A]
        self.coarse_lu = [sla.lu_factor(As[-1].toarray()) for As in self.A]

    def _build(self, op, ragged):
        d = len(op.shape)
        lev = Level(op.shape, op.h, op.t_lo, op.t_hi, op.m_diag, op.dirichlet_mask)
        self.levels = [lev]
        widths = [np.ones(s) for s in op.shape]   # per numpy axis, in finest cells
        while True:
            r = _ratios(lev.shape, ragged)
            if all(x == 1 for x in r):
                break
            cshape = tuple((s + x - 1) // x for s, x in zip(lev.shape, r))
            ch = tuple(lev.h[a] * r[d - 1 - a] for a in range(d))
            facs = [_face_factors(widths[q], r[q]) for q in range(d)]
            widths = [f[2] for f in facs]
            t_lo, t_hi = [], []
            for a in range(d):
                q = d - 1 - a
                shp = [1] * d
                shp[q] = cshape[q]
                t_lo.append(_coarsen_sum(lev.t_lo[a], r, q, 0) * facs[q][0].reshape(shp))
                t_hi.append(_coarsen_sum(lev.t_hi[a], r, q, r[q] - 1) * facs[q][1].reshape(shp))
            cm = _coarsen_sum(lev.m.reshape(lev.shape), r)
            clev = Level(cshape, ch, t_lo, t_hi, cm, op.dirichlet_mask)
            p1 = []
            r1 = []
            for q in range(d):
                a = d - 1 - q
                p1.append(_prolong_1d(lev.shape[q], cshape[q], r[q], op.dirichlet_mask >> (2 * a) & 1,
                                      op.dirichlet_mask >> (2 * a + 1) & 1))
                r1.append(_restrict_1d(lev.shape[q], cshape[q], r[q]))
            lev.P = _kron_all(p1)
            lev.R = _kron_all(r1)
            self.levels.append(clev)
            lev = clev

    def vcycle(self, p, f, lev=0):
        """One V-cycle for (K + tau_p M) e = f on level `lev`, zero initial guess."""
        A = self.A[p][lev]
        if lev == len(self.levels) - 1:
            return sla.lu_solve(self.coarse_lu[p], f)
        L = self.levels[lev]
        D = self.D[p][lev]
        z = np.zeros_like(f)
        for _ in range(NU1):
            for mask in (L.red, L.black):
                r = f - A @ z
                z[mask] += r[mask] / D[mask]
        r = f - A @ z
        ec = self.vcycle(p, L.R @ r, lev + 1)
        z = z + L.P @ ec
        for _ in range(NU2):
            for mask in (L.black, L.red):
                r = f - A @ z
                z[mask] += r[mask] / D[mask]
        return z

    def solve(self, v, p, eps, max_cycles=50, cycles=None):
        """Stationary multigrid iteration for (K + tau_p M) z = v from z = 0.

        Stops when ||v - A z|| <= eps ||v|| (or after max_cycles); with `cycles`
        given it runs exactly that many cycles. Returns (z, cycles_done, ||p||)."""
        A = self.A[p][0]
        z = np.zeros_like(v)
        r = v.copy()
        nr = np.linalg.norm(r)
        nv = np.linalg.norm(v)
        c = 0
        while (c < cycles) if cycles is not None else (nr > eps * nv and c < max_cycles):
            z = z + self.vcycle(p, r)
            c += 1
            r = v - A @ z
            nr = np.linalg.norm(r)
        return z, c, nr


class GMGInner:
    """Inner solve callable for the shifted solver: (v, tau_index, k) -> (z, cycles, ||p||)."""

    def __init__(self, hier: Hierarchy, eps: float, max_cycles: int = 50, replay_cycles=None):
        self.hier = hier
        self.eps = eps
        self.max_cycles = max_cycles
        self.replay = None if replay_cycles is None else list(replay_cycles)

    def __call__(self, v, p, k, eps=None):
        cyc = None if self.replay is None else int(self.replay[k - 1])
        return self.hier.solve(v, p, self.eps if eps is None else eps, self.max_cycles, cyc)
