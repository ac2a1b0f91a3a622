"""Cell-centred finite-volume stiffness K and storage M (oracle).

Statement followed: the phasor equation of Section 5.1 (Eq. phasor1),
  -div(K grad Phi) + i*omega*S_s*Phi = Q0 delta(x - x_s),
with zero head on Dirichlet faces and no flow on the others, discretised on a
uniform box grid by two-point flux finite volumes (the paper uses P1 finite
elements through FEniCS; the finite-volume form keeps the same structure,
K symmetric positive definite and M diagonal and positive, as Section 2 allows).

  interior face between cells c, c' along axis a:
      t = (A_a / h_a) * 2 K_c K_c' / (K_c + K_c'),  A_a = prod_{b != a} h_b
  zero-head boundary face of cell c along axis a (head mirrored in a ghost cell):
      t = 2 K_c A_a / h_a
  (K x)_c = sum_faces t (x_c - x_nb) + sum_boundary_faces t x_c
  M = diag(S_s,c * prod_a h_a)

The matrices are assembled explicitly as scipy CSR from face lists, so the
oracle applies K and M through a general sparse product and never through a
stencil.

Dirichlet mask: bit 2a is the low face and bit 2a+1 the high face of grid axis
a (a = 0 is x, the fastest axis).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class GridOperator:
    shape: tuple             # numpy order, x fastest
    h: tuple                 # grid-axis order (hx, hy[, hz])
    K: sp.csr_matrix         # real symmetric stiffness
    M: sp.csr_matrix         # real diagonal storage
    m_diag: np.ndarray       # diagonal of M
    t_lo: list               # per grid axis: t of the low face of each cell (0 if none)
    t_hi: list               # per grid axis: t of the high face of each cell (0 if none)
    dirichlet_mask: int

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))

    def shifted(self, s: complex) -> sp.csr_matrix:
        return (self.K + s * self.M).tocsr()


def face_transmissibilities(shape, h, cond, dirichlet_mask):
    """t_lo[a], t_hi[a]: transmissibility of each cell's low / high face on grid
    axis a, as full-grid arrays (an interior face appears in both cells)."""
    d = len(shape)
    t_lo, t_hi = [], []
    for a in range(d):
        q = d - 1 - a                      # numpy axis of grid axis a
        area = float(np.prod([h[b] for b in range(d) if b != a]))
        geo = area / h[a]
        lo = np.zeros(shape)
        hi = np.zeros(shape)
        # interior faces: between index i and i+1 along numpy axis q
        k0 = np.take(cond, np.arange(shape[q] - 1), axis=q)
        k1 = np.take(cond, np.arange(1, shape[q]), axis=q)
        tf = geo * 2.0 * k0 * k1 / (k0 + k1)
        sl_hi = [slice(None)] * d
        sl_hi[q] = slice(0, shape[q] - 1)
        sl_lo = [slice(None)] * d
        sl_lo[q] = slice(1, shape[q])
        hi[tuple(sl_hi)] = tf
        lo[tuple(sl_lo)] = tf
        # boundary faces
        first = [slice(None)] * d
        first[q] = slice(0, 1)
        last = [slice(None)] * d
        last[q] = slice(shape[q] - 1, shape[q])
        if dirichlet_mask >> (2 * a) & 1:
            lo[tuple(first)] = 2.0 * geo * cond[tuple(first)]
        if dirichlet_mask >> (2 * a + 1) & 1:
            hi[tuple(last)] = 2.0 * geo * cond[tuple(last)]
        t_lo.append(lo)
        t_hi.append(hi)
    return t_lo, t_hi


def matrix_from_faces(shape, t_lo, t_hi) -> sp.csr_matrix:
    """K = sum over faces t (e_c - e_c')(e_c - e_c')^T + boundary faces t e_c e_c^T."""
    d = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape)
    rows, cols, vals = [], [], []
    diag = np.zeros(shape)
    for a in range(d):
        q = d - 1 - a
        diag += t_lo[a] + t_hi[a]
        c0 = np.take(idx, np.arange(shape[q] - 1), axis=q).ravel()
        c1 = np.take(idx, np.arange(1, shape[q]), axis=q).ravel()
        tf = np.take(t_hi[a], np.arange(shape[q] - 1), axis=q).ravel()
        rows += [c0, c1]
        cols += [c1, c0]
        vals += [-tf, -tf]
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag.ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def assemble(shape, h, cond, ss, dirichlet_mask) -> GridOperator:
    """Build K and M for cell conductivity `cond` and specific storage `ss`."""
    shape = tuple(int(s) for s in shape)
    cond = np.asarray(cond, dtype=np.float64).reshape(shape)
    ss = np.asarray(ss, dtype=np.float64).reshape(shape)
    t_lo, t_hi = face_transmissibilities(shape, h, cond, dirichlet_mask)
    K = matrix_from_faces(shape, t_lo, t_hi)
    m = (ss * float(np.prod(h))).ravel()
    M = sp.diags(m).tocsr()
    return GridOperator(shape, tuple(h), K, M, m, t_lo, t_hi, dirichlet_mask)
