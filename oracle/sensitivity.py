"""Sensitivities of the phasor measurements by the adjoint-state method (oracle).

Test infrastructure: imported by the tests only, never by the product path.

Followed passages:
  Eq. measurement: sensor i records the phasor at its location, h_i = Phi(x_i)
      (the real and imaginary parts are the two coefficients per frequency).
  Eq. adjoint: the adjoint phasor of sensor m at frequency omega solves the same
      operator with the right-hand side -delta(x - x_m); K + sigma M is complex
      symmetric (K, M real symmetric), so the adjoint operator is the operator.
  Eq. sensitivity and Algorithm 6: dh/ds_j is the domain integral of
      [i omega dS_s/ds_j Phi - dQ_0/ds_j] Psi + dK/ds_j grad Phi . grad Psi.
      In the cell-centred discretisation (oracle/operator.py) the same
      derivation reads: A(p) Phi = b, h = e_m^T Phi, A Psi = -e_m give
      dh/dp = Psi^T (dA/dp) Phi, with no conjugation (A^T = A), and dQ_0/dp = 0
      for the spatial parameters below.

Parameters: s = ln K_c and ln S_s,c of every cell c.
  d/d ln S_c:  dA/dp = sigma * M_cc e_c e_c^T           -> sigma M_cc Psi_c Phi_c
  d/d ln K_c:  each face of cell c with transmissibility t contributes
      t (x_c - x_nb)(x_c - x_nb)^T to K (interior face) or t x_c x_c^T
      (zero-head boundary face), so
      interior face:  (dt/dlnK_c) (Psi_c - Psi_nb)(Phi_c - Phi_nb),
                      t = g 2 K_c K_nb / (K_c + K_nb),  dt/dlnK_c = g 2 K_c K_nb^2 / (K_c + K_nb)^2
      boundary face:  (dt/dlnK_c) Psi_c Phi_c,  t = 2 g K_c,  dt/dlnK_c = 2 g K_c
      with g = A_a / h_a the face's area over the cell spacing (the grad Phi .
      grad Psi term of Eq. sensitivity, face by face).

Everything is complex128; the face loops are plain NumPy over each grid axis.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .operator import assemble


def sensitivities(shape, h, cond, ss, dirichlet_mask, sigma, phi, psi):
    """(dh/dlnK, dh/dlnS) per cell for one shift sigma, forward phasor phi and
    adjoint phasor psi (flat, x fastest). Returns two complex arrays of n."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    cond = np.asarray(cond, dtype=np.float64).reshape(shape)
    ss = np.asarray(ss, dtype=np.float64).reshape(shape)
    phi = np.asarray(phi, dtype=np.complex128).reshape(shape)
    psi = np.asarray(psi, dtype=np.complex128).reshape(shape)
    jk = np.zeros(shape, dtype=np.complex128)
    for a in range(d):
        q = d - 1 - a                                   # numpy axis of grid axis a
        g = float(np.prod([h[b] for b in range(d) if b != a])) / h[a]
        lo = [slice(None)] * d
        hi = [slice(None)] * d
        lo[q] = slice(0, shape[q] - 1)                  # cell c of the face (c, c+1)
        hi[q] = slice(1, shape[q])                      # its neighbour
        lo, hi = tuple(lo), tuple(hi)
        kc, kn = cond[lo], cond[hi]
        prod = (psi[lo] - psi[hi]) * (phi[lo] - phi[hi])
        jk[lo] += g * 2.0 * kc * kn ** 2 / (kc + kn) ** 2 * prod
        jk[hi] += g * 2.0 * kn * kc ** 2 / (kc + kn) ** 2 * prod
        first = [slice(None)] * d
        last = [slice(None)] * d
        first[q] = slice(0, 1)
        last[q] = slice(shape[q] - 1, shape[q])
        first, last = tuple(first), tuple(last)
        if dirichlet_mask >> (2 * a) & 1:
            jk[first] += 2.0 * g * cond[first] * psi[first] * phi[first]
        if dirichlet_mask >> (2 * a + 1) & 1:
            jk[last] += 2.0 * g * cond[last] * psi[last] * phi[last]
    vol = float(np.prod(h))
    js = sigma * ss * vol * psi * phi
    return jk.ravel(), js.ravel()


def adjoint_rhs(n, cell):
    """Right-hand side of Eq. adjoint for a sensor in `cell`: -e_cell."""
    r = np.zeros(n, dtype=np.complex128)
    r[cell] = -1.0
    return r


def direct_phasors(shape, h, cond, ss, dirichlet_mask, sigma, rhs):
    """(K + sigma M)^{-1} rhs by sparse LU (small grids)."""
    op = assemble(shape, h, cond, ss, dirichlet_mask)
    return spla.splu(op.shifted(sigma).tocsc()).solve(np.asarray(rhs, dtype=np.complex128))
