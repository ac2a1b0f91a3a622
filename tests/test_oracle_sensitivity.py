"""Pins of the adjoint-state sensitivities (oracle/sensitivity.py) against
things other than the formula itself: finite differences of direct solves,
the scaling identity of the measurement and adjoint reciprocity."""
import numpy as np
import pytest

from oracle.sensitivity import adjoint_rhs, direct_phasors, sensitivities


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    cond = 1e-4 * np.exp(rng.normal(0.0, 1.0, shape))
    ss = 1e-5 * np.exp(rng.normal(0.0, 0.5, shape))
    return cond, ss


CASES = [((4, 5), (10.0, 10.0), 0b0101, 2j * np.pi / 60.0),
         ((6, 3), (12.5, 8.0), 0b1111, 2j * np.pi / 600.0),
         ((3, 3, 4), (10.0, 10.0, 5.0), 0b110011, 2j * np.pi / 30.0)]


def _setup(shape, h, mask, sigma, seed):
    cond, ss = _field(shape, seed)
    n = int(np.prod(shape))
    src, meas = 1, n - 2
    b = np.zeros(n, dtype=np.complex128)
    b[src] = 1.0
    phi = direct_phasors(shape, h, cond, ss, mask, sigma, b)
    psi = direct_phasors(shape, h, cond, ss, mask, sigma, adjoint_rhs(n, meas))
    return cond, ss, b, src, meas, phi, psi


@pytest.mark.parametrize("shape,h,mask,sigma", CASES)
def test_matches_central_differences_of_direct_solves(shape, h, mask, sigma):
    """dh/dlnK_c and dh/dlnS_c against (h(p + d) - h(p - d)) / 2d, every cell."""
    cond, ss, b, src, meas, phi, psi = _setup(shape, h, mask, sigma, 7)
    jk, js = sensitivities(shape, h, cond, ss, mask, sigma, phi, psi)
    n = int(np.prod(shape))
    d = 1e-4
    fk = np.zeros(n, dtype=np.complex128)
    fs = np.zeros(n, dtype=np.complex128)
    for c in range(n):
        for field, out, other in ((cond, fk, "k"), (ss, fs, "s")):
            vals = []
            for sgn in (1.0, -1.0):
                f2 = field.copy().ravel()
                f2[c] *= np.exp(sgn * d)
                f2 = f2.reshape(shape)
                args = (f2, ss) if other == "k" else (cond, f2)
                vals.append(direct_phasors(shape, h, args[0], args[1], mask, sigma, b)[meas])
            out[c] = (vals[0] - vals[1]) / (2 * d)
    assert np.max(np.abs(jk - fk)) <= 1e-6 * np.max(np.abs(fk))
    assert np.max(np.abs(js - fs)) <= 1e-6 * np.max(np.abs(fs))


@pytest.mark.parametrize("shape,h,mask,sigma", [((16, 24), (5.0, 5.0), 0b0011, 2j * np.pi / 100.0),
                                                ((4, 5, 6), (10.0, 10.0, 10.0), 0b111111, 2j * np.pi / 20.0)])
def test_scaling_identity(shape, h, mask, sigma):
    """K and S_s scaled together by a: A -> aA, Phi -> Phi / a, so
    sum_c (dh/dlnK_c + dh/dlnS_c) = d h(a) / d ln a = -h."""
    cond, ss, b, src, meas, phi, psi = _setup(shape, h, mask, sigma, 11)
    jk, js = sensitivities(shape, h, cond, ss, mask, sigma, phi, psi)
    total = jk.sum() + js.sum()
    assert abs(total + phi[meas]) <= 1e-10 * abs(phi[meas])


def test_adjoint_reciprocity_and_no_conjugation():
    """Psi^T b = (A Psi)^T Phi = -Phi(x_m) (A complex symmetric). Conjugating
    Psi (the Hermitian adjoint) breaks both this and the derivative."""
    shape, h, mask, sigma = (5, 6), (10.0, 10.0), 0b1001, 2j * np.pi / 45.0
    cond, ss, b, src, meas, phi, psi = _setup(shape, h, mask, sigma, 3)
    assert abs(psi @ b + phi[meas]) <= 1e-12 * abs(phi[meas])
    assert abs(np.conj(psi) @ b + phi[meas]) > 1e-3 * abs(phi[meas])
    jk, js = sensitivities(shape, h, cond, ss, mask, sigma, phi, psi)
    jk2, js2 = sensitivities(shape, h, cond, ss, mask, sigma, phi, np.conj(psi))
    assert abs(jk2.sum() + js2.sum() + phi[meas]) > 1e-3 * abs(phi[meas])
    assert abs(jk.sum() + js.sum() + phi[meas]) <= 1e-10 * abs(phi[meas])


def test_storage_term_is_local():
    """Only the cell's own storage enters its dh/dlnS: sigma M_cc Psi_c Phi_c."""
    shape, h, mask, sigma = (4, 4), (10.0, 10.0), 0b1111, 2j * np.pi / 90.0
    cond, ss, b, src, meas, phi, psi = _setup(shape, h, mask, sigma, 5)
    _, js = sensitivities(shape, h, cond, ss, mask, sigma, phi, psi)
    c = 6
    assert js[c] == pytest.approx(sigma * ss.ravel()[c] * 100.0 * psi[c] * phi[c], rel=1e-14)
