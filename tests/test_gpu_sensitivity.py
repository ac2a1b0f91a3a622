"""GPU adjoint-state sensitivities (fks_sensitivity) against the oracle
(oracle/sensitivity.py): element by element on seeded phasors, end to end from
GPU forward and adjoint solves, and at the 512 x 512 workload's size."""
import numpy as np
import pytest

from oracle.sensitivity import adjoint_rhs, direct_phasors, sensitivities
from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from csr_util import csr_arrays, fe_like, sparse_problem
from gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _random_phasors(rng, n_m, n_f, n):
    phi = rng.standard_normal((n_f, n)) + 1j * rng.standard_normal((n_f, n))
    psi = rng.standard_normal((n_m, n_f, n)) + 1j * rng.standard_normal((n_m, n_f, n))
    return phi, psi


def _check_against_oracle(pr, phi, psi, jk, js, tol=1e-12):
    for m in range(psi.shape[0]):
        for j, s in enumerate(pr.sigma):
            ok, os_ = sensitivities(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask, s, phi[j], psi[m, j])
            assert np.max(np.abs(jk[m, j] - ok)) <= tol * np.max(np.abs(ok)), (m, j)
            assert np.max(np.abs(js[m, j] - os_)) <= tol * np.max(np.abs(os_)), (m, j)


@pytest.mark.parametrize("shape,mask", [((27, 40), 0b0110), ((7, 9, 10), 0b101101), ((2, 301), 0b0011)])
def test_matches_oracle_elementwise(shape, mask):
    """Random phasors (the formula is bilinear, so any inputs test it): every
    entry within 1e-12 of the oracle; several blocks and a ragged tail, 2D, 3D
    and a two-row grid of odd length, zero-head and no-flow faces mixed; host
    and device arrays."""
    need_gpu()
    import torch
    pr = synth.make_problem(shape, n_f=3, periods=(5.0, 3600.0), n_p=2, seed=41, dirichlet_mask=mask)
    s = Solver(pr)
    rng = np.random.default_rng(5)
    phi, psi = _random_phasors(rng, 2, 3, pr.n)
    jk, js = s.sensitivity(phi, psi)
    _check_against_oracle(pr, phi, psi, jk, js)
    jkd, jsd = s.sensitivity(torch.from_numpy(phi).cuda(), torch.from_numpy(psi).cuda())
    assert np.array_equal(jkd.cpu().numpy(), jk) and np.array_equal(jsd.cpu().numpy(), js)
    s.close()


def test_full_size_512x512():
    """The workload's grid (512 x 512, its field and boundary), four shifts and
    two measurements, device arrays: every entry against the oracle."""
    need_gpu()
    import torch
    pr = synth.workload(2, m_max=100)
    sig = pr.sigma[::50].copy()
    s = Solver(pr)
    rng = np.random.default_rng(6)
    phi, psi = _random_phasors(rng, 2, len(sig), pr.n)
    jk, js = s.sensitivity(torch.from_numpy(phi).cuda(), torch.from_numpy(psi).cuda(), sigma=sig)
    pr.sigma = sig
    _check_against_oracle(pr, phi, psi, jk.cpu().numpy(), js.cpu().numpy())
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_jacobian_from_gpu_solves(precision):
    """Algorithm 6 on the GPU: forward solve, adjoint solves for three sensors
    (right-hand sides -e_m, one batched fks_solve), sensitivities. Against the
    oracle's sensitivities from direct phasors, and the scaling identity
    sum_c (dh/dlnK_c + dh/dlnS_c) = -h on the GPU's own outputs. Both hold to
    the solves' accuracy: with residuals r_Phi, r_Psi of relative size 1e-8,
    sum_c J + h = dPhi_m - Phi^T r_Psi - Psi^T r_Phi, amplified by
    ||Phi|| / |Phi_m| and the conditioning of K + sigma M. Periods of
    300-3600 s and sensors 5-10 cells from the source keep h well above the
    solves' absolute accuracy (the oracle with residuals of that size moves
    both measures by at most 3.4e-7 here; at 5 s periods the phasor decays by
    1e-11 over this grid and h at a far sensor is below the solver's noise)."""
    need_gpu()
    pr = synth.make_problem((40, 48), n_f=6, periods=(300.0, 3600.0), n_p=3, seed=43, m_max=100)
    s = Solver(pr)
    fwd = s.solve(precision=precision, inner_tol=1e-10)
    assert fwd.status == fks.FKS_OK
    sensors = [24 * 48 + 30, 14 * 48 + 18, 28 * 48 + 20]
    b_adj = np.stack([adjoint_rhs(pr.n, m) for m in sensors])
    adj = s.solve(b_adj, precision=precision, inner_tol=1e-10)
    assert adj.status == fks.FKS_OK
    phi = fwd.X[0]
    psi = adj.X
    jk, js = s.sensitivity(phi, psi)
    for mi, m in enumerate(sensors):
        for j, sg in enumerate(pr.sigma):
            h = phi[j, m]
            total = jk[mi, j].sum() + js[mi, j].sum()
            assert abs(total + h) <= 1e-5 * abs(h), (mi, j, abs(total + h) / abs(h))
            ph = direct_phasors(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask, sg, pr.rhs()[:, 0])
            ps = direct_phasors(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask, sg, adjoint_rhs(pr.n, m))
            ok, os_ = sensitivities(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask, sg, ph, ps)
            assert np.max(np.abs(jk[mi, j] - ok)) <= 1e-5 * np.max(np.abs(ok)), (mi, j)
            assert np.max(np.abs(js[mi, j] - os_)) <= 1e-5 * np.max(np.abs(os_)), (mi, j)
    s.close()


def test_invalid_arguments_rejected():
    need_gpu()
    pr = synth.make_problem((16, 16), n_f=2, periods=(5.0, 3600.0), n_p=1, seed=44)
    s = Solver(pr)
    phi = np.zeros((2, pr.n), np.complex128)
    psi = np.zeros((1, 2, pr.n), np.complex128)
    out = np.zeros_like(psi)
    with pytest.raises(fks.FksError):
        fks.fks_sensitivity(s.op, phi, psi, 0, pr.sigma, 2, out, out)
    with pytest.raises(fks.FksError):
        fks.fks_sensitivity(s.op, phi, psi, 1, np.array([np.nan, 1j]), 2, out, out)
    s.close()
    op = fe_like(7, seed=2)
    sp_ = sparse_problem(op.n)
    c = Solver(sp_, csr=csr_arrays(op.K, op.M))
    z = np.zeros((1, op.n), np.complex128)
    with pytest.raises(fks.FksError):
        fks.fks_sensitivity(c.op, z, z[None], 1, np.array([1j]), 1, z[None], z[None])
    c.close()
