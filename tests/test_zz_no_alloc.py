"""fks_precond_apply_noalloc, the allocation-free inner preconditioner apply.

It serves callers that may not allocate device memory (a host framework whose
pool owns the GPU's memory, real-time code that cannot take cudaMalloc's
implicit synchronisation): its scratch is a fixed array inside the library.
It must give what fks_precond_apply gives, call after call, although every
call reuses the same array, and it must leave the device's free memory as it
found it. This file is collected last so that a run that stops at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1212_3660_gb300 import fks, synth
from paper_1212_3660_gb300.solver import Solver

from gpu_util import need_gpu, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_noalloc_matches_precond_apply_on_two_calls(precision):
    need_gpu()
    import torch
    pr = synth.make_problem((64, 64), n_f=2, periods=(5.0, 3600.0), n_p=2, seed=31)
    s = Solver(pr)
    rng = np.random.default_rng(41)
    for call, (tau, eps, cycles) in enumerate([(pr.tau_bar[0], 1e-10, -1), (pr.tau_bar[1], 1e-6, 3)]):
        v = rng.standard_normal(pr.n) + 1j * rng.standard_normal(pr.n)
        v /= np.linalg.norm(v)
        v_d = torch.from_numpy(v).cuda()
        z_ref = torch.zeros_like(v_d)
        z_na = torch.full_like(v_d, complex(7.0, -3.0))       # stale contents must not matter
        _, c_ref, p_ref = fks.fks_precond_apply(s.op, tau, v_d, z_ref, eps, cycles=cycles, precision=precision)
        _, c_na, p_na = fks.fks_precond_apply_noalloc(s.op, tau, v_d, z_na, eps, cycles=cycles, precision=precision)
        torch.cuda.synchronize()
        assert c_na == c_ref, call
        assert rel_err(z_na.cpu().numpy(), z_ref.cpu().numpy()) <= 1e-12, call
        assert abs(p_na - p_ref) <= 1e-9 * p_ref + 1e-15, call
    s.close()


@pytest.mark.parametrize("precision", [fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED])
def test_noalloc_in_place_and_zero_cycles(precision):
    """z may be v itself (v is copied into the fixed array first); a replayed
    count of zero cycles returns z = 0, as fks_precond_apply does."""
    need_gpu()
    import torch
    pr = synth.make_problem((64, 64), n_f=2, periods=(5.0, 3600.0), n_p=1, seed=33)
    s = Solver(pr)
    rng = np.random.default_rng(43)
    v = rng.standard_normal(pr.n) + 1j * rng.standard_normal(pr.n)
    v_d = torch.from_numpy(v).cuda()
    z_ref = torch.zeros_like(v_d)
    fks.fks_precond_apply(s.op, pr.tau_bar[0], v_d, z_ref, 1e-10, precision=precision)
    w_d = v_d.clone()
    fks.fks_precond_apply_noalloc(s.op, pr.tau_bar[0], w_d, w_d, 1e-10, precision=precision)
    torch.cuda.synchronize()
    assert rel_err(w_d.cpu().numpy(), z_ref.cpu().numpy()) <= 1e-12
    for apply in (fks.fks_precond_apply, fks.fks_precond_apply_noalloc):
        z = torch.full_like(v_d, complex(7.0, -3.0))
        _, c, _ = apply(s.op, pr.tau_bar[0], v_d, z, 1e-10, cycles=0, precision=precision)
        torch.cuda.synchronize()
        assert c == 0 and float(z.abs().max()) == 0.0, apply.__name__
    s.close()


def test_noalloc_leaves_free_device_memory_unchanged():
    """On a fresh operator, before any allocating call on it: after one warm-up
    call (which may load kernel code), a further call changes the device's free
    memory by nothing."""
    need_gpu()
    import torch
    pr = synth.make_problem((128, 128), n_f=2, periods=(5.0, 3600.0), n_p=1, seed=35)
    s = Solver(pr)
    rng = np.random.default_rng(45)
    v_d = torch.from_numpy(rng.standard_normal(pr.n) + 1j * rng.standard_normal(pr.n)).cuda()
    z_d = torch.zeros_like(v_d)
    for precision in (fks.FKS_PREC_FP64, fks.FKS_PREC_MIXED):
        fks.fks_precond_apply_noalloc(s.op, pr.tau_bar[0], v_d, z_d, 1e-8, precision=precision)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        fks.fks_precond_apply_noalloc(s.op, pr.tau_bar[0], v_d, z_d, 1e-8, precision=precision)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (precision, free0 - free1)
    s.close()


def test_noalloc_rejects_grids_beyond_its_limit():
    need_gpu()
    import torch
    pr = synth.make_problem((512, 512), n_f=2, periods=(5.0, 3600.0), n_p=1, seed=31)
    s = Solver(pr)
    v = torch.zeros(pr.n, dtype=torch.complex128, device="cuda")
    z = torch.zeros_like(v)
    with pytest.raises(fks.FksError) as e:
        fks.fks_precond_apply_noalloc(s.op, pr.tau_bar[0], v, z, 1e-8)
    assert e.value.status == fks.FKS_ERR_ARG and "65536" in str(e.value)
    s.close()
