"""fks_precond_apply_noalloc, the allocation-free inner preconditioner apply.

It serves callers that may not allocate device memory (a host framework whose
pool owns the GPU's memory, real-time code that cannot take cudaMalloc's
implicit synchronisation): its scratch is a fixed array inside the library.
It must give what fks_precond_apply gives, call after call, although every
call reuses the same array. This file is collected last so that a run that
stops at the first failure has run every other test before it.
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
