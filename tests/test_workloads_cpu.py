"""Host-side pieces of the benchmark workloads and the request binding (no
GPU): the mixed 2D batch generator and the caller-owned output array of a
server request."""
import numpy as np
import pytest

from paper_1212_3660_gb300 import fks, synth


def test_mixed_2d_batch_is_seeded_and_within_its_sides():
    a, b = synth.mix2d_grids(), synth.mix2d_grids()
    assert a == b and len(a) == 32
    sides = [g["shape"][0] for g in a]
    assert all(g["shape"] == (s, s) for g, s in zip(a, sides))
    assert set(sides) <= set(range(128, 385, 32)) and len(set(sides)) > 3
    assert len({g["seed"] for g in a}) == 32             # every aquifer its own field
    assert all(g["n_f"] == 100 and g["n_p"] == 4 and g["periods"] == (5.0, 3600.0) for g in a)
    assert synth.mix2d_grids(seed=1) != a
    p = synth.make_problem(m_max=100, **a[0])
    assert p.n == sides[0] ** 2 and len(p.sigma) == 100 and len(p.tau_bar) == 4
    assert list(p.src_cells) == [synth.center_cell(p.shape)]


def _request(out=None, with_x=True, n=12, n_f=3, n_rhs=2):
    opts, keep = fks.make_options(tol=1e-8, m_max=10)
    b = np.ones((n_rhs, n), np.complex128)
    sig = 1j * np.arange(1, n_f + 1, dtype=np.float64)
    return fks.ServerRequest(None, b, sig, np.array([1j]), opts, keep, n, with_x=with_x, out=out)


def test_request_output_array_is_the_callers():
    out = np.full((2, 3, 12), 7 + 1j)
    r = _request(out=out)
    assert r.X is out and r.c.X == out.ctypes.data
    r = _request(out=np.zeros((2, 3, 12), np.complex128), with_x=False)   # out implies X delivered
    assert r.X is not None and r.c.X == r.X.ctypes.data
    r = _request(with_x=False)
    assert r.X is None and not r.c.X
    r = _request()
    assert r.X.shape == (2, 3, 12) and r.c.X == r.X.ctypes.data


@pytest.mark.parametrize("bad", [np.zeros((2, 3, 11), np.complex128), np.zeros((2, 3, 12), np.complex64),
                                 np.zeros((2, 12, 3), np.complex128).transpose(0, 2, 1)])
def test_request_output_array_is_checked(bad):
    with pytest.raises(ValueError):
        _request(out=bad)
    ro = np.zeros((2, 3, 12), np.complex128)
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        _request(out=ro)
