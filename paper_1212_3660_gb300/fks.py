"""ctypes binding of libfks.so (argument marshalling only).

Every function here has the name of the C entry point it wraps and does no
arithmetic of the method: arrays are passed by pointer (numpy arrays on the
host, torch tensors on the host or the GPU), results come back in the
caller's arrays. The library must have been built (paper_1212_3660_gb300.build);
loading fails loudly otherwise.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfks.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fks.h")

FKS_OK, FKS_NOT_CONVERGED, FKS_BREAKDOWN_EXACT, FKS_INNER_NOT_CONVERGED = 0, 1, 2, 3
FKS_ERR_ARG, FKS_ERR_OOM, FKS_ERR_CUDA, FKS_ERR_TIMEOUT, FKS_ERR_CANCELLED = -1, -2, -3, -4, -5
FKS_FGMRES, FKS_FFOM = 0, 1
FKS_PREC_FP64, FKS_PREC_MIXED, FKS_PREC_MIXED_BF16 = 0, 1, 2
KERNEL_CLASSES = ["smooth", "restrict", "prolong", "coarse", "defect", "correct", "mdot", "maxpy", "givens",
                  "assemble", "tres", "tail", "pre2d", "post2d", "bicgstab", "cluster", "pre3d", "post3d", "coop"]


class fks_c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class fks_options(C.Structure):
    _fields_ = [("tol", C.c_double), ("m_max", C.c_int), ("variant", C.c_int), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("inner_max_cycles", C.c_int),
                ("tau_schedule", C.POINTER(C.c_int32)), ("sched_len", C.c_int),
                ("replay_mode", C.c_int), ("replay_inner_cycles", C.POINTER(C.c_int32)),
                ("replay_mj", C.POINTER(C.c_int32)), ("launch_mode", C.c_int),
                ("inner_steps", C.c_int), ("assembly", C.c_int), ("inner_relax", C.c_double),
                ("restart_len", C.c_int), ("max_restarts", C.c_int)]


class fks_info(C.Structure):
    _fields_ = [("steps", C.POINTER(C.c_int32)), ("inner_cycles", C.POINTER(C.c_int32)),
                ("pnorm", C.POINTER(C.c_double)), ("breakdown", C.POINTER(C.c_int32)),
                ("gmres_alpha", C.c_void_p), ("hbar", C.c_void_p), ("tau_k", C.c_void_p)]


class fks_request(C.Structure):
    _fields_ = [("op", C.c_void_p), ("b", C.c_void_p), ("n_rhs", C.c_int), ("sigma", C.c_void_p), ("n_f", C.c_int),
                ("tau", C.c_void_p), ("n_tau", C.c_int), ("opt", fks_options), ("X", C.c_void_p),
                ("res_est", C.c_void_p), ("res_bound", C.c_void_p), ("res_true", C.c_void_p), ("m_j", C.c_void_p),
                ("shift_status", C.c_void_p), ("timeout_s", C.c_double)]


class FksError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fks status {status}: {msg}")
        self.status = status


_lib = None


def declared_symbols() -> list[str]:
    """Names of the functions declared in include/fks.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fks_[a-z0-9_]+)\s*\(", txt)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1212_3660_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32p, f64p = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_double)
    L.fks_last_error.restype = C.c_char_p
    L.fks_version.restype = C.c_char_p
    L.fks_create.argtypes = [C.POINTER(vp), C.c_int]
    L.fks_destroy.argtypes = [vp]
    L.fks_destroy.restype = None
    L.fks_op_grid.argtypes = [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double), vp, vp, C.c_uint32,
                              C.POINTER(vp)]
    L.fks_op_csr.argtypes = [vp, C.c_int64, vp, vp, vp, vp, vp, vp, C.POINTER(vp)]
    L.fks_op_destroy.argtypes = [vp]
    L.fks_op_amg.argtypes = [vp, C.c_int, C.c_int, C.c_int64, C.c_int]
    L.fks_op_amg_setup.argtypes = [vp, vp, C.c_int, C.c_int, f64p]
    L.fks_op_amg_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.c_int, vp, C.c_int64]
    L.fks_amg_host_shape.argtypes = [C.c_int64, vp, vp, vp, C.c_int, C.c_int64, C.POINTER(C.c_int), vp, vp, vp, vp,
                                     C.c_int, vp, C.c_int64]
    L.fks_op_destroy.restype = None
    L.fks_op_size.argtypes = [vp]
    L.fks_op_size.restype = C.c_int64
    L.fks_solve.argtypes = [vp, vp, C.c_int, vp, C.c_int, vp, C.c_int, C.POINTER(fks_options), vp, vp, vp, vp, vp,
                            vp, C.POINTER(fks_info), vp]
    L.fks_op_apply.argtypes = [vp, fks_c128, vp, vp, C.c_int, vp]
    L.fks_sensitivity.argtypes = [vp, vp, vp, C.c_int, vp, C.c_int, vp, vp, vp]
    L.fks_ritz.argtypes = [vp, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp]
    L.fks_precond_apply.argtypes = [vp, fks_c128, vp, vp, C.c_double, C.c_int, C.c_int, C.c_int, i32p, f64p, vp]
    L.fks_precond_apply_noalloc.argtypes = [vp, fks_c128, vp, vp, C.c_double, C.c_int, C.c_int, C.c_int, i32p,
                                            f64p, vp]
    L.fks_op_autotune.argtypes = [vp, C.c_int, fks_c128, vp, C.POINTER(C.c_int64)]
    L.fks_op_set_fusion.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_set_tiles.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_set_tail.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_set_cluster.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_set_tiles8.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_tiling.argtypes = [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.fks_op_set_zchunk.argtypes = [vp, C.c_int, C.c_int, C.c_int]
    L.fks_set_pdl.argtypes = [C.c_int]
    L.fks_op_set_coop.argtypes = [vp, C.c_int, C.c_int64]
    L.fks_op_coop_max.argtypes = [vp, C.c_int, C.POINTER(C.c_int64)]
    L.fks_set_pdl.restype = C.c_int
    L.fks_op_zchunks.argtypes = [vp, C.c_int, C.POINTER(C.c_int32), C.c_int, C.POINTER(C.c_int)]
    L.fks_server_create.argtypes = [vp, C.c_size_t, C.c_int, C.POINTER(vp)]
    L.fks_server_submit.argtypes = [vp, C.POINTER(fks_request), C.POINTER(C.c_uint64)]
    L.fks_server_poll.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fks_server_wait.argtypes = [vp, C.c_uint64, C.POINTER(C.c_int)]
    L.fks_server_cancel.argtypes = [vp, C.c_uint64]
    L.fks_server_times.argtypes = [vp, C.c_uint64, f64p, f64p, f64p]
    L.fks_server_launches.argtypes = [vp, C.POINTER(C.c_int64)]
    L.fks_server_destroy.argtypes = [vp]
    L.fks_server_destroy.restype = None
    L.fks_debug_fail_allocs.argtypes = [C.c_int]
    L.fks_debug_fail_allocs.restype = None
    L.fks_profile_select.argtypes = [vp, C.c_int, C.c_int]
    L.fks_profile_read.argtypes = [vp, C.POINTER(C.c_int64), f64p, f64p, f64p, C.POINTER(C.c_int64)]
    for name in ("fks_create", "fks_op_grid", "fks_op_csr", "fks_op_amg", "fks_op_amg_setup", "fks_op_amg_info", "fks_amg_host_shape", "fks_solve", "fks_op_apply", "fks_sensitivity", "fks_ritz", "fks_precond_apply", "fks_profile_select",
                 "fks_profile_read", "fks_precond_apply_noalloc", "fks_op_autotune",
                 "fks_op_set_fusion", "fks_op_set_tiles", "fks_op_set_tail", "fks_op_set_cluster", "fks_op_set_tiles8", "fks_op_tiling",
                 "fks_op_set_zchunk", "fks_op_zchunks", "fks_op_set_coop", "fks_op_coop_max",
                 "fks_server_create",
                 "fks_server_submit", "fks_server_poll", "fks_server_wait",
                 "fks_server_cancel", "fks_server_times", "fks_server_launches"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(type(a))


def fks_last_error() -> str:
    return lib().fks_last_error().decode()


def fks_version() -> str:
    return lib().fks_version().decode()


def fks_create(device: int = 0):
    h = C.c_void_p()
    st = lib().fks_create(C.byref(h), device)
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return h


def fks_destroy(ctx) -> None:
    lib().fks_destroy(ctx)


def fks_op_grid(ctx, dim, ncell, h, cond, ss, dirichlet_mask):
    """cond, ss: host float64 arrays of n cells (x fastest)."""
    nc = (C.c_int64 * 3)(*[int(v) for v in (list(ncell) + [1, 1, 1])[:3]])
    hh = (C.c_double * 3)(*[float(v) for v in (list(h) + [1.0, 1.0, 1.0])[:3]])
    cond = np.ascontiguousarray(cond, dtype=np.float64).ravel()
    ss = np.ascontiguousarray(ss, dtype=np.float64).ravel()
    out = C.c_void_p()
    st = lib().fks_op_grid(ctx, int(dim), nc, hh, _ptr(cond), _ptr(ss), int(dirichlet_mask), C.byref(out))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return out


def fks_op_csr(ctx, n, k_rowptr, k_col, k_val, m_rowptr, m_col, m_val):
    """K and M as CSR arrays (row pointers int64, columns int32, values float64), host memory."""
    a = [np.ascontiguousarray(k_rowptr, dtype=np.int64), np.ascontiguousarray(k_col, dtype=np.int32),
         np.ascontiguousarray(k_val, dtype=np.float64), np.ascontiguousarray(m_rowptr, dtype=np.int64),
         np.ascontiguousarray(m_col, dtype=np.int32), np.ascontiguousarray(m_val, dtype=np.float64)]
    out = C.c_void_p()
    st = lib().fks_op_csr(ctx, int(n), *[_ptr(x) for x in a], C.byref(out))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return out


def fks_op_amg(op, enable=True, max_levels=0, max_coarse=0, nu=0):
    """Smoothed-aggregation AMG as the BiCGSTAB preconditioner of a CSR operator (0 = default)."""
    st = lib().fks_op_amg(op, int(bool(enable)), int(max_levels), int(max_coarse), int(nu))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_amg_setup(op, taus, precision=FKS_PREC_FP64) -> float:
    """Builds the hierarchies of K + tau M for the taus; returns the host time in ms."""
    t = np.ascontiguousarray(np.asarray(taus, dtype=np.complex128).ravel())
    ms = C.c_double(0.0)
    st = lib().fks_op_amg_setup(op, _ptr(t), len(t), int(precision), C.byref(ms))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return float(ms.value)


def fks_op_amg_info(op):
    """(level sizes, [aggregates of each level but the coarsest]) of the built hierarchy."""
    nl = C.c_int(0)
    st = lib().fks_op_amg_info(op, C.byref(nl), None, 0, None, 0)
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    sizes = np.zeros(nl.value, np.int64)
    nagg = 0
    st = lib().fks_op_amg_info(op, C.byref(nl), sizes.ctypes.data_as(C.POINTER(C.c_int64)), nl.value, None, 0)
    if st == FKS_OK:
        nagg = int(sizes[:-1].sum())
        agg = np.zeros(max(nagg, 1), np.int32)
        st = lib().fks_op_amg_info(op, C.byref(nl), sizes.ctypes.data_as(C.POINTER(C.c_int64)), nl.value,
                                   _ptr(agg), nagg)
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    out, at = [], 0
    for l in range(len(sizes) - 1):
        out.append(agg[at:at + sizes[l]].copy())
        at += sizes[l]
    return sizes, out


def fks_amg_host_shape(A0, max_levels=0, max_coarse=0):
    """Host-only AMG hierarchy of a complex scipy CSR matrix A0 (sorted columns; no GPU needed):
    dict(sizes, nnz_a, nnz_p, omega, agg=[aggregates of each level but the coarsest])."""
    rp = np.ascontiguousarray(A0.indptr, dtype=np.int64)
    ci = np.ascontiguousarray(A0.indices, dtype=np.int32)
    va = np.ascontiguousarray(A0.data, dtype=np.complex128)
    nl = C.c_int(0)
    cap = 16
    sizes, nnz_a, nnz_p = (np.zeros(cap, np.int64) for _ in range(3))
    om = np.zeros(cap)
    n = A0.shape[0]
    agg = np.zeros(n * 2, np.int32)
    st = lib().fks_amg_host_shape(int(n), _ptr(rp), _ptr(ci), _ptr(va), int(max_levels), int(max_coarse),
                                  C.byref(nl), _ptr(sizes), _ptr(nnz_a), _ptr(nnz_p), _ptr(om), cap, _ptr(agg),
                                  len(agg))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    L = nl.value
    out, at = [], 0
    for l in range(L - 1):
        out.append(agg[at:at + sizes[l]].copy())
        at += int(sizes[l])
    return dict(sizes=sizes[:L].copy(), nnz_a=nnz_a[:L].copy(), nnz_p=nnz_p[:L].copy(), omega=om[:L].copy(), agg=out)


def fks_op_destroy(op) -> None:
    lib().fks_op_destroy(op)


def fks_op_size(op) -> int:
    return int(lib().fks_op_size(op))


def make_options(tol=1e-8, m_max=100, variant=FKS_FGMRES, precision=FKS_PREC_FP64, inner_tol=0.0,
                 inner_max_cycles=50, schedule=(0,), replay_cycles=None, replay_mj=None, launch_mode=0,
                 inner_steps=0, assembly=0, inner_relax=0.0, restart_len=0, max_restarts=0):
    """fks_options plus the arrays it points to (kept alive in the returned tuple)."""
    sched = np.ascontiguousarray(schedule, dtype=np.int32)
    o = fks_options()
    o.tol, o.m_max, o.variant, o.precision = float(tol), int(m_max), int(variant), int(precision)
    o.inner_tol, o.inner_max_cycles = float(inner_tol), int(inner_max_cycles)
    o.tau_schedule = sched.ctypes.data_as(C.POINTER(C.c_int32))
    o.sched_len = len(sched)
    o.launch_mode = int(launch_mode)
    o.inner_steps = int(inner_steps)
    o.assembly = int(assembly)
    o.inner_relax = float(inner_relax)
    o.restart_len = int(restart_len)
    o.max_restarts = int(max_restarts)
    keep = [sched]
    if replay_cycles is not None:
        rc = np.ascontiguousarray(replay_cycles, dtype=np.int32)
        rm = np.ascontiguousarray(replay_mj, dtype=np.int32)
        o.replay_mode = 1
        o.replay_inner_cycles = rc.ctypes.data_as(C.POINTER(C.c_int32))
        o.replay_mj = rm.ctypes.data_as(C.POINTER(C.c_int32))
        keep += [rc, rm]
    return o, keep


def fks_solve(op, b, n_rhs, sigma, n_f, tau, n_tau, options, X, res_est, res_bound, res_true, m_j, shift_status,
              info=None, stream=None):
    """Thin wrapper: every array argument is a numpy array or torch tensor; returns the status."""
    st = lib().fks_solve(op, _ptr(b), int(n_rhs), _ptr(sigma), int(n_f), _ptr(tau), int(n_tau), C.byref(options),
                         _ptr(X), _ptr(res_est), _ptr(res_bound), _ptr(res_true), _ptr(m_j), _ptr(shift_status),
                         C.byref(info) if info is not None else None, stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st


def fks_op_apply(op, s, x, y, n_vec, stream=None):
    st = lib().fks_op_apply(op, fks_c128(complex(s).real, complex(s).imag), _ptr(x), _ptr(y), int(n_vec), stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st


def fks_sensitivity(op, phi, psi, n_m, sigma, n_f, j_lnk, j_lns, stream=None):
    """dh/dlnK and dh/dlnS of every measurement, shift and cell (arrays as numpy or torch)."""
    st = lib().fks_sensitivity(op, _ptr(phi), _ptr(psi), int(n_m), _ptr(sigma), int(n_f), _ptr(j_lnk), _ptr(j_lns),
                               stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st


def fks_ritz(ctx, hbar, tau_k, steps, n_rhs, m_max, theta, status, stream=None):
    """Prop. 1's Ritz values at sigma = 0 of every source (arrays as numpy or torch)."""
    st = lib().fks_ritz(ctx, _ptr(hbar), _ptr(tau_k), _ptr(steps), int(n_rhs), int(m_max), _ptr(theta), _ptr(status),
                        stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st


def fks_precond_apply(op, tau, v, z, eps, max_cycles=50, cycles=-1, precision=FKS_PREC_FP64, stream=None):
    """Returns (status, cycles, ||p||)."""
    oc = C.c_int32(0)
    op_ = C.c_double(0.0)
    st = lib().fks_precond_apply(op, fks_c128(complex(tau).real, complex(tau).imag), _ptr(v), _ptr(z), float(eps),
                                 int(max_cycles), int(cycles), int(precision), C.byref(oc), C.byref(op_), stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st, int(oc.value), float(op_.value)


def fks_precond_apply_noalloc(op, tau, v, z, eps, max_cycles=50, cycles=-1, precision=FKS_PREC_FP64, stream=None):
    """Allocation-free fks_precond_apply (device v, z; fixed scratch in the library). Returns (status, cycles, ||p||)."""
    oc = C.c_int32(0)
    op_ = C.c_double(0.0)
    st = lib().fks_precond_apply_noalloc(op, fks_c128(complex(tau).real, complex(tau).imag), _ptr(v), _ptr(z),
                                         float(eps), int(max_cycles), int(cycles), int(precision), C.byref(oc),
                                         C.byref(op_), stream)
    if st < 0:
        raise FksError(st, fks_last_error())
    return st, int(oc.value), float(op_.value)


def make_info(n_rhs, m_max, n_f=0):
    """fks_info with host arrays; with n_f > 0 also the monitors (Prop. 3's alpha
    per shift, the Hessenberg matrices and the steps' tau)."""
    arrs = dict(steps=np.zeros(n_rhs, np.int32), inner_cycles=np.zeros(n_rhs * m_max, np.int32),
                pnorm=np.zeros(n_rhs * m_max, np.float64), breakdown=np.zeros(n_rhs, np.int32))
    if n_f > 0:
        arrs.update(gmres_alpha=np.zeros((n_rhs, n_f)), hbar=np.zeros((n_rhs, m_max, m_max + 1), np.complex128),
                    tau_k=np.zeros((n_rhs, m_max), np.complex128))
    info = fks_info(arrs["steps"].ctypes.data_as(C.POINTER(C.c_int32)),
                    arrs["inner_cycles"].ctypes.data_as(C.POINTER(C.c_int32)),
                    arrs["pnorm"].ctypes.data_as(C.POINTER(C.c_double)),
                    arrs["breakdown"].ctypes.data_as(C.POINTER(C.c_int32)),
                    *([arrs[k].ctypes.data for k in ("gmres_alpha", "hbar", "tau_k")] if n_f > 0 else [None] * 3))
    info._arrays = arrs   # the struct holds raw pointers into these: they live as long as it does
    return info, arrs


def fks_op_set_tiles(op, precision, max_cells):
    st = lib().fks_op_set_tiles(op, int(precision), int(max_cells))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_set_tail(op, precision, max_cells):
    st = lib().fks_op_set_tail(op, int(precision), int(max_cells))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_set_cluster(op, precision, max_cells):
    st = lib().fks_op_set_cluster(op, int(precision), int(max_cells))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_set_tiles8(op, precision, max_cells):
    st = lib().fks_op_set_tiles8(op, int(precision), int(max_cells))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_set_coop(op, precision, max_cells):
    """Cooperative lower cycle from the first level of at most max_cells cells (0: off)."""
    st = lib().fks_op_set_coop(op, int(precision), int(max_cells))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_coop_max(op, precision):
    v = C.c_int64(0)
    st = lib().fks_op_coop_max(op, int(precision), C.byref(v))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return int(v.value)


def fks_set_pdl(on):
    """Programmatic dependent launch of the multigrid and defect kernels for the
    process (1 on, 0 off, -1 query); returns the previous setting."""
    return int(lib().fks_set_pdl(int(on)))


def fks_op_set_zchunk(op, precision, level, planes):
    """Planes per block of the fused 3D kernels on multigrid level `level` (<= 0: all)."""
    st = lib().fks_op_set_zchunk(op, int(precision), int(level), int(planes))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_op_zchunks(op, precision):
    """The z-chunk of every multigrid level (list of planes per block)."""
    buf = (C.c_int32 * 16)()
    nl = C.c_int(0)
    st = lib().fks_op_zchunks(op, int(precision), buf, 16, C.byref(nl))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return [int(buf[i]) for i in range(nl.value)]


def fks_op_tiling(op, precision):
    """(fusion threshold, 16 x 16 tile threshold, tail threshold, cluster
    threshold, 8 x 8 tile threshold) in cells; the cluster threshold is 0 when
    the cluster kernel is off."""
    a, b, t, c, e = (C.c_int64(0) for _ in range(5))
    st = lib().fks_op_tiling(op, int(precision), C.byref(a), C.byref(b), C.byref(t), C.byref(c), C.byref(e))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return int(a.value), int(b.value), int(t.value), int(c.value), int(e.value)


def fks_op_autotune(op, precision, tau, stream=None):
    """Pick the fused-level threshold for `precision` by timing V-cycles; returns it."""
    ch = C.c_int64(0)
    st = lib().fks_op_autotune(op, int(precision), fks_c128(complex(tau).real, complex(tau).imag), stream,
                               C.byref(ch))
    if st < 0:
        raise FksError(st, fks_last_error())
    return int(ch.value)


def fks_op_set_fusion(op, precision, max_cells):
    st = lib().fks_op_set_fusion(op, int(precision), int(max_cells))
    if st < 0:
        raise FksError(st, fks_last_error())


def fks_profile_select(op, kclass, level=-1):
    """kclass: index or name in KERNEL_CLASSES (None / -1 stops timing)."""
    if isinstance(kclass, str):
        kclass = KERNEL_CLASSES.index(kclass)
    st = lib().fks_profile_select(op, -1 if kclass is None else int(kclass), int(level))
    if st < 0:
        raise FksError(st, fks_last_error())


def fks_profile_read(op):
    """Returns dict(launches, ms, bytes, flops, all_launches) and resets the counters."""
    la, al = C.c_int64(0), C.c_int64(0)
    ms, by, fl = C.c_double(0), C.c_double(0), C.c_double(0)
    st = lib().fks_profile_read(op, C.byref(la), C.byref(ms), C.byref(by), C.byref(fl), C.byref(al))
    if st < 0:
        raise FksError(st, fks_last_error())
    return dict(launches=la.value, ms=ms.value, bytes=by.value, flops=fl.value, all_launches=al.value)


# ---------------------------------------------------------------- serving
# servers not yet destroyed: stopped at interpreter exit, so that the server's
# driver thread never outlives the process's CUDA state
_live_servers = {}


def _destroy_live_servers():
    for key in list(_live_servers):
        lib().fks_server_destroy(_live_servers.pop(key))


atexit.register(_destroy_live_servers)


def fks_server_create(ctx, mem_budget_bytes, lanes=2):
    out = C.c_void_p()
    st = lib().fks_server_create(ctx, int(mem_budget_bytes), int(lanes), C.byref(out))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    _live_servers[out.value] = out
    return out


def fks_server_destroy(srv):
    if _live_servers.pop(srv.value, None) is not None:
        lib().fks_server_destroy(srv)


class ServerRequest:
    """A request and the host arrays it points to (kept alive until done).
    with_x=False submits X = NULL (residuals and statuses only); `out`, if
    given, is the caller's array for X (complex128, C-contiguous, n_rhs x n_f x
    n; for instance a view of page-locked memory reused across requests);
    timeout_s > 0 stops the request with FKS_ERR_TIMEOUT once it has run that
    long."""

    def __init__(self, op, b, sigma, tau, options, keep, n, with_x=True, timeout_s=0.0, out=None):
        b = np.ascontiguousarray(b, dtype=np.complex128)
        self.n_rhs = b.shape[0] if b.ndim == 2 else 1
        self.b = b.reshape(self.n_rhs, n)
        self.sigma = np.ascontiguousarray(sigma, dtype=np.complex128)
        self.tau = np.ascontiguousarray(tau, dtype=np.complex128)
        n_f = len(self.sigma)
        if out is not None:
            if (out.dtype != np.complex128 or out.shape != (self.n_rhs, n_f, n)
                    or not out.flags["C_CONTIGUOUS"] or not out.flags["WRITEABLE"]):
                raise ValueError(f"out: a writeable C-contiguous complex128 array of shape {(self.n_rhs, n_f, n)} "
                                 f"expected, got {out.dtype} {out.shape}")
            with_x = True
        self.X = (out if out is not None else np.zeros((self.n_rhs, n_f, n), np.complex128)) if with_x else None
        self.res_est = np.zeros((self.n_rhs, n_f))
        self.res_bound = np.zeros((self.n_rhs, n_f))
        self.res_true = np.zeros((self.n_rhs, n_f))
        self.m_j = np.zeros((self.n_rhs, n_f), np.int32)
        self.shift_status = np.zeros((self.n_rhs, n_f), np.int32)
        self.keep = keep
        self.c = fks_request(op.value if hasattr(op, "value") else op, self.b.ctypes.data, self.n_rhs,
                             self.sigma.ctypes.data, n_f, self.tau.ctypes.data, len(self.tau), options,
                             self.X.ctypes.data if with_x else None, self.res_est.ctypes.data,
                             self.res_bound.ctypes.data, self.res_true.ctypes.data, self.m_j.ctypes.data,
                             self.shift_status.ctypes.data, float(timeout_s))
        self.ticket = None


def fks_server_submit(srv, req: ServerRequest):
    t = C.c_uint64(0)
    st = lib().fks_server_submit(srv, C.byref(req.c), C.byref(t))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    req.ticket = t.value
    return t.value


def fks_server_poll(srv, ticket):
    d, r = C.c_int(0), C.c_int(0)
    st = lib().fks_server_poll(srv, C.c_uint64(ticket), C.byref(d), C.byref(r))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return bool(d.value), r.value


def fks_server_wait(srv, ticket):
    r = C.c_int(0)
    st = lib().fks_server_wait(srv, C.c_uint64(ticket), C.byref(r))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return r.value


def fks_debug_fail_allocs(count):
    """Test hook: the next `count` workspace reservations fail as out of memory."""
    lib().fks_debug_fail_allocs(int(count))


def fks_server_cancel(srv, ticket):
    st = lib().fks_server_cancel(srv, C.c_uint64(ticket))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())


def fks_server_launches(srv):
    n = C.c_int64(0)
    st = lib().fks_server_launches(srv, C.byref(n))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return int(n.value)


def fks_server_times(srv, ticket):
    a, b, c = C.c_double(0), C.c_double(0), C.c_double(0)
    st = lib().fks_server_times(srv, C.c_uint64(ticket), C.byref(a), C.byref(b), C.byref(c))
    if st != FKS_OK:
        raise FksError(st, fks_last_error())
    return a.value, b.value, c.value
