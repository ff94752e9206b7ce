"""GB300 first-order bilevel topology optimiser (arXiv 2204.06204): Python binding.

The functions below carry the names of the C ABI in ``include/to.h`` and only
marshal arguments: torch tensors become device pointers, the current torch
stream becomes the ``stream`` argument, and non-zero status codes become
``ToError``.  All computation runs in the CUDA library; if it has not been
built, importing the binding's entry points raises (there is no fallback).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _abi
from ._abi import (TO_FP32_MIXED, TO_FP64, TO_INNER_PCG, TO_INNER_PFBTO, TO_INNER_RICHARDSON, TO_INNER_SD,
                   TO_PRECOND_JACOBI,
                   TO_PRECOND_KRYLOV,
                   TO_PRECOND_MG, TO_PRECOND_NONE, ToError, to_stats)

__all__ = ["to_default_params", "to_create", "to_destroy", "to_sizes", "to_set_design", "to_apply_K",
           "to_residual", "to_smooth",
           "to_inner_solve", "to_sensitivity", "to_filter", "to_project", "to_step", "to_step_host", "to_get_stats", "to_get_state",
           "to_set_state", "to_check", "to_barrier_selftest", "to_last_error", "to_project_noalloc", "to_compliance_truncated",
           "to_compliance_truncated_grad", "to_compliance_truncated_id", "to_batch_create", "to_batch_destroy", "to_batch_step", "to_batch_tile", "Batch",
           "Problem", "ToError",
           "TO_FP64", "TO_FP32_MIXED", "TO_PRECOND_JACOBI", "TO_PRECOND_MG", "TO_PRECOND_NONE", "TO_PRECOND_KRYLOV",
           "TO_INNER_SD", "TO_INNER_RICHARDSON", "TO_INNER_PFBTO", "TO_INNER_PCG"]


def _lib():
    return _abi.load()


def _stream(device):
    import torch
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t, dtype, n, name):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} entries, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def to_default_params(**overrides) -> _abi.to_params:
    p = _abi.to_params()
    _lib().to_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def to_create(nx, ny, nz, h, material: dict, load_dof, load_val, fixed_dof, params=None, device=0):
    g = _abi.to_grid(nx, ny, nz, h)
    m = _abi.to_material(**{k: float(material[k]) for k in
                            ("E0", "Emin", "nu", "p", "volfrac", "rmin", "rho_min", "rho_max")})
    ld = np.ascontiguousarray(load_dof, dtype=np.int64)
    lv = np.ascontiguousarray(load_val, dtype=np.float64)
    fd = np.ascontiguousarray(fixed_dof, dtype=np.int64)
    loads = _abi.to_loads(ld.size, ld.ctypes.data_as(C.POINTER(C.c_int64)), lv.ctypes.data_as(C.POINTER(C.c_double)))
    bcs = _abi.to_bcs(fd.size, fd.ctypes.data_as(C.POINTER(C.c_int64)))
    prm = params if params is not None else to_default_params()
    out = C.c_void_p()
    _abi.check(_lib().to_create(C.byref(g), C.byref(m), C.byref(loads), C.byref(bcs), C.byref(prm), int(device),
                                C.byref(out)))
    return out


def to_destroy(P):
    _lib().to_destroy(P)


def to_sizes(P):
    ne, nd = C.c_int64(), C.c_int64()
    _abi.check(_lib().to_sizes(P, C.byref(ne), C.byref(nd)))
    return ne.value, nd.value


class Problem:
    """Owns one ``to_problem``; every method is one C call."""

    def __init__(self, nx, ny, nz, material, load_dof, load_val, fixed_dof, params=None, h=1.0, device=0):
        import torch
        self.params = params if params is not None else to_default_params()
        self.device = torch.device("cuda", device)
        self.dtype = torch.float64 if self.params.precision == TO_FP64 else torch.float32
        self.handle = to_create(nx, ny, nz, h, material, load_dof, load_val, fixed_dof, self.params, device)
        self.n_elem, self.n_dof = to_sizes(self.handle)
        self.grid = (nx, ny, nz)

    @classmethod
    def from_workload(cls, pb, params=None, device=0):
        """Build from a ``workloads.Problem``-like object (attributes nx, ny, nz, h, material, loads, fixtures)."""
        mat = dict(E0=pb.E0, Emin=pb.Emin, nu=pb.nu, p=pb.p, volfrac=pb.volfrac, rmin=pb.rmin,
                   rho_min=pb.rho_min, rho_max=pb.rho_max)
        return cls(pb.nx, pb.ny, pb.nz, mat, pb.load_dof, pb.load_val, pb.fixed_dof, params, pb.h, device)

    def close(self):
        if getattr(self, "handle", None):
            to_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- vectors
    def elem(self):
        import torch
        return torch.empty(self.n_elem, dtype=self.dtype, device=self.device)

    def dof(self):
        import torch
        return torch.empty(self.n_dof, dtype=self.dtype, device=self.device)

    # --- C calls
    def set_design(self, rho):
        to_set_design(self, rho)

    def apply_K(self, u, y=None):
        y = self.dof() if y is None else y
        to_apply_K(self, u, y)
        return y

    def residual(self, u, r=None, z=None, gt=None, want_scalars=True):
        r = self.dof() if r is None else r
        sc = to_residual(self, u, r, z, gt, want_scalars)
        return r, sc

    def smooth(self, x, b, omega, y=None):
        y = self.dof() if y is None else y
        to_smooth(self, x, b, y, omega)
        return y

    def inner_solve(self, u, nsteps, want_res=False):
        return to_inner_solve(self, u, nsteps, want_res)

    def sensitivity(self, u, g=None):
        g = self.elem() if g is None else g
        to_sensitivity(self, u, g)
        return g

    def filter(self, x, y=None, transpose=False):
        y = self.elem() if y is None else y
        to_filter(self, x, y, transpose)
        return y

    def project(self, w, rho=None, want_lambda=True):
        rho = self.elem() if rho is None else rho
        lam = to_project(self, w, rho, want_lambda)
        return rho, lam

    def step(self, n_outer=1, want_stats=True):
        return to_step(self, n_outer, want_stats)

    def get_state(self):
        rho, u = self.elem(), self.dof()
        k, a0 = to_get_state(self, rho, u)
        return rho, u, k, a0

    def set_state(self, rho, u, k, alpha0):
        to_set_state(self, rho, u, k, alpha0)

    def check(self):
        to_check(self)


def _h(P):
    return P.handle if isinstance(P, Problem) else P


def _dt(P):
    return P.dtype


def to_set_design(P, rho):
    _abi.check(_lib().to_set_design(_h(P), _ptr(rho, _dt(P), P.n_elem, "rho"), _stream(P.device)))


def to_apply_K(P, u, y):
    _abi.check(_lib().to_apply_K(_h(P), _ptr(u, _dt(P), P.n_dof, "u"), _ptr(y, _dt(P), P.n_dof, "y"),
                                 _stream(P.device)))


def to_residual(P, u, r, z=None, gt=None, want_scalars=True):
    sc = (C.c_double * 4)()
    _abi.check(_lib().to_residual(_h(P), _ptr(u, _dt(P), P.n_dof, "u"), _ptr(r, _dt(P), P.n_dof, "r"),
                                  _ptr(z, _dt(P), P.n_dof, "z"), _ptr(gt, _dt(P), P.n_elem, "gt"),
                                  sc if want_scalars else None, _stream(P.device)))
    return dict(rz=sc[0], res2=sc[1], res_inf=sc[2], fu=sc[3]) if want_scalars else None


def to_smooth(P, x, b, y, omega):
    _abi.check(_lib().to_smooth(_h(P), _ptr(x, _dt(P), P.n_dof, "x"), _ptr(b, _dt(P), P.n_dof, "b"),
                                _ptr(y, _dt(P), P.n_dof, "y"), float(omega), _stream(P.device)))


def to_inner_solve(P, u, nsteps, want_res=False):
    res = C.c_double()
    _abi.check(_lib().to_inner_solve(_h(P), _ptr(u, _dt(P), P.n_dof, "u"), int(nsteps),
                                     C.byref(res) if want_res else None, _stream(P.device)))
    return res.value if want_res else None


def to_sensitivity(P, u, g):
    _abi.check(_lib().to_sensitivity(_h(P), _ptr(u, _dt(P), P.n_dof, "u"), _ptr(g, _dt(P), P.n_elem, "g"),
                                     _stream(P.device)))


def to_filter(P, x, y, transpose=False):
    _abi.check(_lib().to_filter(_h(P), _ptr(x, _dt(P), P.n_elem, "x"), _ptr(y, _dt(P), P.n_elem, "y"),
                                1 if transpose else 0, _stream(P.device)))


def to_project(P, w, rho, want_lambda=True):
    lam = C.c_double()
    _abi.check(_lib().to_project(_h(P), _ptr(w, _dt(P), P.n_elem, "w"), _ptr(rho, _dt(P), P.n_elem, "rho"),
                                 C.byref(lam) if want_lambda else None, _stream(P.device)))
    return lam.value if want_lambda else None


def to_step(P, n_outer=1, want_stats=True):
    if want_stats:
        arr = (to_stats * max(int(n_outer), 1))()
        _abi.check(_lib().to_step(_h(P), int(n_outer), arr, _stream(P.device)))
        return [arr[i].as_dict() for i in range(int(n_outer))]
    _abi.check(_lib().to_step(_h(P), int(n_outer), None, _stream(P.device)))
    return None


def to_get_state(P, rho=None, u=None, scalars=True):
    """Copy rho and u out; with scalars (the default) also return (k, alpha0), which makes the
    call synchronise; without them the copies stay asynchronous on the current stream."""
    if not scalars:
        _abi.check(_lib().to_get_state(_h(P), _ptr(rho, _dt(P), P.n_elem, "rho"), _ptr(u, _dt(P), P.n_dof, "u"),
                                       None, None, _stream(P.device)))
        return None
    k, a0 = C.c_int64(), C.c_double()
    _abi.check(_lib().to_get_state(_h(P), _ptr(rho, _dt(P), P.n_elem, "rho"), _ptr(u, _dt(P), P.n_dof, "u"),
                                   C.byref(k), C.byref(a0), _stream(P.device)))
    return k.value, a0.value


def to_get_stats(P, n, out):
    """Enqueue the copy of the last to_step call's first n records into `out` (host memory
    of n to_stats records: a pointer, or a buffer with data_ptr(), e.g. a pinned uint8
    tensor) on the current stream; read it after synchronising (to_stats.from_address)."""
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else int(out)
    _abi.check(_lib().to_get_stats(_h(P), int(n), C.c_void_p(ptr), _stream(P.device)))


def _host_ptr(t, dtype, n, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError(f"{name} must be a host tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} entries, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def to_step_host(P, rho_in, rho_out=None, stats_out=None):
    """One outer iteration fed from host memory: rho_in (host tensor, pinned for an
    asynchronous copy) in, the new design into rho_out (host tensor) and the iteration's
    record into stats_out (host buffer of one to_stats with data_ptr(), or None), one
    synchronisation.  Raises ToError with the record's status on a device-side error."""
    dt = _dt(P)
    pin = _host_ptr(rho_in, dt, P.n_elem, "rho_in")
    pout = None if rho_out is None else _host_ptr(rho_out, dt, P.n_elem, "rho_out")
    pst = None if stats_out is None else C.c_void_p(stats_out.data_ptr() if hasattr(stats_out, "data_ptr")
                                                    else int(stats_out))
    _abi.check(_lib().to_step_host(_h(P), pin, pout, pst, _stream(P.device)))


def to_set_state(P, rho=None, u=None, k=1, alpha0=0.0):
    _abi.check(_lib().to_set_state(_h(P), _ptr(rho, _dt(P), P.n_elem, "rho"), _ptr(u, _dt(P), P.n_dof, "u"),
                                   int(k), float(alpha0), _stream(P.device)))


def to_check(P):
    _abi.check(_lib().to_check(_h(P), _stream(P.device)))


def to_barrier_selftest(P, absent_block, spin_limit):
    _abi.check(_lib().to_barrier_selftest(_h(P), int(absent_block), int(spin_limit), _stream(P.device)))


def to_compliance_truncated(P, rho, T, beta, want_J=True):
    J = C.c_double()
    _abi.check(_lib().to_compliance_truncated(_h(P), _ptr(rho, _dt(P), P.n_elem, "rho"), int(T), float(beta),
                                              C.byref(J) if want_J else None, _stream(P.device)))
    return J.value if want_J else None


def to_compliance_truncated_grad(P, scale, g):
    _abi.check(_lib().to_compliance_truncated_grad(_h(P), float(scale), _ptr(g, _dt(P), P.n_elem, "g"),
                                                   _stream(P.device)))


def to_compliance_truncated_id(P):
    i = C.c_int64()
    _abi.check(_lib().to_compliance_truncated_id(_h(P), C.byref(i)))
    return i.value


def to_batch_create(problems):
    arr = (C.c_void_p * len(problems))(*[_h(p).value for p in problems])
    out = C.c_void_p()
    _abi.check(_lib().to_batch_create(arr, len(problems), C.byref(out)))
    return out


def to_batch_destroy(B):
    _lib().to_batch_destroy(B)


def to_batch_tile(B):
    kc, us = C.c_int32(), C.c_double()
    _abi.check(_lib().to_batch_tile(B, C.byref(kc), C.byref(us)))
    return kc.value, us.value


def to_batch_step(B, n_problems, n_outer, device, want_stats=True):
    if want_stats:
        arr = (to_stats * (n_problems * max(int(n_outer), 1)))()
        _abi.check(_lib().to_batch_step(B, int(n_outer), arr, _stream(device)))
        return [[arr[p * n_outer + i].as_dict() for i in range(n_outer)] for p in range(n_problems)]
    _abi.check(_lib().to_batch_step(B, int(n_outer), None, _stream(device)))
    return None


class Batch:
    """Many Problems advanced together (one launch per phase); keeps them alive."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.device = self.problems[0].device
        self.handle = to_batch_create(self.problems)

    def step(self, n_outer=1, want_stats=True):
        return to_batch_step(self.handle, len(self.problems), n_outer, self.device, want_stats)

    def tile(self):
        """(planes per operator tile, microseconds of one batched K u) picked by the autotuner."""
        return to_batch_tile(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            to_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def to_project_noalloc(w, rho, vbar, lo=0.0, hi=1.0, want_lambda=True):
    """Projection onto X without a problem and without any device allocation
    (for callers that may not allocate device memory); see include/to.h."""
    import torch
    if w.dtype not in (torch.float32, torch.float64) or rho.dtype != w.dtype:
        raise TypeError("w and rho must both be float32 or both float64")
    n = w.numel()
    prec = TO_FP64 if w.dtype == torch.float64 else TO_FP32_MIXED
    lam = C.c_double()
    _abi.check(_lib().to_project_noalloc(_ptr(w, w.dtype, n, "w"), _ptr(rho, w.dtype, n, "rho"), n, prec,
                                         float(vbar), float(lo), float(hi), C.byref(lam) if want_lambda else None,
                                         _stream(w.device)))
    return lam.value if want_lambda else None


def to_last_error() -> str:
    m = _lib().to_last_error()
    return m.decode() if m else ""
