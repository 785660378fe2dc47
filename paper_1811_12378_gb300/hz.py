"""Python binding of libhz: argument marshalling over the C ABI in include/hz.h.

Every step of the method runs in libhz's CUDA kernels; this module only converts torch
tensors and numpy arrays into pointers and sizes.  torch supplies device memory and
streams.  If the library is missing, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

HZ_C128 = 0
HZ_MIXED_C64 = 1
HZ_MIXED_C64_FCI32 = 2
HZ_MIXED_C64_FF = 3

# discretisations of hz_grid.discretization
HZ_DISC_FD7 = 0
HZ_DISC_SPECTRAL = 1

STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of memory",
          4: "not converged", 5: "breakdown", 6: "diverged", 7: "set-up failed", 8: "timeout"}

# every exported symbol declared in include/hz.h
EXPORTS = ["hz_problem_create", "hz_plan", "hz_problem_destroy", "hz_problem_get_info",
           "hz_problem_nodes", "hz_problem_set_nodes", "hz_apply_shifted", "hz_apply_2x2",
           "hz_shifted_solve",
           "hz_fci", "hz_solve", "hz_solve_batched", "hz_profile_enable", "hz_profile_read",
           "hz_problem_fused_tail", "hz_problem_fused_arnoldi", "hz_problem_set_spin_limit",
           "hz_residual_noalloc", "hz_net_param_count", "hz_net_create", "hz_net_destroy",
           "hz_net_set_params", "hz_net_get_params", "hz_net_forward", "hz_net_train_step",
           "hz_net_train_fields", "hz_problem_set_preconditioner", "hz_conv3d",
           "hz_conv3d_backward", "hz_conv3d_workspace_bytes", "hz_problem_set_inner_ilu",
           "hz_ilu0_apply", "hz_problem_set_inner_invlap", "hz_invlap_apply",
           "hz_status_string", "hz_last_error", "hz_launch_count"]

# kernel classes of hz_profile_read
PROF_POLY, PROF_STENCIL, PROF_KRYLOV = 0, 1, 2


class HzGrid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double),
                ("omega", C.c_double), ("layer_cells", C.c_int), ("sigma_max", C.c_double),
                ("discretization", C.c_int)]


class HzContour(C.Structure):
    _fields_ = [("J", C.c_int), ("t", C.c_double), ("eps", C.c_double), ("qmax", C.c_int),
                ("reduction", C.c_double)]


class HzLimits(C.Structure):
    _fields_ = [("nrhs_max", C.c_int), ("restart_max", C.c_int), ("inner_k_max", C.c_int),
                ("autotune", C.c_int), ("flags", C.c_int)]


# hz_limits.flags bits
HZ_LIMIT_SWEEPS_C64 = 1
HZ_LIMIT_Z_C64 = 2
HZ_LIMIT_CASE_TWO = 4


class HzSolveOpts(C.Structure):
    _fields_ = [("restart_m", C.c_int), ("inner_k", C.c_int), ("rtol", C.c_double),
                ("max_cycles", C.c_int), ("precision", C.c_int), ("fixed_its", C.c_int)]


class HzSolveStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("its", C.c_int), ("matvecs", C.c_longlong),
                ("converged", C.c_int), ("rel_res_true", C.c_double)]


class HzInfo(C.Structure):
    _fields_ = [("s", C.c_double), ("b1", C.c_double), ("b2", C.c_double),
                ("rho2", C.c_double), ("J", C.c_int), ("stages", C.c_int), ("n", C.c_longlong),
                ("tile_poly_zc", C.c_int * 3), ("tile_poly_rows", C.c_int * 3),
                ("tile_stencil_zc", C.c_int), ("tile_stencil_rows", C.c_int)]


class HzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libhz: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libhz (building it first if needed).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libhz is not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    P = C.c_void_p
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    lib.hz_problem_create.argtypes = [C.POINTER(HzGrid), dp, C.POINTER(HzContour),
                                      C.POINTER(HzLimits), C.POINTER(P)]
    lib.hz_plan.argtypes = [C.POINTER(HzGrid), dp, C.POINTER(HzContour), C.POINTER(HzInfo),
                            dp, dp, dp, dp, ip, dp, ip]
    lib.hz_problem_destroy.argtypes = [P]
    lib.hz_problem_get_info.argtypes = [P, C.POINTER(HzInfo)]
    lib.hz_problem_nodes.argtypes = [P, dp, dp, dp, dp, ip, dp, ip]
    lib.hz_problem_set_nodes.argtypes = [P, C.c_int, dp, dp, dp, dp, ip, ip]
    lib.hz_apply_shifted.argtypes = [P, C.c_double, C.c_double, P, P, C.c_int, C.c_int, P]
    lib.hz_apply_2x2.argtypes = [P, C.c_double, C.c_double, P, P, C.c_int, C.c_int, P]
    lib.hz_shifted_solve.argtypes = [P, C.c_int, P, P, C.c_int, C.c_int, P]
    lib.hz_fci.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, P]
    lib.hz_solve.argtypes = [P, P, P, C.c_int, C.POINTER(HzSolveOpts), C.POINTER(HzSolveStats), P]
    lib.hz_solve_batched.argtypes = [C.POINTER(P), C.c_int, C.POINTER(P), C.POINTER(P),
                                     C.POINTER(C.c_int), C.POINTER(HzSolveOpts),
                                     C.POINTER(HzSolveStats), P]
    lib.hz_profile_enable.argtypes = [P, C.c_int]
    lib.hz_problem_fused_tail.argtypes = [P, C.c_int]
    lib.hz_problem_fused_arnoldi.argtypes = [P, C.c_int]
    lib.hz_problem_set_spin_limit.argtypes = [P, C.c_longlong]
    lib.hz_profile_read.argtypes = [P, C.c_int, C.POINTER(C.c_longlong), dp, dp, dp]
    lib.hz_residual_noalloc.argtypes = [C.POINTER(HzGrid), P, C.c_double, P, C.c_double, P, P, P,
                                        C.c_int, P]
    fp = C.POINTER(C.c_float)
    lib.hz_net_param_count.argtypes = []
    lib.hz_net_param_count.restype = C.c_longlong
    lib.hz_net_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(P)]
    lib.hz_net_destroy.argtypes = [P]
    lib.hz_net_set_params.argtypes = [P, fp]
    lib.hz_net_get_params.argtypes = [P, fp]
    lib.hz_net_forward.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, P]
    lib.hz_net_train_step.argtypes = [P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, P,
                                      dp, P]
    lib.hz_net_train_fields.argtypes = [P, P, P, P, C.c_int, C.c_float, dp, P]
    lib.hz_problem_set_preconditioner.argtypes = [P, P, C.c_int]
    lib.hz_problem_set_inner_ilu.argtypes = [P, C.c_int]
    lib.hz_ilu0_apply.argtypes = [P, P, P, C.c_int, P]
    lib.hz_problem_set_inner_invlap.argtypes = [P, C.c_int]
    lib.hz_invlap_apply.argtypes = [P, P, P, C.c_int, P]
    lib.hz_conv3d.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P, P, C.c_int,
                              C.c_int, P, P, P]
    lib.hz_conv3d_backward.argtypes = [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P,
                                       C.c_int, P, P, P, P]
    lib.hz_conv3d_workspace_bytes.argtypes = [C.c_int, C.c_int]
    lib.hz_conv3d_workspace_bytes.restype = C.c_longlong
    lib.hz_status_string.argtypes = [C.c_int]
    lib.hz_status_string.restype = C.c_char_p
    lib.hz_last_error.argtypes = []
    lib.hz_last_error.restype = C.c_char_p
    lib.hz_launch_count.argtypes = []
    lib.hz_launch_count.restype = C.c_ulonglong
    for name in EXPORTS:
        fn = getattr(lib, name)
        if name not in ("hz_status_string", "hz_last_error", "hz_launch_count",
                        "hz_net_param_count", "hz_conv3d_workspace_bytes"):
            fn.restype = C.c_int
    _lib = lib
    return lib


def _check(status: int, lib=None, allow=()):
    if status != 0 and status not in allow:
        lib = lib or load()
        raise HzError(status, lib.hz_last_error().decode())
    return status


def launch_count() -> int:
    return int(load().hz_launch_count())


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _grid(nx, ny, nz, h, omega, layer_cells, sigma_max, discretization=HZ_DISC_FD7):
    return HzGrid(int(nx), int(ny), int(nz), float(h), float(omega), int(layer_cells),
                  float(sigma_max), int(discretization))


def _tables_from(buf):
    z, sg, z0, dl, q, nu, sw = buf
    return {"z": z[0::2] + 1j * z[1::2], "sigma": sg[0::2] + 1j * sg[1::2],
            "z0": z0[0::2] + 1j * z0[1::2], "delta": dl.copy(), "q": q.copy(), "nu": nu.copy(),
            "sweeps": sw.copy()}


def _new_tables(J):
    return (np.zeros(2 * J), np.zeros(2 * J), np.zeros(2 * J), np.zeros(J),
            np.zeros(J, dtype=np.int32), np.zeros(J), np.zeros(J, dtype=np.int32))


def plan(c: np.ndarray, h: float, omega: float, layer_cells: int, sigma_max: float, J: int,
         t: float, eps: float, qmax: int = 5, reduction: float = 5.0,
         discretization: int = HZ_DISC_FD7):
    """Host-only set-up of libhz (no GPU): (info dict, node tables dict)."""
    lib = load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    nz, ny, nx = c.shape
    g = _grid(nx, ny, nz, h, omega, layer_cells, sigma_max, discretization)
    co = HzContour(int(J), float(t), float(eps), int(qmax), float(reduction))
    info = HzInfo()
    tb = _new_tables(J)
    _check(lib.hz_plan(C.byref(g), _dp(c), C.byref(co), C.byref(info), _dp(tb[0]), _dp(tb[1]),
                       _dp(tb[2]), _dp(tb[3]), _ip(tb[4]), _dp(tb[5]), _ip(tb[6])), lib)
    return _info_dict(info), _tables_from(tb)


def _info_dict(info: HzInfo):
    return {"s": info.s, "b1": info.b1, "b2": info.b2, "rho2": info.rho2, "J": info.J,
            "stages": info.stages, "n": info.n,
            "tile_poly_zc": list(info.tile_poly_zc), "tile_poly_rows": list(info.tile_poly_rows),
            "tile_stencil": [info.tile_stencil_zc, info.tile_stencil_rows]}


@dataclass
class SolveStats:
    cycles: int
    its: int
    matvecs: int
    converged: bool
    rel_res_true: float


def _stream(stream):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


def _dev_ptr(t, dtype, n):
    import torch
    if not t.is_cuda:
        raise ValueError("libhz fields must be CUDA tensors")
    if t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("fields must be contiguous")
    if t.numel() % n:
        raise ValueError(f"field size {t.numel()} is not a multiple of the grid size {n}")
    return C.c_void_p(t.data_ptr()), t.numel() // n


class Problem:
    """A Helmholtz problem on the current CUDA device (wraps hz_problem_create).

    c: wavespeed, numpy (nz, ny, nx).  All fields passed to the methods are contiguous CUDA
    tensors of shape (nvec, nz, ny, nx) (or any shape with nvec*n elements), complex128 unless
    a complex64 precision is asked for.
    """

    def __init__(self, c, h, omega, layer_cells, sigma_max, J, t, eps, qmax=5, reduction=5.0,
                 nrhs_max=1, restart_max=30, inner_k_max=8, autotune=True, flags=0,
                 discretization=HZ_DISC_FD7):
        self._lib = load()
        c = np.ascontiguousarray(c, dtype=np.float64)
        self.shape = c.shape
        nz, ny, nx = c.shape
        self.n = nx * ny * nz
        g = _grid(nx, ny, nz, h, omega, layer_cells, sigma_max, discretization)
        co = HzContour(int(J), float(t), float(eps), int(qmax), float(reduction))
        lim = HzLimits(int(nrhs_max), int(restart_max), int(inner_k_max), 1 if autotune else 0,
                       int(flags))
        handle = C.c_void_p()
        _check(self._lib.hz_problem_create(C.byref(g), _dp(c), C.byref(co), C.byref(lim),
                                           C.byref(handle)), self._lib)
        self._h = handle
        self.nrhs_max = nrhs_max
        self.case_two = bool(int(flags) & HZ_LIMIT_CASE_TWO)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hz_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def info(self):
        info = HzInfo()
        _check(self._lib.hz_problem_get_info(self._h, C.byref(info)), self._lib)
        return _info_dict(info)

    def fused_tail(self, mode=1):
        """Complex64 FCI steps 3-5: 1 one cooperative kernel (default), 2 the same with the
        norm after the second Gram-Schmidt pass always summed, 0 (or False) one kernel per
        piece."""
        _check(self._lib.hz_problem_fused_tail(self._h, int(mode)), self._lib)

    def fused_arnoldi(self, mode=1):
        """Float-pair outer Arnoldi step: 1 one cooperative kernel (default), 2 the same with
        the last norm always summed, 0 (or False) five kernels."""
        _check(self._lib.hz_problem_fused_arnoldi(self._h, int(mode)), self._lib)

    def set_preconditioner(self, net=None, mode: int = 0):
        """Right preconditioner of solve(): 0 FCI; 1 the network; 2 network then FCI on its
        residual; 3 FCI then the network on its residual (hz_problem_set_preconditioner)."""
        _check(self._lib.hz_problem_set_preconditioner(
            self._h, net._h if net is not None else None, int(mode)), self._lib)

    def set_inner_ilu(self, on: bool = True):
        """ILU(0) of the 7-point Laplacian as the inner GMRES's right preconditioner."""
        _check(self._lib.hz_problem_set_inner_ilu(self._h, 1 if on else 0), self._lib)

    def ilu0_apply(self, t, out=None, stream=None):
        """z = M^{-1} t with the ILU(0) factors (complex128 fields of the grid)."""
        import torch
        tp, nvec = _dev_ptr(t, torch.complex128, self.n)
        z = torch.empty_like(t) if out is None else out
        zp, _ = _dev_ptr(z, torch.complex128, self.n)
        _check(self._lib.hz_ilu0_apply(self._h, tp, zp, nvec, _stream(stream)), self._lib)
        return z

    def set_inner_invlap(self, on: bool = True):
        """Spectral problems: the regularised inverse Laplacian 1/max(lambda, 1) as the inner
        GMRES's right preconditioner (hz_problem_set_inner_invlap)."""
        _check(self._lib.hz_problem_set_inner_invlap(self._h, 1 if on else 0), self._lib)

    def invlap_apply(self, t, out=None, stream=None):
        """z = M^{-1} t with the regularised inverse Laplacian (complex128 fields)."""
        import torch
        tp, nvec = _dev_ptr(t, torch.complex128, self.n)
        z = torch.empty_like(t) if out is None else out
        zp, _ = _dev_ptr(z, torch.complex128, self.n)
        _check(self._lib.hz_invlap_apply(self._h, tp, zp, nvec, _stream(stream)), self._lib)
        return z

    def set_spin_limit(self, polls: int = -1):
        """Poll limit of the cooperative kernels' grid barriers (-1: the default, ~1 s)."""
        _check(self._lib.hz_problem_set_spin_limit(self._h, int(polls)), self._lib)

    def profile(self, on: bool = True):
        """Start (and zero) or stop per-kernel-class CUDA-event timing."""
        _check(self._lib.hz_profile_enable(self._h, 1 if on else 0), self._lib)

    def profile_read(self, cls: int, flops: bool = False):
        """(launches, milliseconds, algorithmic bytes[, float64 flops]) of a kernel class since
        profile()."""
        nl, ms, by, fl = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
        _check(self._lib.hz_profile_read(self._h, int(cls), C.byref(nl), C.byref(ms),
                                         C.byref(by), C.byref(fl)), self._lib)
        if flops:
            return int(nl.value), float(ms.value), float(by.value), float(fl.value)
        return int(nl.value), float(ms.value), float(by.value)

    def nodes(self):
        J = self.info["J"]
        tb = _new_tables(J)
        _check(self._lib.hz_problem_nodes(self._h, _dp(tb[0]), _dp(tb[1]), _dp(tb[2]), _dp(tb[3]),
                                          _ip(tb[4]), _dp(tb[5]), _ip(tb[6])), self._lib)
        return _tables_from(tb)

    def set_nodes(self, z, sigma, z0, delta, q, sweeps):
        z = np.asarray(z, dtype=np.complex128)
        J = len(z)
        zr = np.ascontiguousarray(np.stack([z.real, z.imag], 1).ravel())
        s = np.asarray(sigma, dtype=np.complex128)
        sr = np.ascontiguousarray(np.stack([s.real, s.imag], 1).ravel())
        z0 = np.asarray(z0, dtype=np.complex128)
        z0r = np.ascontiguousarray(np.stack([z0.real, z0.imag], 1).ravel())
        dl = np.ascontiguousarray(delta, dtype=np.float64)
        qq = np.ascontiguousarray(q, dtype=np.int32)
        sw = np.ascontiguousarray(sweeps, dtype=np.int32)
        _check(self._lib.hz_problem_set_nodes(self._h, J, _dp(zr), _dp(sr), _dp(z0r), _dp(dl),
                                              _ip(qq), _ip(sw)), self._lib)

    def apply_shifted(self, x, z=0.0, out=None, precision=None, stream=None):
        import torch
        prec = precision if precision is not None else (
            HZ_MIXED_C64 if x.dtype == torch.complex64 else HZ_C128)
        dt = torch.complex64 if prec == HZ_MIXED_C64 else torch.complex128
        xp, nvec = _dev_ptr(x, dt, self.n)
        y = torch.empty_like(x) if out is None else out
        yp, _ = _dev_ptr(y, dt, self.n)
        z = complex(z)
        _check(self._lib.hz_apply_shifted(self._h, z.real, z.imag, xp, yp, nvec, prec,
                                          _stream(stream)), self._lib)
        return y

    def apply_2x2(self, x, z=0.0, out=None, precision=None, stream=None):
        """Case Two: ((iC - I) - zI) x on vectors of two stacked fields (x1; x2)."""
        import torch
        prec = precision if precision is not None else (
            HZ_MIXED_C64 if x.dtype == torch.complex64 else HZ_C128)
        dt = torch.complex64 if prec == HZ_MIXED_C64 else torch.complex128
        xp, nvec = _dev_ptr(x, dt, 2 * self.n)
        y = torch.empty_like(x) if out is None else out
        yp, _ = _dev_ptr(y, dt, 2 * self.n)
        z = complex(z)
        _check(self._lib.hz_apply_2x2(self._h, z.real, z.imag, xp, yp, nvec, prec,
                                      _stream(stream)), self._lib)
        return y

    def shifted_solve(self, node, f, out=None, precision=None, stream=None):
        import torch
        prec = precision if precision is not None else (
            HZ_MIXED_C64 if f.dtype == torch.complex64 else HZ_C128)
        dt = torch.complex64 if prec == HZ_MIXED_C64 else torch.complex128
        nf = self.n * (2 if self.case_two else 1)
        fp, nvec = _dev_ptr(f, dt, nf)
        y = torch.empty_like(f) if out is None else out
        yp, _ = _dev_ptr(y, dt, nf)
        _check(self._lib.hz_shifted_solve(self._h, int(node), fp, yp, nvec, prec,
                                          _stream(stream)), self._lib)
        return y

    def fci(self, r, inner_k=4, precision=HZ_C128, out=None, stream=None):
        import torch
        nf = self.n * (2 if self.case_two else 1)
        rp, nvec = _dev_ptr(r, torch.complex128, nf)
        y = torch.empty_like(r) if out is None else out
        yp, _ = _dev_ptr(y, torch.complex128, nf)
        _check(self._lib.hz_fci(self._h, rp, yp, nvec, int(inner_k), int(precision),
                                _stream(stream)), self._lib)
        return y

    def solve(self, f, restart=30, inner_k=4, rtol=1e-8, max_cycles=50, precision=HZ_C128,
              fixed_its=0, out=None, stream=None, check=True):
        """FGMRES(restart) with FCI; f in physical units.  Returns (u, [SolveStats])."""
        import torch
        fp, nrhs = _dev_ptr(f, torch.complex128, self.n)
        if self.case_two:  # Y = (i u; u): two fields per right-hand side
            u = torch.empty((nrhs, 2 * self.n), dtype=torch.complex128,
                            device=f.device) if out is None else out
        else:
            u = torch.empty_like(f) if out is None else out
        up, _ = _dev_ptr(u, torch.complex128, self.n * (2 if self.case_two else 1))
        opts = HzSolveOpts(int(restart), int(inner_k), float(rtol), int(max_cycles),
                           int(precision), int(fixed_its))
        st = (HzSolveStats * max(nrhs, 1))()
        status = self._lib.hz_solve(self._h, fp, up, nrhs, C.byref(opts), st, _stream(stream))
        _check(status, self._lib, allow=() if check else (4,))
        stats = [SolveStats(s.cycles, s.its, s.matvecs, bool(s.converged), s.rel_res_true)
                 for s in st[:nrhs]]
        return u, stats


def solve_batched(problems, fs, restart=30, inner_k=4, rtol=1e-8, max_cycles=50,
                  precision=HZ_C128, fixed_its=0, outs=None, stream=None, check=True):
    """hz_solve_batched over several Problems: fs[i] holds problem i's right-hand sides.
    Returns ([u_i], [[SolveStats] per problem])."""
    import torch
    lib = load()
    k = len(problems)
    us = [torch.empty_like(f) for f in fs] if outs is None else outs
    P = C.c_void_p
    hp = (P * k)(*[p._h for p in problems])
    fp = (P * k)()
    up = (P * k)()
    nr = (C.c_int * k)()
    for i, (pr, f, u) in enumerate(zip(problems, fs, us)):
        fp[i], nr[i] = _dev_ptr(f, torch.complex128, pr.n)
        up[i], _ = _dev_ptr(u, torch.complex128, pr.n)
    opts = HzSolveOpts(int(restart), int(inner_k), float(rtol), int(max_cycles), int(precision),
                       int(fixed_its))
    tot = max(1, sum(nr))
    st = (HzSolveStats * tot)()
    status = lib.hz_solve_batched(hp, k, fp, up, nr, C.byref(opts), st, _stream(stream))
    _check(status, lib, allow=() if check else (4,))
    out, off = [], 0
    for i in range(k):
        out.append([SolveStats(s.cycles, s.its, s.matvecs, bool(s.converged), s.rel_res_true)
                    for s in st[off:off + nr[i]]])
        off += nr[i]
    return us, out


# ---------------------------------------------------------------------------- learned part
# The network's 3x3x3 convolutions in parameter order: (name, input channels, output channels)
NET_CONVS = [("e1a", 8, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32),
             ("e3a", 32, 64), ("e3b", 64, 64), ("ba", 64, 128), ("bb", 128, 128),
             ("d3a", 192, 64), ("d3b", 64, 64), ("d2a", 96, 32), ("d2b", 32, 32),
             ("d1a", 48, 16), ("d1b", 16, 16)]


def flatten_params(params: dict) -> np.ndarray:
    """The flat float32 parameter array of include/hz.h from {name.w, name.b, head.w, head.b}."""
    parts = []
    for name, _, _ in NET_CONVS:
        parts += [np.ravel(params[name + ".w"]), np.ravel(params[name + ".b"])]
    parts += [np.ravel(params["head.w"]), np.ravel(params["head.b"])]
    return np.ascontiguousarray(np.concatenate(parts), dtype=np.float32)


def unflatten_params(flat: np.ndarray) -> dict:
    out, off = {}, 0
    for name, ci, co in NET_CONVS:
        out[name + ".w"] = flat[off:off + co * 27 * ci].reshape(co, 27, ci)
        off += co * 27 * ci
        out[name + ".b"] = flat[off:off + co]
        off += co
    out["head.w"] = flat[off:off + 32].reshape(2, 16)
    out["head.b"] = flat[off + 32:off + 34]
    return out


def init_params(seed: int) -> dict:
    """Seeded starting weights: He-normal 3x3x3 weights (std sqrt(2 / fan_in)), zero biases,
    head weights of std 1/4 (fan-in 16)."""
    g = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co in NET_CONVS:
        p[name + ".w"] = g.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci))
        p[name + ".b"] = np.zeros(co)
    p["head.w"] = g.standard_normal((2, 16)) / 4.0
    p["head.b"] = np.zeros(2)
    return p


class Net:
    """The learned right preconditioner's network on the current CUDA device (hz_net_create):
    activation storage for up to batch_max volumes of D x H x W voxels."""

    def __init__(self, D, H, W, batch_max=1):
        self._lib = load()
        h = C.c_void_p()
        _check(self._lib.hz_net_create(int(D), int(H), int(W), int(batch_max), C.byref(h)),
               self._lib)
        self._h = h
        self.n_params = int(self._lib.hz_net_param_count())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hz_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        if a.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {a.size}")
        _check(self._lib.hz_net_set_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))),
               self._lib)

    def get_params(self) -> np.ndarray:
        a = np.empty(self.n_params, dtype=np.float32)
        _check(self._lib.hz_net_get_params(self._h, a.ctypes.data_as(C.POINTER(C.c_float))),
               self._lib)
        return a

    def forward(self, x, stream=None):
        """y = N(x) for a float32 CUDA tensor x of shape (B, D, H, W, 8)."""
        import torch
        B, D, H, W, c = x.shape
        if c != 8 or x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x: contiguous float32 CUDA tensor (B, D, H, W, 8)")
        y = torch.empty((B, D, H, W, 2), dtype=torch.float32, device=x.device)
        _check(self._lib.hz_net_forward(self._h, C.c_void_p(x.data_ptr()),
                                        C.c_void_p(y.data_ptr()), B, D, H, W, _stream(stream)),
               self._lib)
        return y

    def train_step(self, x, target, lr=0.0, want_grads=False, stream=None):
        """One step (loss, gradients, Adam with lr) on float32 CUDA tensors x (B, D, H, W, 8)
        and target (B, D, H, W, 2).  Returns (loss, flat gradient tensor or None)."""
        import torch
        B, D, H, W, _ = x.shape
        g = torch.empty(self.n_params, dtype=torch.float32, device=x.device) if want_grads else None
        loss = C.c_double()
        _check(self._lib.hz_net_train_step(self._h, C.c_void_p(x.data_ptr()),
                                           C.c_void_p(target.data_ptr()), B, D, H, W,
                                           float(lr), C.c_void_p(g.data_ptr()) if g is not None
                                           else None, C.byref(loss), _stream(stream)), self._lib)
        return float(loss.value), g

    def train_fields(self, problem, r, e, lr, stream=None):
        """One training step on complex128 field pairs (r, e) of a Problem's grid."""
        import torch
        rp, nv = _dev_ptr(r, torch.complex128, problem.n)
        ep, _ = _dev_ptr(e, torch.complex128, problem.n)
        loss = C.c_double()
        _check(self._lib.hz_net_train_fields(self._h, problem._h, rp, ep, nv, float(lr),
                                             C.byref(loss), _stream(stream)), self._lib)
        return float(loss.value)


def _ws(lib, cin, cout, device):
    import torch
    nbytes = int(lib.hz_conv3d_workspace_bytes(int(cin), int(cout)))
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def conv3d(x, w, bias=None, relu=False, stream=None):
    """y = conv3(x, w) + bias on the tensor cores: x bf16 CUDA (B, D, H, W, Cin), w float32
    (Cout, 27, Cin); returns float32 (B, D, H, W, Cout)."""
    import torch
    lib = load()
    B, D, H, W, cin = x.shape
    cout = w.shape[0]
    y = torch.empty((B, D, H, W, cout), dtype=torch.float32, device=x.device)
    ws = _ws(lib, cin, cout, x.device)
    _check(lib.hz_conv3d(C.c_void_p(x.data_ptr()), B, D, H, W, cin, C.c_void_p(w.data_ptr()),
                         C.c_void_p(bias.data_ptr()) if bias is not None else None, cout,
                         1 if relu else 0, C.c_void_p(y.data_ptr()), C.c_void_p(ws.data_ptr()),
                         _stream(stream)), lib)
    return y


def conv3d_backward(x, g, w, want_dx=True, stream=None):
    """(dx, dw) of conv3 for bf16 CUDA x (B, D, H, W, Cin), bf16 g (B, D, H, W, Cout) and
    float32 w (Cout, 27, Cin)."""
    import torch
    lib = load()
    B, D, H, W, cin = x.shape
    cout = g.shape[-1]
    dw = torch.empty((cout, 27, cin), dtype=torch.float32, device=x.device)
    dx = torch.empty((B, D, H, W, cin), dtype=torch.float32, device=x.device) if want_dx else None
    ws = _ws(lib, cin, cout, x.device)
    _check(lib.hz_conv3d_backward(C.c_void_p(x.data_ptr()), C.c_void_p(g.data_ptr()), B, D, H, W,
                                  cin, C.c_void_p(w.data_ptr()), cout,
                                  C.c_void_p(dx.data_ptr()) if dx is not None else None,
                                  C.c_void_p(dw.data_ptr()), C.c_void_p(ws.data_ptr()),
                                  _stream(stream)), lib)
    return dx, dw
