"""Thin ctypes binding of libmh3d.so (include/mh3d.h).

Argument marshalling only: every step of the operator and the solver runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  The
functions carry the C names; tensors are checked for device, dtype, size and
contiguity before their pointers are passed.  There is no fallback: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_void_p, c_char_p, c_ulonglong
from typing import Optional, Sequence

from . import build as _build

MH3D_OK = 0
MH3D_ERR_INVALID_ARG = 1
MH3D_ERR_UNSUPPORTED_SIZE = 2
MH3D_ERR_OOM = 3
MH3D_ERR_CUDA = 4
MH3D_ERR_NONFINITE = 5
MH3D_ERR_NOT_CONVERGED = 6
MH3D_ERR_TIMEOUT = 7
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "OOM", 4: "CUDA", 5: "NONFINITE",
                6: "NOT_CONVERGED", 7: "TIMEOUT"}


class mh3d_geometry(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("voxel_mm", c_double * 3), ("drive_axis", c_int), ("ds_factor", c_int),
                ("ds_offset", c_int), ("pad", c_int * 3), ("k_min", c_int), ("k_max", c_int),
                ("gamma_per_mm", c_double), ("gammaA", c_double), ("transverse_ratio", c_double),
                ("theta", POINTER(c_double)), ("sensitivity_dev", c_void_p)]


class mh3d_solve_opts(ctypes.Structure):
    _fields_ = [("reg_kind", c_int), ("lambda_", c_double), ("alpha", c_double), ("shell", c_int),
                ("solver", c_int), ("rel_tol", c_double), ("max_iter", c_int), ("fixed_iters", c_int),
                ("x0_dev", c_void_p), ("normal_mode", c_int), ("apg_tau", c_double),
                ("lambda_relative", c_int), ("cg_variant", c_int), ("x0_fallback", c_int),
                ("fp32_scalar_div", c_int)]


class mh3d_solve_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("rel_res_recurrence", c_double), ("rel_res_true", c_double),
                ("history", POINTER(c_double)), ("status", c_int), ("x0_rejected", c_int), ("tau", c_double)]


class MH3DError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

EXPORTS = ["mh3d_plan_create", "mh3d_plan_destroy", "mh3d_forward", "mh3d_adjoint", "mh3d_normal", "mh3d_solve",
           "mh3d_solve_host", "mh3d_solve_batched", "mh3d_forward_noalloc", "mh3d_operator_norm2", "mh3d_last_error",
           "mh3d_plan_workspace_bytes", "mh3d_version", "mh3d_plan_autotune", "mh3d_plan_spectra", "mh3d_mhad",
           "mh3d_mhad_warm_start", "mh3d_estimate_phase", "mh3d_general_set_psf", "mh3d_general_forward",
           "mh3d_general_adjoint", "mh3d_dot", "mh3d_solve_batched_warm", "mh3d_general_solve", "mh3d_plan_tuning"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmh3d.so (building it with nvcc if missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libmh3d.so not found at {path}; run paper_2503_13802_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = c_void_p
    lib.mh3d_plan_create.argtypes = [POINTER(mh3d_geometry), P, POINTER(c_void_p)]
    lib.mh3d_plan_destroy.argtypes = [P]
    lib.mh3d_forward.argtypes = [P, P, P, P]
    lib.mh3d_adjoint.argtypes = [P, P, P, P]
    lib.mh3d_normal.argtypes = [P, P, P, POINTER(mh3d_solve_opts), P]
    lib.mh3d_solve.argtypes = [P, P, POINTER(mh3d_solve_opts), P, POINTER(mh3d_solve_info), P]
    lib.mh3d_solve_host.argtypes = [P, P, POINTER(mh3d_solve_opts), P, POINTER(mh3d_solve_info), P]
    lib.mh3d_solve_batched.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p), POINTER(mh3d_solve_opts),
                                       POINTER(c_void_p), POINTER(mh3d_solve_info), P]
    lib.mh3d_operator_norm2.argtypes = [P, POINTER(c_double)]
    lib.mh3d_plan_autotune.argtypes = [P, P, POINTER(c_int)]
    lib.mh3d_plan_spectra.argtypes = [P, P, P, P, P, P]
    lib.mh3d_forward_noalloc.argtypes = [POINTER(mh3d_geometry), P, P, P]
    lib.mh3d_mhad.argtypes = [P, P, c_double, c_int, P, P]
    lib.mh3d_mhad_warm_start.argtypes = [P, P, c_double, P, P, P]
    lib.mh3d_estimate_phase.argtypes = [P, P, c_double, POINTER(c_double), POINTER(c_int), P]
    lib.mh3d_general_set_psf.argtypes = [P, P]
    lib.mh3d_general_forward.argtypes = [P, P, P, P, P]
    lib.mh3d_general_adjoint.argtypes = [P, P, P, P, P]
    lib.mh3d_dot.argtypes = [P, P, P, ctypes.c_longlong, POINTER(c_double), P]
    lib.mh3d_general_solve.argtypes = [P, P, P, POINTER(mh3d_solve_opts), P, POINTER(mh3d_solve_info), P]
    lib.mh3d_plan_tuning.argtypes = [P, ctypes.c_char_p, c_int]
    lib.mh3d_solve_batched_warm.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p), POINTER(mh3d_solve_opts),
                                            POINTER(c_void_p), POINTER(c_void_p), POINTER(mh3d_solve_info), P]
    lib.mh3d_last_error.argtypes = [P]
    lib.mh3d_last_error.restype = c_char_p
    lib.mh3d_plan_workspace_bytes.argtypes = [P]
    lib.mh3d_plan_workspace_bytes.restype = c_ulonglong
    lib.mh3d_version.restype = c_char_p
    for name in EXPORTS:
        if name not in ("mh3d_last_error", "mh3d_plan_workspace_bytes", "mh3d_version"):
            getattr(lib, name).restype = c_int
    _lib = lib
    return lib


def _stream_ptr(stream) -> int:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check(plan, status: int):
    if status not in (MH3D_OK,):
        msg = load().mh3d_last_error(plan).decode() if plan else ""
        raise MH3DError(status, msg)


def _dev_ptr(t, dtype, numel: int, what: str) -> int:
    import torch

    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: expected a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{what}: tensor must be on a CUDA device")
    if t.dtype != dtype:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous tensor of {numel} elements, got {tuple(t.shape)}")
    return t.data_ptr()


class Plan:
    """Owns an mh3d_plan and the tensors it borrows (sensitivity map)."""

    def __init__(self, n: Sequence[int], voxel_mm=(1.0, 1.0, 1.0), ds_factor: int = 1, ds_offset: int = 0,
                 k_min: int = 2, k_max: int = 5, gamma_per_mm: float = 1.387016, gammaA: float = 2.0,
                 transverse_ratio: float = 0.5, theta: Optional[Sequence[float]] = None, sensitivity=None,
                 stream=None, pad: Sequence[int] = (0, 0, 0)):
        """n: the field of view (nx, ny, nz); pad: boundary padding voxels per
        side (px a multiple of ds_factor).  Images and the sensitivity live on
        the padded grid (shape); portraits on the field of view's mesh."""
        import torch

        lib = load()
        self.n = tuple(int(v) for v in n)
        self.pad = tuple(int(v) for v in pad)
        self.K = k_max - k_min + 1
        self.ds_factor = ds_factor
        nx, ny, nz = self.n
        px, py, pz = self.pad
        self.N = (nx + 2 * px) * (ny + 2 * py) * (nz + 2 * pz)
        self.shape = (nz + 2 * pz, ny + 2 * py, nx + 2 * px)
        self.portrait_shape = (self.K, nz, ny, nx // ds_factor)
        self.sensitivity = None
        if sensitivity is not None:
            s = sensitivity if isinstance(sensitivity, torch.Tensor) else torch.as_tensor(sensitivity)
            s = s.to(device="cuda", dtype=torch.float32).contiguous()
            self.sensitivity = s
        g = mh3d_geometry()
        g.n[:] = [nx, ny, nz]
        g.voxel_mm[:] = list(voxel_mm)
        g.drive_axis = 0
        g.ds_factor, g.ds_offset = ds_factor, ds_offset
        g.pad[:] = list(self.pad)
        g.k_min, g.k_max = k_min, k_max
        g.gamma_per_mm, g.gammaA, g.transverse_ratio = gamma_per_mm, gammaA, transverse_ratio
        self._theta = None
        if theta is not None:
            self._theta = (c_double * self.K)(*[float(t) for t in theta])
            g.theta = ctypes.cast(self._theta, POINTER(c_double))
        g.sensitivity_dev = (_dev_ptr(self.sensitivity, torch.float32, self.N, "sensitivity")
                             if self.sensitivity is not None else None)
        h = c_void_p()
        st = lib.mh3d_plan_create(ctypes.byref(g), c_void_p(_stream_ptr(stream)), ctypes.byref(h))
        if st != MH3D_OK:
            raise MH3DError(st, "mh3d_plan_create: " + (lib.mh3d_last_error(None) or b"").decode())
        self.handle = h

    def __del__(self):
        try:
            if getattr(self, "handle", None) and self.handle.value:
                load().mh3d_plan_destroy(self.handle)
                self.handle = c_void_p()
        except Exception:
            pass

    def workspace_bytes(self) -> int:
        return int(load().mh3d_plan_workspace_bytes(self.handle))


def mh3d_forward(plan: Plan, rho, d, stream=None):
    import torch

    lib = load()
    p_rho = _dev_ptr(rho, torch.float32, plan.N, "rho")
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    _check(plan.handle, lib.mh3d_forward(plan.handle, c_void_p(p_rho), c_void_p(p_d), c_void_p(_stream_ptr(stream))))
    return d


def mh3d_adjoint(plan: Plan, d, rho, stream=None):
    import torch

    lib = load()
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    p_rho = _dev_ptr(rho, torch.float32, plan.N, "rho")
    _check(plan.handle, lib.mh3d_adjoint(plan.handle, c_void_p(p_d), c_void_p(p_rho), c_void_p(_stream_ptr(stream))))
    return rho


def mh3d_general_set_psf(plan: Plan, h):
    """PSF samples of the general model (include/mh3d.h): h is a float32
    array of K*3*N values, layout [k][j][z][y][x], at the grid's minimal-image
    offsets (a numpy array or a CPU tensor)."""
    import numpy as np

    lib = load()
    a = np.ascontiguousarray(np.asarray(h, dtype=np.float32))
    if a.size != plan.K * 3 * plan.N:
        raise ValueError(f"h: need {plan.K * 3 * plan.N} float32 values, got {a.size}")
    _check(plan.handle, lib.mh3d_general_set_psf(plan.handle, c_void_p(a.ctypes.data)))


def _bvec_ptr(plan: Plan, bvec) -> Optional[int]:
    import torch

    return None if bvec is None else _dev_ptr(bvec, torch.float32, 3 * plan.N, "bvec")


def mh3d_general_forward(plan: Plan, rho, d, bvec=None, stream=None):
    """d = A rho for the general model; bvec: 3*N float32 on the device, or
    None for b = (1, 0, 0)."""
    import torch

    lib = load()
    p_rho = _dev_ptr(rho, torch.float32, plan.N, "rho")
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    p_b = _bvec_ptr(plan, bvec)
    _check(plan.handle, lib.mh3d_general_forward(plan.handle, c_void_p(p_rho), c_void_p(p_b), c_void_p(p_d),
                                                 c_void_p(_stream_ptr(stream))))
    return d


def mh3d_general_adjoint(plan: Plan, d, out, bvec=None, stream=None):
    """out = A^T d for the general model."""
    import torch

    lib = load()
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    p_o = _dev_ptr(out, torch.float32, plan.N, "out")
    p_b = _bvec_ptr(plan, bvec)
    _check(plan.handle, lib.mh3d_general_adjoint(plan.handle, c_void_p(p_d), c_void_p(p_b), c_void_p(p_o),
                                                 c_void_p(_stream_ptr(stream))))
    return out


def mh3d_general_solve(plan: Plan, d, opts: mh3d_solve_opts, rho, bvec=None, stream=None,
                       allow_not_converged: bool = True):
    """CG on (A^T A + lambda I) rho = A^T d for the general model (absolute
    lambda).  Returns a dict with iters, residuals, status and history."""
    import torch

    lib = load()
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    p_r = _dev_ptr(rho, torch.float32, plan.N, "rho")
    p_b = _bvec_ptr(plan, bvec)
    if opts.x0_dev:
        _dev_ptr(opts._x0_ref, torch.float32, plan.N, "x0")
    info, hist = _info(opts.max_iter + 1)
    st = lib.mh3d_general_solve(plan.handle, c_void_p(p_d), c_void_p(p_b), ctypes.byref(opts), c_void_p(p_r),
                                ctypes.byref(info), c_void_p(_stream_ptr(stream)))
    if st != MH3D_OK and not (allow_not_converged and st == MH3D_ERR_NOT_CONVERGED):
        _check(plan.handle, st)
    return {"iters": info.iters, "rel_res_recurrence": info.rel_res_recurrence, "rel_res_true": info.rel_res_true,
            "status": info.status, "history": [hist[i] for i in range(min(info.iters, opts.max_iter) + 1)]}


def make_opts(lam: float = 1e-3, reg_kind: int = 0, alpha: float = 0.0, shell: int = 2, solver: int = 0,
              rel_tol: float = 1e-4, max_iter: int = 1000, fixed_iters: bool = False, x0=None,
              normal_mode: int = 0, apg_tau: float = 0.0, lam_relative: bool = False,
              cg_variant: int = 0, x0_fallback: bool = False, fp32_scalar_div: bool = False) -> mh3d_solve_opts:
    """lam_relative: lam multiplies ||A||_2^2 (b = 1), see mh3d_operator_norm2.
    fp32_scalar_div: CG's beta and alpha as FP32 quotients instead of FP64."""
    o = mh3d_solve_opts()
    o.reg_kind, o.lambda_, o.alpha, o.shell, o.solver = reg_kind, lam, alpha, shell, solver
    o.rel_tol, o.max_iter, o.fixed_iters = rel_tol, max_iter, int(bool(fixed_iters))
    o.x0_dev = x0.data_ptr() if x0 is not None else None
    o.normal_mode, o.apg_tau = normal_mode, apg_tau
    o.lambda_relative = int(bool(lam_relative))
    o.cg_variant = int(cg_variant)
    o.x0_fallback = int(bool(x0_fallback))
    o.fp32_scalar_div = int(bool(fp32_scalar_div))
    o._x0_ref = x0
    return o


def mh3d_normal(plan: Plan, p, q, opts: mh3d_solve_opts, stream=None):
    import torch

    lib = load()
    pp = _dev_ptr(p, torch.float32, plan.N, "p")
    pq = _dev_ptr(q, torch.float32, plan.N, "q")
    _check(plan.handle, lib.mh3d_normal(plan.handle, c_void_p(pp), c_void_p(pq), ctypes.byref(opts),
                                        c_void_p(_stream_ptr(stream))))
    return q


def _info(history_len: int):
    info = mh3d_solve_info()
    hist = (c_double * history_len)()
    info.history = ctypes.cast(hist, POINTER(c_double))
    return info, hist


def mh3d_solve(plan: Plan, d, opts: mh3d_solve_opts, rho, stream=None, allow_not_converged: bool = True):
    """Returns a dict with iters, residuals, status and the residual history."""
    import torch

    lib = load()
    n_d = plan.K * plan.portrait_shape[1] * plan.portrait_shape[2] * plan.portrait_shape[3]
    p_d = _dev_ptr(d, torch.complex64, n_d, "d")
    p_rho = _dev_ptr(rho, torch.float32, plan.N, "rho")
    if opts.x0_dev:
        _dev_ptr(opts._x0_ref, torch.float32, plan.N, "x0")
    info, hist = _info(opts.max_iter + 1)
    st = lib.mh3d_solve(plan.handle, c_void_p(p_d), ctypes.byref(opts), c_void_p(p_rho), ctypes.byref(info),
                        c_void_p(_stream_ptr(stream)))
    if st != MH3D_OK and not (allow_not_converged and st == MH3D_ERR_NOT_CONVERGED):
        _check(plan.handle, st)
    return {"iters": info.iters, "rel_res_recurrence": info.rel_res_recurrence, "rel_res_true": info.rel_res_true,
            "status": info.status, "x0_rejected": info.x0_rejected, "tau": info.tau,
            "history": [hist[i] for i in range(min(info.iters, opts.max_iter) + 1)]}


def mh3d_dot(plan: Plan, a, b, stream=None) -> float:
    """sum a_i b_i of two float32 CUDA tensors of equal length, as the
    solvers' inner products are computed (float pairs, one FP64 total)."""
    import torch

    lib = load()
    n = a.numel()
    pa = _dev_ptr(a, torch.float32, n, "a")
    pb = _dev_ptr(b, torch.float32, n, "b")
    out = c_double(0.0)
    _check(plan.handle, lib.mh3d_dot(plan.handle, c_void_p(pa), c_void_p(pb), n, ctypes.byref(out),
                                     c_void_p(_stream_ptr(stream))))
    return out.value


def mh3d_solve_host(plan: Plan, d_host, opts: mh3d_solve_opts, rho_host, stream=None):
    """d_host / rho_host: CPU tensors (pinned for speed), complex64 / float32."""
    import torch

    lib = load()
    for t, dt, what in ((d_host, torch.complex64, "d_host"), (rho_host, torch.float32, "rho_host")):
        if t.is_cuda or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"{what}: need a contiguous CPU tensor of {dt}")
    info, hist = _info(opts.max_iter + 1)
    st = lib.mh3d_solve_host(plan.handle, c_void_p(d_host.data_ptr()), ctypes.byref(opts),
                             c_void_p(rho_host.data_ptr()), ctypes.byref(info), c_void_p(_stream_ptr(stream)))
    if st not in (MH3D_OK, MH3D_ERR_NOT_CONVERGED):
        _check(plan.handle, st)
    return {"iters": info.iters, "rel_res_true": info.rel_res_true, "status": info.status}


def mh3d_solve_batched(plans: Sequence[Plan], ds, opts: mh3d_solve_opts, rhos, stream=None, x0s=None):
    """Solves every volume (its own plan, portraits ds[i], image rhos[i]) in
    one call: for CG, one CUDA graph with an independent branch per volume.
    x0s (optional): one warm start per volume (mh3d_solve_batched_warm).
    Returns one info dict per volume."""
    import torch

    lib = load()
    n = len(plans)
    hp = (c_void_p * n)(*[p.handle.value for p in plans])
    dp = (c_void_p * n)()
    rp = (c_void_p * n)()
    xp = (c_void_p * n)()
    for i, (p, d, r) in enumerate(zip(plans, ds, rhos)):
        n_d = p.K * p.portrait_shape[1] * p.portrait_shape[2] * p.portrait_shape[3]
        dp[i] = _dev_ptr(d, torch.complex64, n_d, f"d[{i}]")
        rp[i] = _dev_ptr(r, torch.float32, p.N, f"rho[{i}]")
        if x0s is not None:
            xp[i] = _dev_ptr(x0s[i], torch.float32, p.N, f"x0[{i}]")
    infos = (mh3d_solve_info * n)()
    if x0s is None:
        st = lib.mh3d_solve_batched(hp, n, dp, ctypes.byref(opts), rp, infos, c_void_p(_stream_ptr(stream)))
    else:
        st = lib.mh3d_solve_batched_warm(hp, n, dp, ctypes.byref(opts), xp, rp, infos,
                                         c_void_p(_stream_ptr(stream)))
    if st not in (MH3D_OK, MH3D_ERR_NOT_CONVERGED):
        _check(plans[0].handle if n else None, st)
    return [{"iters": infos[i].iters, "rel_res_recurrence": infos[i].rel_res_recurrence,
             "rel_res_true": infos[i].rel_res_true, "status": infos[i].status,
             "x0_rejected": infos[i].x0_rejected} for i in range(n)]


def mh3d_forward_noalloc(n, rho, d, voxel_mm=(1.0, 1.0, 1.0), ds_factor: int = 1, ds_offset: int = 0,
                         k_min: int = 2, k_max: int = 5, gamma_per_mm: float = 1.387016, gammaA: float = 2.0,
                         transverse_ratio: float = 0.5, theta=None, sensitivity=None, stream=None):
    """d = A rho without a plan and without any device allocation.

    For callers that cannot allocate device memory when they need the
    operator (a fixed memory budget owned by another pool, a frozen
    real-time memory plan): the library keeps the tables and intermediate
    volumes in one fixed device array (grids up to 2,097,152 voxels).  Calls
    share that array, so calls that overlap on the GPU race; issue them on
    one stream.  The first call on a device resolves the array's address.  A
    call on a capturing stream is refused (MH3D_ERR_INVALID_ARG): each call
    uploads its tables from a host buffer freed on return.  `sensitivity`
    must already be a float32 CUDA tensor (this call does not copy it to the
    device).
    """
    import torch

    lib = load()
    nx, ny, nz = (int(v) for v in n)
    K = k_max - k_min + 1
    g = mh3d_geometry()
    g.n[:] = [nx, ny, nz]
    g.voxel_mm[:] = list(voxel_mm)
    g.drive_axis = 0
    g.ds_factor, g.ds_offset = ds_factor, ds_offset
    g.pad[:] = [0, 0, 0]
    g.k_min, g.k_max = k_min, k_max
    g.gamma_per_mm, g.gammaA, g.transverse_ratio = gamma_per_mm, gammaA, transverse_ratio
    th = None
    if theta is not None:
        th = (c_double * K)(*[float(t) for t in theta])
        g.theta = ctypes.cast(th, POINTER(c_double))
    N = nx * ny * nz
    g.sensitivity_dev = _dev_ptr(sensitivity, torch.float32, N, "sensitivity") if sensitivity is not None else None
    p_rho = _dev_ptr(rho, torch.float32, N, "rho")
    p_d = _dev_ptr(d, torch.complex64, K * nz * ny * (nx // ds_factor), "d")
    st = lib.mh3d_forward_noalloc(ctypes.byref(g), c_void_p(p_rho), c_void_p(p_d), c_void_p(_stream_ptr(stream)))
    if st != MH3D_OK:
        raise MH3DError(st, "mh3d_forward_noalloc")
    return d


def mh3d_mhad(plan: Plan, d, lam: float, out, upsample: bool = False, stream=None):
    """MHAD native image of the portraits d (include/mh3d.h): out has
    nz*ny*mx floats (upsample False) or N floats (True)."""
    import torch

    lib = load()
    K, nz, ny, mx = plan.portrait_shape
    p_d = _dev_ptr(d, torch.complex64, K * nz * ny * mx, "d")
    p_o = _dev_ptr(out, torch.float32, plan.N if upsample else nz * ny * mx, "out")
    _check(plan.handle, lib.mh3d_mhad(plan.handle, c_void_p(p_d), c_double(lam), c_int(1 if upsample else 0),
                                      c_void_p(p_o), c_void_p(_stream_ptr(stream))))
    return out


def mh3d_mhad_warm_start(plan: Plan, d, lam: float, x0, alpha=None, stream=None):
    """x0 = alpha * (upsampled MHAD image / b), alpha the least-squares
    scale on the data; alpha (optional) is a float64 device tensor of one
    element receiving it."""
    import torch

    lib = load()
    K, nz, ny, mx = plan.portrait_shape
    p_d = _dev_ptr(d, torch.complex64, K * nz * ny * mx, "d")
    p_x = _dev_ptr(x0, torch.float32, plan.N, "x0")
    p_a = _dev_ptr(alpha, torch.float64, 1, "alpha") if alpha is not None else None
    _check(plan.handle, lib.mh3d_mhad_warm_start(plan.handle, c_void_p(p_d), c_double(lam), c_void_p(p_x),
                                                 c_void_p(p_a), c_void_p(_stream_ptr(stream))))
    return x0


def mh3d_estimate_phase(plan: Plan, d, frac: float = 0.5, stream=None):
    """(theta [K], resolved [K]) estimated from the portraits d (see
    include/mh3d.h): numpy arrays; resolved[k] = 0 where theta_k is known
    modulo pi only."""
    import numpy as np
    import torch

    lib = load()
    K, nz, ny, mx = plan.portrait_shape
    p_d = _dev_ptr(d, torch.complex64, K * nz * ny * mx, "d")
    th = (c_double * K)()
    res = (c_int * K)()
    _check(plan.handle, lib.mh3d_estimate_phase(plan.handle, c_void_p(p_d), c_double(frac), th, res,
                                                c_void_p(_stream_ptr(stream))))
    return np.array(th[:], dtype=np.float64), np.array(res[:], dtype=np.int32)


def mh3d_operator_norm2(plan: Plan) -> float:
    out = c_double()
    _check(plan.handle, load().mh3d_operator_norm2(plan.handle, ctypes.byref(out)))
    return out.value


def mh3d_plan_autotune(plan: Plan, stream=None) -> int:
    """Times the operators' launch variants and keeps the fastest for this
    plan (see mh3d_plan_tuning for the choices); returns the tile width."""
    c = c_int(0)
    _check(plan.handle, load().mh3d_plan_autotune(plan.handle, c_void_p(_stream_ptr(stream)), ctypes.byref(c)))
    return c.value


def mh3d_plan_tuning(plan: Plan) -> dict:
    """The plan's current launch choices (0 = the library's default)."""
    import json

    buf = ctypes.create_string_buffer(512)
    _check(plan.handle, load().mh3d_plan_tuning(plan.handle, buf, 512))
    return json.loads(buf.value.decode())


def mh3d_plan_spectra(plan: Plan, stream=None):
    """(X [K, nx], Y [ny], Z [nz], phase [K]) complex64 device tensors: the
    plan's spectral tables (see include/mh3d.h)."""
    import torch

    nz, ny, nx = plan.shape
    X = torch.empty((plan.K, nx), dtype=torch.complex64, device="cuda")
    Y = torch.empty(ny, dtype=torch.complex64, device="cuda")
    Z = torch.empty(nz, dtype=torch.complex64, device="cuda")
    ph = torch.empty(plan.K, dtype=torch.complex64, device="cuda")
    _check(plan.handle, load().mh3d_plan_spectra(plan.handle, c_void_p(X.data_ptr()), c_void_p(Y.data_ptr()),
                                                 c_void_p(Z.data_ptr()), c_void_p(ph.data_ptr()),
                                                 c_void_p(_stream_ptr(stream))))
    return X, Y, Z, ph


def mh3d_version() -> str:
    return load().mh3d_version().decode()
