"""GB300-native MH3D (arXiv 2503.13802): the multi-harmonic portrait forward
operator, its adjoint and the regularised least-squares solve, as
hand-written sm_103a CUDA behind the C ABI in include/mh3d.h.

This package is the thin Python side: ``build`` compiles libmh3d.so in-tree
with nvcc, ``mh3d`` marshals torch tensors into the C calls.  There is no
CPU fallback.
"""
from . import build
from .mh3d import (MH3DError, Plan, load, make_opts, mh3d_adjoint, mh3d_dot, mh3d_estimate_phase, mh3d_forward, mh3d_mhad,
                   mh3d_general_adjoint, mh3d_general_forward, mh3d_general_set_psf, mh3d_general_solve, mh3d_mhad_warm_start,
                   mh3d_normal, mh3d_solve, mh3d_forward_noalloc, mh3d_operator_norm2, mh3d_plan_autotune, mh3d_plan_tuning,
                   mh3d_plan_spectra, mh3d_solve_batched, mh3d_solve_host, mh3d_version)

__all__ = ["build", "MH3DError", "Plan", "load", "make_opts", "mh3d_adjoint", "mh3d_dot", "mh3d_estimate_phase", "mh3d_forward",
           "mh3d_general_adjoint", "mh3d_general_forward", "mh3d_general_set_psf", "mh3d_general_solve", "mh3d_mhad",
           "mh3d_mhad_warm_start", "mh3d_normal", "mh3d_forward_noalloc", "mh3d_operator_norm2", "mh3d_plan_autotune", "mh3d_plan_tuning",
           "mh3d_plan_spectra", "mh3d_solve", "mh3d_solve_batched", "mh3d_solve_host", "mh3d_version"]
