"""Shared case builders for the parity tests: one parameter dict builds both
the oracle geometry and the GPU plan, so both sides see the same model."""
import numpy as np

import oracle
import workloads as W


def params(n, s=1, r=0, kmin=2, kmax=5, theta=None, voxel=(1.0, 1.0, 1.0), gamma=1.387016, gammaA=2.0,
           tratio=0.5):
    return dict(n=tuple(n), s=s, r=r, kmin=kmin, kmax=kmax, theta=theta, voxel=tuple(voxel), gamma=gamma,
                gammaA=gammaA, tratio=tratio)


def oracle_geom(p):
    return oracle.Geometry(n=p["n"], voxel_mm=p["voxel"], ds_factor=p["s"], ds_offset=p["r"], k_min=p["kmin"],
                           k_max=p["kmax"], gamma_per_mm=p["gamma"], gammaA=p["gammaA"],
                           transverse_ratio=p["tratio"], theta=p["theta"])


def gpu_plan(p, sens=None):
    from paper_2503_13802_gb300 import Plan

    return Plan(p["n"], voxel_mm=p["voxel"], ds_factor=p["s"], ds_offset=p["r"], k_min=p["kmin"], k_max=p["kmax"],
                gamma_per_mm=p["gamma"], gammaA=p["gammaA"], transverse_ratio=p["tratio"], theta=p["theta"],
                sensitivity=sens)


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def sens_map(p, kind="gaussian"):
    nx, ny, nz = p["n"]
    return W.sensitivity((nx, ny, nz), p["voxel"], kind=kind)


# Operator parity cases: small enough for the FP64 oracle in seconds, spanning
# several CTA tiles and ragged tails (row counts not a multiple of the
# row-pair tile, column counts not a multiple of the T-pass tile), every
# radix (2, 3, 4, 8), odd nx (scalar path), degenerate axes of length 1,
# downsampling with offsets and nonzero phases.
OP_CASES = {
    "cube32_k4": params((32, 32, 32), kmin=2, kmax=5),
    "ds2_theta": params((64, 24, 18), s=2, r=1, kmin=2, kmax=9, theta=list(np.linspace(-2.5, 2.0, 8))),
    "ds3_radix3": params((96, 12, 9), s=3, r=2, kmin=3, kmax=6, theta=[0.3, -0.7, 1.1, 2.9]),
    "odd_nx27": params((27, 6, 16), s=3, r=0, kmin=2, kmax=4, theta=[0.5, 0.25, -1.0]),
    "line_1d": params((128, 1, 1), s=2, kmin=2, kmax=9),
    "plane_2d": params((48, 36, 1), s=1, kmin=2, kmax=3, voxel=(0.5, 1.5, 1.0)),
    "tall_z": params((8, 3, 192), s=4, r=3, kmin=2, kmax=3),
    "long_x256": params((256, 4, 6), s=1, kmin=2, kmax=17, gammaA=1.0),
    # the specialised lengths of the batched size classes (96 and 192 on
    # every axis kind: drive with s = 2, transverse y and z)
    "spec96": params((96, 96, 32), s=2, kmin=2, kmax=9),
    "spec192": params((192, 192, 16), s=2, kmin=2, kmax=5, theta=[0.4, -0.9, 1.7, 2.2]),
    "spec192_z": params((64, 32, 192), s=2, kmin=2, kmax=5),
    # (nx, nz) pairs of the fused T_z + normal pass (one y-slab per cluster of
    # two CTAs), with few y-slabs so the oracle stays fast
    "zx128": params((128, 6, 64), s=2, kmin=2, kmax=9, theta=[0.2, -0.4, 0.9, 1.3, -2.0, 2.6, 0.0, -1.1]),
    "zx64": params((64, 4, 64), s=2, kmin=2, kmax=5),
    "zx96": params((96, 3, 64), s=2, r=1, kmin=2, kmax=9),
    "zx192": params((192, 2, 96), s=2, kmin=2, kmax=5),      # not fused (separate passes)
    # an odd harmonic count on the specialised drive-axis passes (the
    # adjoint's last round of two harmonics holds one)
    "oddk5": params((128, 6, 32), s=2, kmin=2, kmax=6, theta=[0.3, -1.2, 2.2, 0.7, -0.4]),
    # the warp-centric drive-axis passes (n_x = 128, s = 2): an odd row count
    # that leaves the last warp's last pencil with one row (27 rows), and the
    # most harmonics a plan takes (31)
    "warp_ragged27": params((128, 3, 9), s=2, r=1, kmin=2, kmax=4, theta=[0.9, -2.1, 0.4]),
    "warp_k31": params((128, 4, 4), s=2, kmin=2, kmax=32, gammaA=1.0),
}
