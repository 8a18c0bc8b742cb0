"""The forward operator for callers that cannot allocate device memory.

mh3d_forward_noalloc needs no plan: a caller that runs under a fixed
device-memory budget (another framework's pool, a frozen real-time memory
plan) cannot call cudaMalloc, so it cannot create a plan either.  The entry
point keeps its tables and intermediate volumes in one fixed device array
inside the library.  These tests call it through the C ABI twice in a row,
with different geometries and inputs, and compare each result with
mh3d_forward on a plan (the existing entry point) at the tolerance of the
other operator tests.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from tests._cases import gpu_plan, params, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


def _case(p, seed, with_sens):
    nx, ny, nz = p["n"]
    K = p["kmax"] - p["kmin"] + 1
    rho = torch.as_tensor(W.random_volume((nz, ny, nx), seed), dtype=torch.float32, device="cuda").contiguous()
    sens = None
    if with_sens:
        sens = torch.as_tensor(W.sensitivity((nx, ny, nz)), dtype=torch.float32, device="cuda").contiguous()
    d = torch.empty((K, nz, ny, nx // p["s"]), dtype=torch.complex64, device="cuda")
    return rho, sens, d


def _noalloc(p, rho, sens, d):
    from paper_2503_13802_gb300 import mh3d_forward_noalloc

    return mh3d_forward_noalloc(p["n"], rho, d, voxel_mm=p["voxel"], ds_factor=p["s"], ds_offset=p["r"],
                                k_min=p["kmin"], k_max=p["kmax"], gamma_per_mm=p["gamma"], gammaA=p["gammaA"],
                                transverse_ratio=p["tratio"], theta=p["theta"], sensitivity=sens)


def _planned(p, rho, sens):
    from paper_2503_13802_gb300 import mh3d_forward

    plan = gpu_plan(p, sens)
    nx, ny, nz = p["n"]
    K = p["kmax"] - p["kmin"] + 1
    d = torch.empty((K, nz, ny, nx // p["s"]), dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, rho, d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


def test_noalloc_forward_matches_planned_forward_twice():
    cases = [
        (params((128, 128, 64), s=2, kmin=2, kmax=9), 11, True),
        (params((96, 24, 18), s=3, r=1, kmin=3, kmax=6, theta=[0.4, -1.0, 2.2, 0.1]), 12, False),
    ]
    for p, seed, with_sens in cases:          # two calls in a row, different geometry and data
        rho, sens, d = _case(p, seed, with_sens)
        _noalloc(p, rho, sens, d)
        torch.cuda.synchronize()
        got = d.cpu().numpy()
        ref = _planned(p, rho, sens)
        assert np.isfinite(got).all()
        assert rel_l2(got, ref) <= TOL, rel_l2(got, ref)


def test_noalloc_forward_rejects_grids_beyond_scratch():
    from paper_2503_13802_gb300 import MH3DError

    p = params((256, 128, 128), s=1, kmin=2, kmax=3)      # 4,194,304 voxels > 2,097,152
    nx, ny, nz = p["n"]
    rho = torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda")
    d = torch.empty((2, nz, ny, nx), dtype=torch.complex64, device="cuda")
    with pytest.raises(MH3DError) as e:
        _noalloc(p, rho, None, d)
    assert "UNSUPPORTED_SIZE" in str(e.value)
