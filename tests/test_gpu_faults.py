"""Failure handling without a GPU fault, trap or hang.

* Injected allocation failures (host-side hook MH3D_DEBUG_FAIL_ALLOC=k: the
  k-th device or pinned allocation of a plan creation fails): every
  clean-up path returns MH3D_ERR_OOM with a message, frees what it had
  taken, and the library stays usable.
* A bounded device wait that runs out (MH3D_DEBUG_WAIT_TIMEOUT=1: the
  transverse pass's tile barrier expects 16 bytes that no copy delivers):
  the CTAs give up after the %globaltimer limit, the solve stops on the
  device and returns MH3D_ERR_TIMEOUT, and the context stays usable.
* Guard bands: outputs written into the middle of larger buffers leave the
  bands around them untouched (out-of-bounds writes would show).
"""
import time

import numpy as np
import pytest

import workloads as W
from tests._cases import gpu_plan, oracle_geom, params, sens_map

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_injected_allocation_failures_clean_up(monkeypatch):
    from paper_2503_13802_gb300 import MH3DError, mh3d_forward

    p = params((32, 32, 32), s=2, kmin=2, kmax=5)
    g = oracle_geom(p)
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    for k in range(1, 12):
        monkeypatch.setenv("MH3D_DEBUG_FAIL_ALLOC", str(k))
        try:
            plan = gpu_plan(p, sens_map(p))
        except MH3DError as e:
            assert "OOM" in str(e) and len(str(e)) > 6, str(e)
            failed += 1
            continue
        del plan
        break
    assert failed >= 4, failed          # tables, workspace, flags, pinned flags, pinned scalars
    monkeypatch.delenv("MH3D_DEBUG_FAIL_ALLOC")
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)   # nothing of size leaked
    plan = gpu_plan(p, sens_map(p))
    d = torch.empty(g.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, torch.ones(g.shape, device="cuda"), d)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(d)).all()


def test_bounded_wait_timeout_is_reported(monkeypatch):
    from paper_2503_13802_gb300 import MH3DError, make_opts, mh3d_solve

    p = params((32, 32, 32), s=1, kmin=2, kmax=5)
    g = oracle_geom(p)
    d = torch.as_tensor(W.random_portraits(g.portrait_shape, 2).astype(np.complex64), device="cuda")
    x = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    monkeypatch.setenv("MH3D_DEBUG_WAIT_TIMEOUT", "1")
    plan = gpu_plan(p, None)
    t0 = time.time()
    with pytest.raises(MH3DError) as e:
        mh3d_solve(plan, d, make_opts(lam=1e-3, lam_relative=True, max_iter=50), x)
    assert "TIMEOUT" in str(e.value)
    assert time.time() - t0 < 30.0
    monkeypatch.delenv("MH3D_DEBUG_WAIT_TIMEOUT")
    plan2 = gpu_plan(p, None)
    info = mh3d_solve(plan2, d, make_opts(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=400), x)
    assert info["status"] == 0


def _banded(n, dtype, sentinel, band=8192):
    buf = torch.full((n + 2 * band,), sentinel, dtype=dtype, device="cuda")
    return buf, buf[band:band + n], band


def _bands_intact(buf, band, sentinel):
    head, tail = buf[:band], buf[-band:]
    return bool((head == sentinel).all()) and bool((tail == sentinel).all())


@pytest.mark.parametrize("name", ["ds2_theta", "spec96", "odd_nx27", "warp_ragged27", "zx128"])
def test_outputs_stay_inside_their_buffers(name):
    from tests._cases import OP_CASES
    from paper_2503_13802_gb300 import make_opts, mh3d_adjoint, mh3d_forward, mh3d_normal, mh3d_solve

    p = OP_CASES[name]
    g = oracle_geom(p)
    plan = gpu_plan(p, sens_map(p))
    N = int(np.prod(g.shape))
    KM = int(np.prod(g.portrait_shape))
    rho = torch.as_tensor(W.random_volume(g.shape, 1), dtype=torch.float32, device="cuda").contiguous()
    sc = complex(12345.0, -12345.0)
    dbuf, d, band = _banded(KM, torch.complex64, sc)
    mh3d_forward(plan, rho, d.view(g.portrait_shape))
    torch.cuda.synchronize()
    assert _bands_intact(dbuf, band, sc)
    rbuf, r, band = _banded(N, torch.float32, 12345.0)
    mh3d_adjoint(plan, d.view(g.portrait_shape), r.view(g.shape))
    torch.cuda.synchronize()
    assert _bands_intact(rbuf, band, 12345.0)
    qbuf, q, band = _banded(N, torch.float32, 12345.0)
    mh3d_normal(plan, rho, q.view(g.shape), make_opts(lam=1e-2))
    torch.cuda.synchronize()
    assert _bands_intact(qbuf, band, 12345.0)
    xbuf, xx, band = _banded(N, torch.float32, 12345.0)
    mh3d_solve(plan, d.view(g.portrait_shape), make_opts(lam=1e-2, lam_relative=True, max_iter=20), xx.view(g.shape))
    assert _bands_intact(xbuf, band, 12345.0)


def test_noalloc_forward_refuses_stream_capture():
    """mh3d_forward_noalloc uploads its tables from a host buffer freed when
    the call returns, so a captured call would replay a copy from freed
    memory: on a capturing stream it returns MH3D_ERR_INVALID_ARG and issues
    nothing, and the capture itself ends normally."""
    from paper_2503_13802_gb300 import MH3DError, mh3d_forward_noalloc

    nx, ny, nz = 32, 16, 8
    rho = torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda")
    d = torch.empty((2, nz, ny, nx), dtype=torch.complex64, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(graph, stream=s):
        d.zero_()
        try:
            mh3d_forward_noalloc((nx, ny, nz), rho, d, k_min=2, k_max=3, stream=s)
        except MH3DError as e:
            err = e
    assert err is not None and "INVALID_ARG" in str(err)
    graph.replay()
    torch.cuda.synchronize()
    assert float(torch.abs(d).max()) == 0.0
