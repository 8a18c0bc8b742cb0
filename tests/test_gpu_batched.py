"""Batched CG (mh3d_solve_batched): one CUDA graph with an independent branch
per volume, volumes of different sizes.

* Every volume of a batch must equal, bit for bit, the same volume solved
  alone by mh3d_solve: the branches launch the same kernels with the same
  launch shapes, and every reduction has a fixed order.  (In a batch the
  fused T_z + drive-axis normal pass loads its epilogue operands late, to
  keep its occupancy beside the other volumes' kernels; alone it loads
  them before the transform.  The arithmetic is the same; the 64x32x64
  volume takes that pass.)
* One volume is compared with the FP64 oracle's CG at a fixed iteration
  count (rel. L2 <= 1e-4, as for single solves).
* At the full size classes of the 64-volume workload (64^3, 96x96x64,
  128x128x64, 192x192x96; K = 8, s = 2, Gaussian b, 25 dB), each volume's
  true residual meets the stopping rule.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import gpu_plan, oracle_geom, params, rel_l2, sens_map

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SMALL = [
    params((64, 64, 32), s=2, kmin=2, kmax=9),
    params((32, 32, 32), s=1, kmin=2, kmax=5),
    params((96, 96, 64), s=2, kmin=2, kmax=9),
    params((64, 64, 32), s=2, kmin=2, kmax=9),
    params((48, 32, 32), s=2, kmin=2, kmax=5),    # drive length 48: runtime-general X kernels
    params((64, 32, 64), s=2, kmin=2, kmax=9),    # the fused cluster normal pass (n_x = 64, n_z = 64)
]


def _case(p, seed, snr_db=25.0):
    """Oracle-made noisy portraits of a seeded phantom (small grids)."""
    g = oracle_geom(p)
    b = sens_map(p)
    rho = W.phantom(p["n"], p["voxel"], seed, 12, 1)
    clean = oracle.forward(g, rho, b)
    sig2 = np.sum(np.abs(clean) ** 2) / (clean.size * 10 ** (snr_db / 10))
    d = clean + math.sqrt(sig2) * W.unit_complex_noise(clean.shape, seed)
    return g, b, d


def _dev(a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype).contiguous()


def _opts(**kw):
    from paper_2503_13802_gb300 import make_opts

    base = dict(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=400)
    base.update(kw)
    return make_opts(**base)


def _small_batch(seed0=500):
    plans, ds, cases = [], [], []
    for i, p in enumerate(SMALL):
        g, b, d = _case(p, seed0 + i)
        plans.append(gpu_plan(p, b))
        ds.append(_dev(d, torch.complex64))
        cases.append((g, b, d))
    return plans, ds, cases


def _solve_each(plans, ds, opts):
    from paper_2503_13802_gb300 import mh3d_solve

    out = []
    for pl, d in zip(plans, ds):
        x = torch.empty(pl.shape, dtype=torch.float32, device="cuda")
        info = mh3d_solve(pl, d, opts, x)
        out.append((x.cpu().numpy(), info))
    return out


def _solve_batch(plans, ds, opts):
    from paper_2503_13802_gb300 import mh3d_solve_batched

    xs = [torch.empty(pl.shape, dtype=torch.float32, device="cuda") for pl in plans]
    infos = mh3d_solve_batched(plans, ds, opts, xs)
    return [x.cpu().numpy() for x in xs], infos


@pytest.mark.parametrize("variant", [0, 1])
def test_batched_equals_single_solves_bit_for_bit(variant):
    plans, ds, _ = _small_batch()
    opts = _opts(cg_variant=variant)
    alone = _solve_each(plans, ds, opts)
    xs, infos = _solve_batch(plans, ds, opts)
    for v, ((xa, ia), xb, ib) in enumerate(zip(alone, xs, infos)):
        assert ib["iters"] == ia["iters"], (v, ib, ia)
        assert ib["status"] == ia["status"] == 0, (v, ib, ia)
        assert np.array_equal(xa, xb), (v, float(np.abs(xa - xb).max()))
        assert ib["rel_res_true"] == ia["rel_res_true"]
        assert ib["rel_res_true"] <= 1.5e-4, (v, ib)


def test_batched_graph_reuse_with_new_data():
    """A second call with other portraits (other device pointers) reuses the
    cached graph: the portraits are staged into the plans' own buffers."""
    plans, ds, _ = _small_batch(600)
    opts = _opts()
    _solve_batch(plans, ds, opts)
    ds2 = [torch.flip(d, dims=[1]).contiguous() for d in ds]
    xs, infos = _solve_batch(plans, ds2, opts)
    alone = _solve_each(plans, ds2, opts)
    for (xa, ia), xb, ib in zip(alone, xs, infos):
        assert ib["iters"] == ia["iters"]
        assert np.array_equal(xa, xb)


def test_batched_volume_matches_oracle_at_fixed_iterations():
    plans, ds, cases = _small_batch(700)
    opts = _opts(fixed_iters=1, max_iter=30)
    xs, infos = _solve_batch(plans, ds, opts)
    v = 1                                           # 32^3, K = 4, s = 1
    g, b, d = cases[v]
    xo, it, _ = oracle.cg(g, d, b, oracle.SolveOpts(lam=1e-3, lam_relative=True, rel_tol=0.0, max_iter=30))
    assert infos[v]["iters"] == 30 and it == 30
    assert rel_l2(xs[v], xo) <= 1e-4, rel_l2(xs[v], xo)


def test_batched_rejects_warm_start_and_repeated_plans():
    from paper_2503_13802_gb300 import MH3DError, make_opts, mh3d_solve_batched

    plans, ds, _ = _small_batch(800)
    xs = [torch.empty(pl.shape, dtype=torch.float32, device="cuda") for pl in plans]
    with pytest.raises(MH3DError) as e:
        mh3d_solve_batched([plans[0], plans[0]], [ds[0], ds[0]], _opts(), [xs[0], xs[0]])
    assert "INVALID_ARG" in str(e.value)
    x0 = torch.zeros(plans[0].shape, dtype=torch.float32, device="cuda")
    with pytest.raises(MH3DError) as e:
        mh3d_solve_batched(plans[:1], ds[:1], make_opts(lam=1e-3, lam_relative=True, x0=x0), xs[:1])
    assert "INVALID_ARG" in str(e.value)


def test_batched_warm_starts_equal_single_warm_solves():
    """mh3d_solve_batched_warm: a warm start per volume (here 0.8 times a
    zero-start solution, and one deliberately bad guess that the fallback
    rejects) gives, for every volume, the single warm-started solve bit for
    bit, with fewer iterations than the zero start where the guess is good."""
    from paper_2503_13802_gb300 import mh3d_solve, mh3d_solve_batched

    plans, ds, _ = _small_batch(900)
    opts = _opts(x0_fallback=True)
    zero = _solve_each(plans, ds, opts)
    x0s = [_dev(0.8 * xz, torch.float32) for xz, _ in zero]
    x0s[1] = _dev(1e3 * W.random_volume(plans[1].shape, 5), torch.float32)   # rejected by the fallback
    xs = [torch.empty(pl.shape, dtype=torch.float32, device="cuda") for pl in plans]
    infos = mh3d_solve_batched(plans, ds, opts, xs, x0s=x0s)
    for v, (pl, d, x0) in enumerate(zip(plans, ds, x0s)):
        from paper_2503_13802_gb300 import make_opts

        xa = torch.empty(pl.shape, dtype=torch.float32, device="cuda")
        ia = mh3d_solve(pl, d, make_opts(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=400, x0=x0,
                                         x0_fallback=True), xa)
        assert infos[v]["iters"] == ia["iters"] and infos[v]["x0_rejected"] == ia["x0_rejected"], (v, infos[v], ia)
        assert torch.equal(xs[v], xa), v
        if v == 1:
            assert infos[v]["x0_rejected"] == 1 and infos[v]["iters"] == zero[v][1]["iters"]
        else:
            assert infos[v]["x0_rejected"] == 0 and infos[v]["iters"] < zero[v][1]["iters"], (v, infos[v])


def test_batched_full_size_classes_residual_property():
    """Two volumes of each size class of the 64-volume workload, portraits
    made by the FP64 oracle: every volume reaches rel. residual 1e-4 by its
    true residual, which the oracle evaluates for the GPU solution in FP64
    (||A^T d - (A^T A + lambda I) x|| / ||A^T d|| with the oracle's own
    ||A||_2^2 for the relative lambda), and one of each class equals its
    single solve bit for bit."""
    wl = W.WORKLOADS["mh_128x128x64_k8_s2"]
    plans, ds, cases = [], [], []
    for i, n in enumerate([c for c in W.BATCH_SIZE_CLASSES for _ in range(2)]):
        p = params(n, s=2, kmin=2, kmax=9)
        g = oracle_geom(p)
        b = sens_map(p)
        tables = oracle.psf_tables(g)
        rho = W.phantom(n, (1.0, 1.0, 1.0), 1000 + i, wl.n_blobs, wl.n_lines)
        clean = oracle.forward(g, rho, b, tables)
        sig2 = np.sum(np.abs(clean) ** 2) / (clean.size * 10 ** (wl.snr_db / 10))
        d = clean + math.sqrt(sig2) * W.unit_complex_noise(clean.shape, 1000 + i)
        plans.append(gpu_plan(p, b))
        ds.append(_dev(d, torch.complex64))
        cases.append((g, b, tables, d))
    opts = _opts(max_iter=wl.max_iter)
    xs, infos = _solve_batch(plans, ds, opts)
    for v, (inf, (g, b, tables, d)) in enumerate(zip(infos, cases)):
        assert inf["status"] == 0, (v, inf)
        o = oracle.SolveOpts(lam=1e-3, lam_relative=True)
        rhs = oracle.adjoint(g, d, b, tables)
        res = rhs - oracle.normal_apply(g, xs[v].astype(np.float64), b, o, tables)
        rel = float(np.linalg.norm(res) / np.linalg.norm(rhs))
        assert rel <= 1.5e-4, (v, g.n, rel, inf)
    alone = _solve_each(plans[::2], ds[::2], opts)
    for (xa, ia), xb, ib in zip(alone, xs[::2], infos[::2]):
        assert ia["iters"] == ib["iters"]
        assert np.array_equal(xa, xb)
