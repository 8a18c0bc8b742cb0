"""The learned warm start end to end on a small grid (32 x 32 x 32, K = 4,
s = 1): training lowers the loss, CG from the learned x0 meets the stopping
rule and reaches the same solution as the zero start, and the device-side
fallback leaves no solve worse off than the zero start."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N = (32, 32, 32)


def _setup(n_train=8, seed0=10000):
    from paper_2503_13802_gb300 import Plan, make_opts, mh3d_forward, mh3d_solve
    from paper_2503_13802_gb300.warmstart import WarmStart

    b = W.sensitivity(N, (1.0, 1.0, 1.0), kind="gaussian")
    plan = Plan(N, ds_factor=1, k_min=2, k_max=5, sensitivity=b)
    opts = make_opts(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500)

    def portraits(seed):
        rho, snr = W.learned_case(N, (1.0, 1.0, 1.0), seed)
        d = torch.empty(plan.portrait_shape, dtype=torch.complex64, device="cuda")
        mh3d_forward(plan, torch.as_tensor(rho, dtype=torch.float32, device="cuda").contiguous(), d)
        sig2 = float(torch.sum(torch.abs(d.to(torch.complex128)) ** 2)) / (d.numel() * 10 ** (snr / 10))
        g = torch.Generator(device="cuda").manual_seed(seed)
        return (d + math.sqrt(sig2) * torch.randn(d.shape, generator=g, dtype=torch.complex64,
                                                  device="cuda")).contiguous()

    ws = WarmStart(plan, channels=(8, 16, 32))
    ws.init_params(3)
    rhs, tgt = [], []
    x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    for sd in range(seed0, seed0 + n_train):
        d = portraits(sd)
        rhs.append(ws.back_projection(d, torch.empty_like(x)))
        info = mh3d_solve(plan, d, opts, x)
        assert info["status"] == 0
        tgt.append(x.clone())
    return plan, opts, ws, portraits, rhs, tgt


def test_training_lowers_the_loss_and_warm_start_converges():
    from paper_2503_13802_gb300 import mh3d_solve

    plan, opts, ws, portraits, rhs, tgt = _setup()
    before = np.mean([ws.loss(r, t) for r, t in zip(rhs, tgt)])
    hist = ws.fit(rhs, tgt, epochs=25, lr_max=2e-3, lr_min=2e-5, seed=4)
    after = np.mean([ws.loss(r, t) for r, t in zip(rhs, tgt)])
    assert after < 0.5 * before, (before, after, hist[-3:])
    d = portraits(20000)
    x0 = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    xw = torch.empty_like(x0)
    i0 = mh3d_solve(plan, d, opts, x0)
    iw = ws.solve(d, xw, lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500)
    assert iw["status"] == 0 and iw["rel_res_true"] <= 1.5e-4, iw
    diff = float(torch.linalg.vector_norm(xw - x0) / torch.linalg.vector_norm(x0))
    # Both iterates have residuals <= 1e-4 ||A^T d|| of the same SPD system,
    # whose condition number with lambda = 1e-3 ||A||^2 is at most 1e3: they
    # differ by at most about 2e-1 relative, far less in practice.
    assert diff <= 5e-2, diff


def test_untrained_guess_is_rejected_or_helps():
    """An untrained network gives an arbitrary guess; with the fallback the
    solve never takes more iterations than the zero start by more than the
    set-up of one iteration."""
    from paper_2503_13802_gb300 import mh3d_solve

    plan, opts, ws, portraits, _, _ = _setup(n_train=0)
    d = portraits(20001)
    x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    i0 = mh3d_solve(plan, d, opts, x)
    iw = ws.solve(d, x, lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500)
    assert iw["status"] == 0
    if iw["x0_rejected"]:
        assert iw["iters"] == i0["iters"]
    else:
        assert iw["history"][0] < 1.0


def test_save_and_load_reproduce_the_prediction(tmp_path):
    from paper_2503_13802_gb300.warmstart import WarmStart

    plan, opts, ws, portraits, rhs, tgt = _setup(n_train=2)
    ws.fit(rhs, tgt, epochs=2, seed=1)
    d = portraits(20002)
    a = ws.predict(d).clone()
    path = str(tmp_path / "ws.npz")
    ws.save(path)
    ws2 = WarmStart(plan, channels=ws.channels)
    ws2.load(path)
    b = ws2.predict(d)
    assert torch.equal(a, b)


def test_trained_network_gain_in_iterations_on_held_out_volumes():
    """What the trained network gains over the zero start, in CG iterations
    to the same stopping rule (rel. residual 1e-4), on four held-out volumes
    (seeds 20010..20013).  The learned x0 starts below the zero start's
    residual on every volume, but here that buys no iterations: the
    measured counts were 61, 53, 48, 51 from x0 against 60, 52, 47, 48 from
    zero (a 3 % loss), because the error the guess leaves lies in the slowly
    converging directions CG spends its iterations on.  The test records
    the counts and bounds the loss at 10 %; bench.py --learned reports the
    same trade on the 128x128x64 workload (4.8 % fewer iterations, but
    slower once the network's inference is counted)."""
    from paper_2503_13802_gb300 import mh3d_solve

    plan, opts, ws, portraits, rhs, tgt = _setup(n_train=8)
    ws.fit(rhs, tgt, epochs=25, lr_max=2e-3, lr_min=2e-5, seed=4)
    x = torch.empty(plan.shape, dtype=torch.float32, device="cuda")
    zero, warm, r0 = [], [], []
    for sd in range(20010, 20014):
        d = portraits(sd)
        i0 = mh3d_solve(plan, d, opts, x)
        iw = ws.solve(d, x, lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500)
        assert i0["status"] == 0 and iw["status"] == 0, (i0, iw)
        zero.append(i0["iters"])
        warm.append(iw["iters"])
        r0.append(iw["history"][0])
    print(f"zero-start iterations {zero}, warm-start {warm}, initial rel. residual of x0 {np.round(r0, 3).tolist()}")
    assert max(r0) < 1.0, r0
    assert np.mean(warm) <= 1.10 * np.mean(zero), (warm, zero)
