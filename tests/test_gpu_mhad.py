"""The MHAD native image (App. D, Eq. mhadM) and the warm start built on it,
through the C ABI (mh3d_mhad, mh3d_mhad_warm_start), against the FP64 oracle
(oracle.mhad on the de-phased portraits Re(e^{-i theta_k} d_k)).

Error bar.  The image is a per-bin filter of FP32 transforms of length mx,
summed over harmonics, so its error is the round-off of one transform pair
scaled by the filter's gain (with unitary-normalised transforms the map
D_k -> image has norm max_m |W_k(m)|):
    ||err|| <= 4 eps (log2 mx + 3) sum_k max_m |W_k(m)| ||D_k||,   eps = 2^-24,
W_k(m) = conj(Fhat(m)^{k-1}) / (c_k (sum_j |Fhat(m)^{j-1}|^2 + lambda)),
Fhat(m) = 2 i sin(2 pi m / mx), computed here in FP64.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import OP_CASES, gpu_plan, oracle_geom, params, rel_l2, sens_map

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24

CASES = {
    "cube32_k4": (OP_CASES["cube32_k4"], 1e-2),        # s = 1, mx = 32: specialised pass
    "ds2_theta": (OP_CASES["ds2_theta"], 1e-2),        # s = 2, offset 1, 432 rows (ragged tile)
    "ds3_radix3": (OP_CASES["ds3_radix3"], 1e-3),      # k_min = 3
    "odd_nx27": (OP_CASES["odd_nx27"], 1e-2),          # mx = 9: odd, no Nyquist bin, general pass
    "line_1d": (OP_CASES["line_1d"], 1e-4),            # one row
    "long_x256": (OP_CASES["long_x256"], 1e-2),        # K = 16, mx = 256
    "spec192": (OP_CASES["spec192"], 1e-2),            # mx = 96
}


def _dephased(g, d):
    th = g.theta_array()
    return [np.real(np.exp(-1j * th[j]) * d[j]) for j in range(g.K)]


def _gain(g, mx, lam):
    m = np.arange(mx)
    fh = 2j * np.sin(2 * np.pi * m / mx)
    pw = [fh ** (k - 1) for k in range(g.k_min, g.k_max + 1)]
    den = lam + sum(np.abs(p) ** 2 for p in pw)
    return [float(np.max(np.abs(p) / (oracle.ck(k, g.gammaA) * den)))
            for k, p in zip(range(g.k_min, g.k_max + 1), pw)]


def _bound(g, D, lam):
    mx = D[0].shape[-1]
    gains = _gain(g, mx, lam)
    return 4 * EPS32 * (math.log2(mx) + 3) * sum(gk * np.linalg.norm(Dk) for gk, Dk in zip(gains, D))


def _portraits(g, seed):
    """complex64 portraits; the oracle sees the same rounded values."""
    d64 = W.random_portraits(g.portrait_shape, seed).astype(np.complex64)
    return d64, d64.astype(np.complex128)


def _mhad_gpu(plan, d64, lam, upsample):
    from paper_2503_13802_gb300 import mh3d_mhad

    K, nz, ny, mx = plan.portrait_shape
    out = torch.empty(plan.N if upsample else nz * ny * mx, dtype=torch.float32, device="cuda")
    mh3d_mhad(plan, torch.as_tensor(d64).cuda(), lam, out, upsample=upsample)
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_mhad_image_matches_oracle(name):
    p, lam = CASES[name]
    g = oracle_geom(p)
    plan = gpu_plan(p)
    d64, d = _portraits(g, 300 + len(name))
    D = _dephased(g, d)
    ref = oracle.mhad(D, [oracle.ck(k, g.gammaA) for k in range(g.k_min, g.k_max + 1)], lam, axis=-1,
                      k_min=g.k_min)
    got = _mhad_gpu(plan, d64, lam, False).reshape(ref.shape)
    err = float(np.linalg.norm(got - ref))
    assert err <= _bound(g, D, lam), (name, err, _bound(g, D, lam), rel_l2(got, ref))


@pytest.mark.parametrize("name", ["ds2_theta", "ds3_radix3", "odd_nx27", "cube32_k4", "spec192"])
def test_mhad_upsampled_is_the_band_limited_interpolation(name):
    """The model-grid image (a) equals the oracle's portrait-mesh image on
    model rows s i' + ds_offset and (b) has no drive-axis spectrum outside
    the mesh's band |w| <= mx/2.  (a) and (b) fix it uniquely."""
    p, lam = CASES[name]
    g = oracle_geom(p)
    plan = gpu_plan(p)
    d64, d = _portraits(g, 400 + len(name))
    D = _dephased(g, d)
    ref = oracle.mhad(D, [oracle.ck(k, g.gammaA) for k in range(g.k_min, g.k_max + 1)], lam, axis=-1,
                      k_min=g.k_min)
    up = _mhad_gpu(plan, d64, lam, True).reshape(g.shape)
    s, r = g.ds_factor, g.ds_offset
    err = float(np.linalg.norm(up[..., r::s] - ref))
    assert err <= _bound(g, D, lam), (err, _bound(g, D, lam))
    nx = g.n[0]
    mx = nx // s
    spec = np.fft.fft(up, axis=-1)
    w = np.fft.fftfreq(nx, 1.0 / nx)
    outside = np.abs(w) > mx / 2
    assert np.linalg.norm(spec[..., outside]) <= 1e-5 * np.linalg.norm(spec), name


def test_mhad_full_size_128x128x64_k8():
    """The bench geometry (K = 8, s = 2) with portraits of a phantom made by
    the GPU forward operator plus 25 dB noise; the oracle's closed form runs
    whole at this size (FFTs only)."""
    from paper_2503_13802_gb300 import Plan, mh3d_forward

    wl = W.WORKLOADS["mh_128x128x64_k8_s2"]
    p = params(wl.n, s=2, kmin=2, kmax=9)
    g = oracle_geom(p)
    b = W.sensitivity(wl.n, (1.0, 1.0, 1.0), kind="gaussian")
    plan = Plan(wl.n, ds_factor=2, k_min=2, k_max=9, sensitivity=b)
    rho = W.phantom(wl.n, (1.0, 1.0, 1.0), 7, wl.n_blobs, wl.n_lines)
    dt = torch.empty(plan.portrait_shape, dtype=torch.complex64, device="cuda")
    mh3d_forward(plan, torch.as_tensor(rho, dtype=torch.float32).cuda().contiguous(), dt)
    sig = math.sqrt(float(torch.sum(torch.abs(dt.to(torch.complex128)) ** 2)) / (dt.numel() * 10 ** 2.5))
    dt = (dt + sig * torch.as_tensor(W.unit_complex_noise(tuple(dt.shape), 7).astype(np.complex64)).cuda())
    d64 = dt.contiguous().cpu().numpy()
    lam = 1e-2
    D = _dephased(g, d64.astype(np.complex128))
    ref = oracle.mhad(D, [oracle.ck(k, g.gammaA) for k in range(2, 10)], lam, axis=-1, k_min=2)
    got = _mhad_gpu(plan, d64, lam, False).reshape(ref.shape)
    err = float(np.linalg.norm(got - ref))
    assert err <= _bound(g, D, lam), (err, _bound(g, D, lam))
    assert rel_l2(got, ref) <= 1e-5, rel_l2(got, ref)


def test_warm_start_scale_is_the_least_squares_fit():
    """x0 = alpha u, u = upsampled image / b, alpha = Re<A u, d> / ||A u||^2:
    alpha and x0 checked against the FP64 oracle's forward operator applied
    to the GPU's u."""
    from paper_2503_13802_gb300 import mh3d_mhad_warm_start

    p = OP_CASES["ds2_theta"]
    g = oracle_geom(p)
    b = sens_map(p)
    plan = gpu_plan(p, b)
    rho = W.phantom(p["n"], p["voxel"], 5, 10, 1)
    d = oracle.forward(g, rho, b)
    d = d + 0.05 * np.sqrt(np.mean(np.abs(d) ** 2)) * W.unit_complex_noise(d.shape, 5)
    d64 = d.astype(np.complex64)
    lam = 1e-2
    up = _mhad_gpu(plan, d64, lam, True).reshape(g.shape)
    u = np.where(b > 0, up / np.where(b > 0, b, 1.0), 0.0)
    Au = oracle.forward(g, u, b)
    alpha_ref = float(np.real(np.vdot(Au, d64.astype(np.complex128))) / np.vdot(Au, Au).real)
    x0 = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    al = torch.zeros(1, dtype=torch.float64, device="cuda")
    mh3d_mhad_warm_start(plan, torch.as_tensor(d64).cuda(), lam, x0, alpha=al)
    alpha = float(al.item())
    assert abs(alpha - alpha_ref) <= 1e-5 * abs(alpha_ref), (alpha, alpha_ref)
    assert rel_l2(x0.cpu().numpy(), alpha_ref * u) <= 2e-5


def test_warm_start_solve_converges_to_the_zero_start_solution():
    from paper_2503_13802_gb300 import make_opts, mh3d_mhad_warm_start, mh3d_solve

    p = OP_CASES["ds2_theta"]
    g = oracle_geom(p)
    b = sens_map(p)
    plan = gpu_plan(p, b)
    rho = W.phantom(p["n"], p["voxel"], 6, 10, 1)
    d = oracle.forward(g, rho, b)
    d = (d + 0.05 * np.sqrt(np.mean(np.abs(d) ** 2)) * W.unit_complex_noise(d.shape, 6)).astype(np.complex64)
    dt = torch.as_tensor(d).cuda()
    x_zero = torch.empty(g.shape, dtype=torch.float32, device="cuda")
    i0 = mh3d_solve(plan, dt, make_opts(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500), x_zero)
    x0 = torch.empty_like(x_zero)
    mh3d_mhad_warm_start(plan, dt, 1e-2, x0)
    xw = torch.empty_like(x_zero)
    iw = mh3d_solve(plan, dt, make_opts(lam=1e-3, lam_relative=True, rel_tol=1e-4, max_iter=500, x0=x0,
                                        x0_fallback=True), xw)
    assert i0["status"] == 0 and iw["status"] == 0
    assert iw["rel_res_true"] <= 1.5e-4
    assert rel_l2(xw.cpu().numpy(), x_zero.cpu().numpy()) <= 5e-2


def test_mhad_zero_portraits_and_invalid_lambda():
    from paper_2503_13802_gb300 import MH3DError, mh3d_mhad, mh3d_mhad_warm_start

    p = OP_CASES["cube32_k4"]
    plan = gpu_plan(p, sens_map(p))
    d = torch.zeros(plan.portrait_shape, dtype=torch.complex64, device="cuda")
    out = torch.full((plan.N,), 7.0, dtype=torch.float32, device="cuda")
    mh3d_mhad(plan, d, 1e-3, out, upsample=True)
    assert float(out.abs().max()) == 0.0
    al = torch.full((1,), 3.0, dtype=torch.float64, device="cuda")
    mh3d_mhad_warm_start(plan, d, 1e-3, out, alpha=al)
    assert float(al.item()) == 0.0 and float(out.abs().max()) == 0.0
    for lam in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(MH3DError) as e:
            mh3d_mhad(plan, d, lam, out, upsample=True)
        assert "INVALID_ARG" in str(e.value)
