"""Portrait phase calibration (Sec. 4.4) on the GPU (mh3d_estimate_phase)
against the FP64 oracle's estimate_phase on the same complex64 portraits,
and against the phases that generated the portraits.

Parity: both sides sum the same samples (the high-SNR selection compares
|d| with frac max |d|, FP32 on the GPU and FP64 in the oracle, so a sample
within rounding of the threshold may fall either way); theta within 1e-4
rad and the same resolved flags."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from tests._cases import gpu_plan, oracle_geom, params

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "s1": params((48, 16, 12), s=1, kmin=3, kmax=6),
    "s1_k2": params((32, 24, 16), s=1, kmin=2, kmax=7),
    "s2": params((64, 12, 8), s=2, kmin=2, kmax=9),
}


def _data(p, snr_db, seed):
    K = p["kmax"] - p["kmin"] + 1
    theta = np.random.default_rng(seed).uniform(-np.pi, np.pi, K)
    q = dict(p)
    q["theta"] = list(theta)
    g = oracle_geom(q)
    rho = W.phantom(p["n"], p["voxel"], seed, 6, 1)
    d = oracle.forward(g, rho)
    if snr_db is not None:
        d = d + math.sqrt(float(np.mean(np.abs(d) ** 2)) / 10 ** (snr_db / 10)) * W.unit_complex_noise(d.shape, seed)
    return theta, g, d.astype(np.complex64)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("snr", [None, 25.0])
def test_phase_matches_oracle_and_generating_phases(name, snr):
    from paper_2503_13802_gb300 import mh3d_estimate_phase

    p = CASES[name]
    theta, g, d = _data(p, snr, 60 + len(name))
    plan = gpu_plan(p)                               # the plan's own phases are zero
    est, res = mh3d_estimate_phase(plan, torch.as_tensor(d).cuda())
    ref, ref_res = oracle.estimate_phase(g, d.astype(np.complex128))
    assert np.array_equal(res, ref_res), (res, ref_res)
    assert np.abs(np.angle(np.exp(1j * (est - ref)))).max() <= 1e-4, (est, ref)
    tol = 1e-5 if snr is None else 0.1
    err = np.angle(np.exp(1j * (est - theta)))
    err_pi = np.angle(np.exp(2j * (est - theta))) / 2
    if res.any():
        assert np.abs(err[res == 1]).max() <= tol, err
    assert np.abs(err_pi).max() <= tol, err_pi
    assert res.all() if p["s"] == 1 else not res.any()


def test_phase_with_the_plan_phases_and_invalid_frac():
    """The estimate does not depend on the plan's own theta; frac outside
    (0, 1] is refused."""
    from paper_2503_13802_gb300 import MH3DError, mh3d_estimate_phase

    p = CASES["s1"]
    theta, g, d = _data(p, None, 71)
    q = dict(p)
    q["theta"] = [0.5, -0.3, 1.1, 2.0]
    plan = gpu_plan(q)
    est, res = mh3d_estimate_phase(plan, torch.as_tensor(d).cuda())
    assert res.all()
    assert np.abs(np.angle(np.exp(1j * (est - theta)))).max() <= 1e-5
    for frac in (0.0, 1.5, -0.2):
        with pytest.raises(MH3DError) as e:
            mh3d_estimate_phase(plan, torch.as_tensor(d).cuda(), frac=frac)
        assert "INVALID_ARG" in str(e.value)
