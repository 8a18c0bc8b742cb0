"""Seeded synthetic inputs for MH3D workloads.

This module is shared by the tests, the benchmark and the FP64 oracle's
callers.  It holds NO arithmetic of the method (no PSF, no operator, no
solver): only random streams, phantoms, a receive-sensitivity map and unit
complex noise.  The caller scales the noise to an SNR with the signal it
computed itself.

Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014).  Output i of stream `seed` is
mix(seed + (i+1) * 0x9E3779B97F4A7C15) with the published mix function, so
the stream is counter-based and vectorises.  Uniforms take the top 53 bits;
normals use the Box-Muller transform (Box and Muller, 1958).

The paper measures on its own scanner data (VivoTrax phantoms, a head
mannequin, lymph-node phantoms), none of which is public; these synthetic
phantoms stand in for them.  Draw order for one volume (stream = seed):
  per blob  : sigma, cx, cy, cz, amplitude            (5 uniforms)
  per line  : fwhm, amplitude, x0, y0, z0, x1, y1, z1 (8 uniforms)
Noise uses stream seed ^ 0x5DEECE66D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
NOISE_STREAM_XOR = 0x5DEECE66D


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    z = splitmix64(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Stream:
    """Sequential view of one counter-based stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def uniform(self, count: int = 1, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = uniform01(self.seed, self.pos, count)
        self.pos += count
        return lo + (hi - lo) * u

    def normal(self, count: int) -> np.ndarray:
        """Standard normals by Box-Muller, two per pair of uniforms."""
        npair = (count + 1) // 2
        u = self.uniform(2 * npair)
        u1 = 1.0 - u[0::2]                      # (0, 1]
        u2 = u[1::2]
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * npair)
        z[0::2] = rad * np.cos(2.0 * np.pi * u2)
        z[1::2] = rad * np.sin(2.0 * np.pi * u2)
        return z[:count]


def voxel_coords(n: Sequence[int], voxel_mm: Sequence[float]):
    """Voxel-centre coordinates (mm) per axis: (i - (n-1)/2) * delta."""
    return [(np.arange(n[a]) - (n[a] - 1) / 2.0) * voxel_mm[a] for a in range(3)]


def sensitivity(n: Sequence[int], voxel_mm: Sequence[float] = (1.0, 1.0, 1.0),
                kind: str = "gaussian", frac: float = 0.6) -> Optional[np.ndarray]:
    """Receive-sensitivity map b (float64 [nz][ny][nx]), peak 1 at the centre:
    b = exp(-sum_a x_a^2 / (2 (frac * n_a * delta_a)^2)).  kind='uniform'
    returns None (b = 1)."""
    if kind == "uniform":
        return None
    xs = voxel_coords(n, voxel_mm)
    g = [np.exp(-xs[a] ** 2 / (2.0 * (frac * n[a] * voxel_mm[a]) ** 2)) for a in range(3)]
    return g[2][:, None, None] * g[1][None, :, None] * g[0][None, None, :]


def _gauss1d(x, c, s):
    return np.exp(-((x - c) ** 2) / (2.0 * s * s))


def phantom(n: Sequence[int], voxel_mm: Sequence[float], seed: int, n_blobs: int,
            n_lines: int = 0, log_amplitudes: bool = False) -> np.ndarray:
    """Sum of Gaussian blobs (sigma ~ U(1.5, 4) mm, centres >= 3 sigma from the
    faces, amplitude U(0.2, 1) or 10^U(-3, 0)) and line segments (Gaussian
    cross-section, FWHM ~ U(1, 2) mm, amplitude U(0.2, 1), endpoints uniform
    inside a 3 mm margin).  float64 [nz][ny][nx], nonnegative."""
    st = Stream(seed)
    xs = voxel_coords(n, voxel_mm)
    half = [xs[a][-1] + 0.5 * voxel_mm[a] for a in range(3)]   # FOV half-widths
    vol = np.zeros((n[2], n[1], n[0]))
    for _ in range(n_blobs):
        u = st.uniform(5)
        sig = 1.5 + 2.5 * u[0]
        c = []
        for a in range(3):
            lim = max(half[a] - 3.0 * sig, 0.0)
            c.append(-lim + 2.0 * lim * u[1 + a])
        amp = 10.0 ** (-3.0 + 3.0 * u[4]) if log_amplitudes else 0.2 + 0.8 * u[4]
        gx, gy, gz = (_gauss1d(xs[a], c[a], sig) for a in range(3))
        vol += amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    if n_lines:
        Z, Yg, Xg = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
        for _ in range(n_lines):
            u = st.uniform(8)
            fwhm = 1.0 + u[0]
            amp = 0.2 + 0.8 * u[1]
            lim = [max(half[a] - 3.0, 0.0) for a in range(3)]
            p0 = np.array([-lim[a] + 2 * lim[a] * u[2 + a] for a in range(3)])
            p1 = np.array([-lim[a] + 2 * lim[a] * u[5 + a] for a in range(3)])
            dvec = p1 - p0
            L2 = float(dvec @ dvec)
            t = ((Xg - p0[0]) * dvec[0] + (Yg - p0[1]) * dvec[1] + (Z - p0[2]) * dvec[2])
            t = np.clip(t / L2, 0.0, 1.0) if L2 > 0 else np.zeros_like(Xg)
            dist2 = ((Xg - p0[0] - t * dvec[0]) ** 2 + (Yg - p0[1] - t * dvec[1]) ** 2
                     + (Z - p0[2] - t * dvec[2]) ** 2)
            s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
            vol += amp * np.exp(-dist2 / (2.0 * s * s))
    return vol


def _box(x, lo, hi):
    """Index range of the sorted coordinates x that lie in [lo, hi]."""
    return int(np.searchsorted(x, lo, "left")), int(np.searchsorted(x, hi, "right"))


def learned_case(n: Sequence[int], voxel_mm: Sequence[float], seed: int, n_lines: int = 3):
    """One volume of the learned-warm-start workload: (phantom, snr_db).

    Blob count log-uniform in [5, 200], SNR U(15, 40) dB, then blobs as in
    `phantom` (sigma ~ U(1.5, 4) mm, centres >= 3 sigma from the faces,
    amplitude U(0.2, 1)) and `n_lines` line segments (FWHM U(1, 2) mm,
    amplitude U(0.2, 1), endpoints inside a 3 mm margin).  Each blob and line
    is evaluated only inside its box of +-4 sigma (where the Gaussian has
    fallen below e^-8 of its peak) so that thousands of volumes stay cheap.
    Draw order (stream = seed): count, SNR, then 5 uniforms per blob and 8
    per line, as in `phantom`."""
    st = Stream(seed)
    u0 = st.uniform(2)
    nb = int(round(math.exp(math.log(5.0) + (math.log(200.0) - math.log(5.0)) * u0[0])))
    snr_db = 15.0 + 25.0 * u0[1]
    xs = voxel_coords(n, voxel_mm)
    half = [xs[a][-1] + 0.5 * voxel_mm[a] for a in range(3)]
    vol = np.zeros((n[2], n[1], n[0]))
    for _ in range(nb):
        u = st.uniform(5)
        sig = 1.5 + 2.5 * u[0]
        c = []
        for a in range(3):
            lim = max(half[a] - 3.0 * sig, 0.0)
            c.append(-lim + 2.0 * lim * u[1 + a])
        amp = 0.2 + 0.8 * u[4]
        r = [_box(xs[a], c[a] - 4.0 * sig, c[a] + 4.0 * sig) for a in range(3)]
        gx, gy, gz = (_gauss1d(xs[a][r[a][0]:r[a][1]], c[a], sig) for a in range(3))
        vol[r[2][0]:r[2][1], r[1][0]:r[1][1], r[0][0]:r[0][1]] += \
            amp * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    for _ in range(n_lines):
        u = st.uniform(8)
        fwhm = 1.0 + u[0]
        amp = 0.2 + 0.8 * u[1]
        lim = [max(half[a] - 3.0, 0.0) for a in range(3)]
        p0 = np.array([-lim[a] + 2 * lim[a] * u[2 + a] for a in range(3)])
        p1 = np.array([-lim[a] + 2 * lim[a] * u[5 + a] for a in range(3)])
        s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
        r = [_box(xs[a], min(p0[a], p1[a]) - 4.0 * s, max(p0[a], p1[a]) + 4.0 * s) for a in range(3)]
        Z, Yg, Xg = np.meshgrid(xs[2][r[2][0]:r[2][1]], xs[1][r[1][0]:r[1][1]], xs[0][r[0][0]:r[0][1]],
                                indexing="ij")
        dvec = p1 - p0
        L2 = float(dvec @ dvec)
        t = ((Xg - p0[0]) * dvec[0] + (Yg - p0[1]) * dvec[1] + (Z - p0[2]) * dvec[2])
        t = np.clip(t / L2, 0.0, 1.0) if L2 > 0 else np.zeros_like(Xg)
        dist2 = ((Xg - p0[0] - t * dvec[0]) ** 2 + (Yg - p0[1] - t * dvec[1]) ** 2
                 + (Z - p0[2] - t * dvec[2]) ** 2)
        vol[r[2][0]:r[2][1], r[1][0]:r[1][1], r[0][0]:r[0][1]] += amp * np.exp(-dist2 / (2.0 * s * s))
    return vol, snr_db


# Seeds of the learned-warm-start workload (128x128x64, K = 8, s = 2).
LEARNED_TRAIN_SEEDS = tuple(range(10000, 12000))
LEARNED_TEST_SEEDS = tuple(range(20000, 20200))


def unit_complex_noise(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    """Circular complex Gaussian noise with E|n|^2 = 1 (re, im ~ N(0, 1/2))."""
    st = Stream(int(seed) ^ NOISE_STREAM_XOR)
    cnt = int(np.prod(shape))
    z = st.normal(2 * cnt) * math.sqrt(0.5)
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


def random_volume(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    """Standard normal test volume (for operator parity, not a phantom)."""
    return Stream(seed).normal(int(np.prod(shape))).reshape(shape)


def random_portraits(shape: Tuple[int, ...], seed: int) -> np.ndarray:
    """Standard complex normal test portraits (re, im ~ N(0, 1))."""
    z = Stream(seed).normal(2 * int(np.prod(shape)))
    return (z[0::2] + 1j * z[1::2]).reshape(shape)


@dataclass
class Workload:
    """One named synthetic workload: grid, harmonics, downsampling, phantom
    recipe, SNR and solve settings.  `lam` is relative to ||A||_2^2 (b = 1):
    the PSF's overall scale is a free constant of the model."""

    name: str
    n: Tuple[int, int, int]
    k_min: int
    k_max: int
    ds_factor: int
    sens: str
    n_blobs: int
    n_lines: int
    snr_db: float
    lam: float
    rel_tol: float
    max_iter: int
    fixed_iters: bool = False
    log_amplitudes: bool = False
    voxel_mm: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    seeds: Tuple[int, ...] = (0,)


# The five synthetic workloads (drive axis x, 1 mm voxels).
WORKLOADS = {
    "plain_fp64_32cube": Workload("plain_fp64_32cube", (32, 32, 32), 2, 5, 1, "uniform", 5, 0,
                                  30.0, 1e-3, 0.0, 100, fixed_iters=True, seeds=tuple(range(10))),
    "mh_128x128x64_k8_s2": Workload("mh_128x128x64_k8_s2", (128, 128, 64), 2, 9, 2, "gaussian",
                                    40, 3, 25.0, 1e-3, 1e-4, 2000, seeds=tuple(range(10))),
    "precision_256x256x128_k16": Workload("precision_256x256x128_k16", (256, 256, 128), 2, 17, 1,
                                          "uniform", 200, 0, 30.0, 1e-3, 1e-4, 2000,
                                          log_amplitudes=True, seeds=tuple(range(5))),
}

# Size classes of the batched workload: 64 volumes drawn uniformly (seeded).
BATCH_SIZE_CLASSES = ((64, 64, 64), (96, 96, 64), (128, 128, 64), (192, 192, 96))


def batch_sizes(nvol: int = 64, seed: int = 777) -> list:
    u = uniform01(seed, 0, nvol)
    idx = np.minimum((u * len(BATCH_SIZE_CLASSES)).astype(int), len(BATCH_SIZE_CLASSES) - 1)
    return [BATCH_SIZE_CLASSES[i] for i in idx]
