"""Seeded synthetic VLA-like imaging problems (input generator only).

This module draws every random quantity of a test or benchmark problem and
nothing else: uv/w coordinates, a continuous sky made of Gaussian blobs with
power-law spectra, its visibilities, and complex Gaussian noise.  It holds
none of the imaging method's arithmetic (no interpolation kernel, no FFT, no
sparse matrix, no proximal operator); both the FP64 oracle and the CUDA
library consume its output.

The visibilities are the exact continuous Fourier transform of the blob sky
(including the small-field w-term chirp of Sec. 3.2), evaluated analytically,
so that the data do not depend on either implementation of the measurement
operator of Eq. 1.  The recipe (uv mixture, blob statistics, 40 dB input SNR,
blocks, channel frequencies) stands in for the VLA Cyg A data of Sec. 5.1,
which is not available.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field

import numpy as np

# Named workloads.  Sizes follow the imaging configurations the library is
# measured on; small ones are parity cases the oracle finishes in seconds.
WORKLOADS = {
    # 128x128, 4 channels, 2e4 visibilities/channel, 2 blocks, no w-term,
    # 2x2 facets with 10% overlap, one spectral sub-cube, 50 iterations.
    "small_128": dict(config_id=1, ny=128, nx=128, L=4, M=20000, B=2, C=1,
                      qy=2, qx=2, overlap=0.1, w_max=0.0, n_iter=50, n_reweight=0),
    # 1024x1024, 16 channels, 1e6 visibilities/channel in 4 blocks, w-terms
    # uniform on [0, 2000] wavelengths (7..15 taps per dimension), 4x4 facets,
    # 2 spectral sub-cubes, 200 iterations with one reweighting.
    "vla_1024": dict(config_id=2, ny=1024, nx=1024, L=16, M=1_000_000, B=4, C=2,
                     qy=4, qx=4, overlap=0.1, w_max=2000.0, n_iter=200, n_reweight=1),
    # 2048x2048, 32 channels, 4e6 visibilities/channel in 8 blocks, 8x8 facets,
    # 4 sub-cubes, no w-term, 300 iterations.
    "vla_2048": dict(config_id=3, ny=2048, nx=2048, L=32, M=4_000_000, B=8, C=4,
                     qy=8, qx=8, overlap=0.1, w_max=0.0, n_iter=300, n_reweight=0),
    # Profiling case of the same kernels: 1024x1024, 8 channels (one sub-cube),
    # 5e5 visibilities/channel with w-terms; ~6 GB on the device, inputs > L2.
    "prof_1024": dict(config_id=4, ny=1024, nx=1024, L=8, M=500_000, B=4, C=1,
                      qy=4, qx=4, overlap=0.1, w_max=2000.0, n_iter=20, n_reweight=0),
    # Profiling case of the 2048x2048 configuration: its per-channel density
    # (4e6 visibilities per channel in 8 blocks over a 4096^2 grid, no w-term)
    # on 4 channels of one sub-cube; about 8 GB on the device.
    "prof_2048": dict(config_id=5, ny=2048, nx=2048, L=4, M=4_000_000, B=8, C=1,
                      qy=8, qx=8, overlap=0.1, w_max=0.0, n_iter=20, n_reweight=0),
    # Parity-test shapes: several tiles, ragged sizes, w-terms, two sub-cubes.
    "mid_w": dict(config_id=11, ny=96, nx=160, L=4, M=12000, B=3, C=2,
                  qy=3, qx=2, overlap=0.15, w_max=2000.0, n_iter=20, n_reweight=1),
    "tiny": dict(config_id=12, ny=32, nx=48, L=2, M=700, B=2, C=1,
                 qy=2, qx=2, overlap=0.2, w_max=0.0, n_iter=10, n_reweight=0),
    # The 32-channel facet Gram of the 2048x2048 mixed-precision configuration
    # (8x8 facets, 10% overlap) as one sub-cube, with few visibilities: the
    # Gram, the 32x32 eigendecomposition and the apply do not depend on M.
    "gram32_2048": dict(config_id=13, ny=2048, nx=2048, L=32, M=200_000, B=8, C=1,
                        qy=8, qx=8, overlap=0.1, w_max=0.0, n_iter=20, n_reweight=0),
}


@dataclass
class Problem:
    """One synthetic wideband imaging problem (all arrays on the host, FP64)."""
    name: str
    ny: int
    nx: int
    L: int
    C: int
    B: int
    qy: int
    qx: int
    overlap: float
    w_max: float
    pixel_size: float            # radians per pixel (delta l)
    freqs: np.ndarray            # (L,) channel frequency / nu_0
    omega: np.ndarray            # (L, M, 2) radians per pixel, [..,0] along y (rows), [..,1] along x
    w: np.ndarray                # (L, M) w coordinate in wavelengths
    y: np.ndarray                # (L, M) complex128 raw (not whitened) visibilities
    sigma: np.ndarray            # (L,) noise standard deviation of each channel
    block_offsets: np.ndarray    # (L, B+1) int64 offsets of the data blocks inside each channel
    x_true: np.ndarray           # (L, ny, nx) blob sky sampled at pixel centres
    n_iter: int = 0
    n_reweight: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def M(self) -> int:
        return self.omega.shape[1]


def workload_seed(config_id: int, trial: int = 0) -> int:
    return 7604 + 100 * config_id + trial


def _draw_uv(rng: np.random.Generator, M: int) -> np.ndarray:
    """90% isotropic Gaussian (sd 0.25*pi) kept inside [-pi, pi)^2, 10% uniform."""
    n_unif = M // 10
    n_gauss = M - n_unif
    out = np.empty((M, 2))
    got = 0
    while got < n_gauss:
        cand = rng.normal(0.0, 0.25 * math.pi, size=(2 * (n_gauss - got) + 16, 2))
        ok = np.all((cand >= -math.pi) & (cand < math.pi), axis=1)
        cand = cand[ok][: n_gauss - got]
        out[got: got + len(cand)] = cand
        got += len(cand)
    out[n_gauss:] = rng.uniform(-math.pi, math.pi, size=(n_unif, 2))
    perm = rng.permutation(M)
    return out[perm]


def _blob_ft(o1: np.ndarray, o2: np.ndarray, a: np.ndarray, c1: float, c2: float, s: float) -> np.ndarray:
    """Fourier transform of the blob exp(-|t-c|^2/(2 s^2)) times the w-term
    chirp exp(i pi a |t|^2), at frequencies (o1, o2):
    prod_d int exp(-(t-c_d)^2/(2 s^2) + i pi a t^2 - i o_d t) dt
      = (pi / alpha) exp(-(q1^2 + q2^2)/(4 alpha) + i (pi a |c|^2 - o.c)),
    alpha = 1/(2 s^2) - i pi a, q_d = 2 pi a c_d - o_d (written around t = c so
    that no large exponent cancels)."""
    alpha = 1.0 / (2.0 * s * s) - 1j * math.pi * a
    q1 = 2.0 * math.pi * a * c1 - o1
    q2 = 2.0 * math.pi * a * c2 - o2
    return (math.pi / alpha) * np.exp(-(q1 * q1 + q2 * q2) / (4.0 * alpha)
                                      + 1j * (math.pi * a * (c1 * c1 + c2 * c2) - o1 * c1 - o2 * c2))


def make_problem(name: str = "small_128", trial: int = 0, M: int | None = None,
                 n_blobs: int = 20, snr_db: float = 40.0, **overrides) -> Problem:
    """Draw the problem of workload ``name`` with seed 7604 + 100*config_id + trial."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    if M is not None:
        spec["M"] = M
    seed = workload_seed(spec["config_id"], trial)
    rng = np.random.Generator(np.random.Philox(seed))
    ny, nx, L, Mv, B = spec["ny"], spec["nx"], spec["L"], spec["M"], spec["B"]
    w_max = float(spec["w_max"])
    # Field of view chosen so that the chirp of the largest w sweeps about
    # 4 cells of the 2x oversampled grid: FoV^2 = 2 / w_max.
    n_max = max(ny, nx)
    fov = math.sqrt(2.0 / w_max) if w_max > 0 else 0.05
    pixel_size = fov / n_max

    freqs = 1.0 + np.arange(L) / max(L - 1, 1)        # nu_l / nu_0 on [1, 2]
    scale = freqs / freqs[-1]                          # uv drawn at the top channel
    uv_top = _draw_uv(rng, Mv)
    w_top = rng.uniform(0.0, w_max, size=Mv) if w_max > 0 else np.zeros(Mv)
    omega = scale[:, None, None] * uv_top[None, :, :]
    w = scale[:, None] * w_top[None, :]

    # Blob sky (pixel coordinates n = i - N/2).
    my, mx = 0.1 * ny, 0.1 * nx
    cy = rng.uniform(-ny / 2 + my, ny / 2 - my, size=n_blobs)
    cx = rng.uniform(-nx / 2 + mx, nx / 2 - mx, size=n_blobs)
    fwhm = rng.uniform(2.0, 8.0, size=n_blobs)
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    amp = np.exp(rng.uniform(math.log(0.1), math.log(1.0), size=n_blobs))
    alpha = rng.uniform(-1.0, 0.0, size=n_blobs)
    amp_l = amp[None, :] * freqs[:, None] ** alpha[None, :]          # (L, n_blobs)

    n1 = np.arange(ny) - ny // 2
    n2 = np.arange(nx) - nx // 2
    x_true = np.zeros((L, ny, nx))
    for b in range(n_blobs):
        gy = np.exp(-((n1 - cy[b]) ** 2) / (2 * s[b] ** 2))
        gx = np.exp(-((n2 - cx[b]) ** 2) / (2 * s[b] ** 2))
        x_true += amp_l[:, b, None, None] * (gy[:, None] * gx[None, :])[None]

    y = np.zeros((L, Mv), dtype=np.complex128)
    sigma = np.zeros(L)
    chunk = 1 << 16

    def sky_vis(job):
        l, s0 = job
        sl = slice(s0, min(Mv, s0 + chunk))
        a_l = w[l, sl] * pixel_size ** 2
        acc = np.zeros(sl.stop - sl.start, dtype=np.complex128)
        o1, o2 = omega[l, sl, 0], omega[l, sl, 1]
        for b in range(n_blobs):
            acc += amp_l[l, b] * _blob_ft(o1, o2, a_l, cy[b], cx[b], s[b])
        y[l, sl] = acc

    jobs = [(l, s0) for l in range(L) for s0 in range(0, Mv, chunk)]
    if len(jobs) > 4:      # numpy ufuncs release the GIL: threads share the work
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 1)) as ex:
            list(ex.map(sky_vis, jobs))
    else:
        for j in jobs:
            sky_vis(j)
    for l in range(L):
        sigma[l] = np.linalg.norm(y[l]) / math.sqrt(Mv) * 10.0 ** (-snr_db / 20.0)
    noise = (rng.standard_normal((L, Mv)) + 1j * rng.standard_normal((L, Mv))) / math.sqrt(2.0)
    y += sigma[:, None] * noise

    bo = np.array([[(b * Mv) // B for b in range(B + 1)] for _ in range(L)], dtype=np.int64)
    return Problem(name=name, ny=ny, nx=nx, L=L, C=spec["C"], B=B, qy=spec["qy"], qx=spec["qx"],
                   overlap=spec["overlap"], w_max=w_max, pixel_size=pixel_size, freqs=freqs,
                   omega=omega, w=w, y=y, sigma=sigma, block_offsets=bo, x_true=x_true,
                   n_iter=spec["n_iter"], n_reweight=spec["n_reweight"], seed=seed)


def random_image(shape, seed: int, nonneg: bool = True) -> np.ndarray:
    """Seeded test image/cube (uniform on [0,1) or standard normal)."""
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.uniform(0.0, 1.0, size=shape) if nonneg else rng.standard_normal(shape)


def random_vis(shape, seed: int) -> np.ndarray:
    """Seeded complex standard-normal vector."""
    rng = np.random.Generator(np.random.Philox(seed))
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def random_dde(L: int, M: int, seed: int, spread: float = 0.1) -> np.ndarray:
    """Seeded synthetic DDE kernels (L, M, 5, 5) complex128: the Fourier
    representation of smooth direction-dependent gains, i.e. 1 at the centre
    tap plus complex perturbations that decay with the tap distance
    (spread * exp(-|delta|^2 / 2) standard deviation)."""
    rng = np.random.Generator(np.random.Philox(seed))
    d = np.arange(5) - 2
    env = spread * np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / 2.0)
    k = (rng.standard_normal((L, M, 5, 5)) + 1j * rng.standard_normal((L, M, 5, 5))) / math.sqrt(2.0)
    k *= env[None, None]
    k[:, :, 2, 2] += 1.0
    return k
