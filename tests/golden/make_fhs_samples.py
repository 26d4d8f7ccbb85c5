"""Writes fhs_<n>_samples.npz beside this file: the FP64 oracle's PDFB run on
the geometry of one of the two imaging workloads, at 3e4 visibilities per
channel instead of 1e6 or 4e6 so that the oracle finishes:

  1024  1024 x 1024, 16 channels in 2 spectral sub-cubes of 8, 4 x 4 facets
        with 10 % overlap, w-projection up to 2000 wavelengths, 4 data blocks
        per channel; 10 PDFB iterations with one reweighting after the fifth
        (about three minutes per iteration and sub-cube on one core)
  2048  2048 x 2048, 32 channels in 4 spectral sub-cubes of 8, 8 x 8 facets
        with 10 % overlap, no w-term, 8 data blocks per channel; 6 PDFB
        iterations with one reweighting after the third (about nine minutes
        per iteration and sub-cube on one core)

Reweighting is Sec. 2.2.3.  The runs are far too slow for a test, so the file
keeps the step sizes, the regularisation and seeded samples of every part of
the final state, in the layouts of the library's state transfer:

  X     image, [L][ny][nx]                         32768 samples
  v     data dual, [L][M] complex, caller's order  16384 samples
  W     SARA dual, [L][n_coef]                     32768 samples
  P     nuclear dual, per sub-cube and facet
        [L_c][wy][wx], concatenated                 32768 samples
  w21   l21 weights, [C][n_coef]                   16384 samples
  wnuc  nuclear weights, [C][Q][L_c]               all of them

The GPU parity test rebuilds the same problem from the input generator and
compares these samples element by element.  Each sub-cube is an independent
problem (Eq. 3), so each runs in a process of its own.  Only the oracle and
the input generator are called.  Run from the repository root:

    python tests/golden/make_fhs_samples.py 1024
    python tests/golden/make_fhs_samples.py 2048
"""
from __future__ import annotations

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

# side -> (workload, visibilities per channel, iterations, reweightings)
RUNS = {"1024": ("vla_1024", 30_000, 10, 1), "2048": ("vla_2048", 30_000, 6, 1)}
MU, MU_BAR = 0.05, 0.5


def out_path(side):
    return os.path.join(HERE, "fhs_%s_samples.npz" % side)


def problem(side):
    from paper_2209_07604_gb300 import synth
    workload, m_per_channel = RUNS[side][:2]
    return synth.make_problem(workload, M=m_per_channel)


def steps_for(P):
    """tau = 0.99/3, sigma0 = 1/max facet coverage, sigma1 = 1 (the library's
    defaults) and sigma2 = 1 / (1.02 max ||Phi_l||^2) over the lowest and the
    highest channel (ARPACK's Lanczos on the FP64 operator)."""
    from oracle import nufft as onf, pdfb, prox
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    ends = [0, P.L - 1]
    op = onf.Operator(P.omega[ends], P.w[ends], P.sigma[ends], geom)
    nrm = max(op.norm2_eigsh(0), op.norm2_eigsh(1))
    cov = prox.facet_coverage(P.ny, P.nx, prox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap)).max()
    return pdfb.Steps(tau=0.99 / 3.0, sigma0=1.0 / cov, sigma1=1.0, sigma2=1.0 / (1.02 * nrm))


def run_subcube(args):
    side, c, steps = args
    from oracle import pdfb
    n_iter, n_reweight = RUNS[side][2:]
    P = problem(side)
    ch = list(range(c, P.L, P.C))
    o = pdfb.FHS(P.omega[ch], P.w[ch], P.y[ch], P.sigma[ch], P.block_offsets[ch], P.ny, P.nx, 1, P.qy, P.qx,
                 P.overlap, mu=MU, mu_bar=MU_BAR, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size,
                 steps=steps)
    t0 = time.time()
    o.run(n_iter, n_reweight)
    print("sub-cube %d: %d iterations in %.0f s" % (c, n_iter, time.time() - t0), flush=True)
    return c, o.X, np.stack(o.v), o.W[0], [p for p in o.P[0]], o.w21[0], np.stack(o.wnuc[0])


def main(side):
    workload, m_per_channel, n_iter, n_reweight = RUNS[side]
    P = problem(side)
    steps = steps_for(P)
    print("steps", steps, flush=True)
    with mp.get_context("spawn").Pool(P.C) as pool:
        parts = sorted(pool.map(run_subcube, [(side, c, steps) for c in range(P.C)]), key=lambda t: t[0])
    L, C = P.L, P.C
    Lc = L // C
    X = np.zeros((L, P.ny, P.nx))
    v = np.zeros((L, P.omega.shape[1]), dtype=np.complex128)
    n_coef = parts[0][3].shape[1]
    W = np.zeros((L, n_coef))
    for c, Xc, vc, Wc, _, _, _ in parts:
        ch = list(range(c, L, C))
        X[ch], v[ch], W[ch] = Xc, vc, Wc
    Pn = np.concatenate([p.ravel() for part in parts for p in part[4]])
    w21 = np.stack([part[5] for part in parts])
    wnuc = np.stack([part[6] for part in parts])              # [C][Q][L_c]
    rng = np.random.Generator(np.random.Philox(7604 + int(side)))
    out = dict(workload=workload, m_per_channel=m_per_channel, n_iter=n_iter, n_reweight=n_reweight, mu=MU,
               mu_bar=MU_BAR, tau=steps.tau, sigma0=steps.sigma0, sigma1=steps.sigma1, sigma2=steps.sigma2,
               n_coef=n_coef, wnuc=wnuc.ravel(), lc=Lc)
    for name, arr, n in (("X", X.ravel(), 32768), ("v", v.ravel(), 16384), ("W", W.ravel(), 32768),
                         ("P", Pn, 32768), ("w21", w21.ravel(), 16384)):
        idx = np.sort(rng.choice(arr.size, size=n, replace=False))
        out[name + "_idx"] = idx.astype(np.int64)
        out[name] = arr[idx]
        out[name + "_absmax"] = np.abs(arr).max()
        out[name + "_norm"] = np.linalg.norm(arr)
    np.savez_compressed(out_path(side), **out)
    print("wrote", out_path(side), os.path.getsize(out_path(side)), "bytes")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "1024")
