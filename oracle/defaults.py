"""Oracle dirty image, residual and regularisation defaults.

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

* PSF normalisation (Sec. 5.3): eta_l = 1 / (Re Phi_l^dagger Phi_l delta)(centre),
  delta the unit image at the phase centre, so that eta_l Phi_l^dagger Phi_l has
  peak 1 there.
* Residual (Sec. 5.3): r_l = eta_l Re Phi_l^dagger (y_l - Phi_l x_l), with the
  whitened data y_l (Theta_l applied); the dirty image is r for x = 0.
* Regularisation defaults (the paper defers the heuristics to Part I; the
  reading used here is the dirty-image form): with X the dirty cube,
  mu_bar = 1 / sum_{c,q} ||S_q X_c||_* (facet nuclear norms of every
  sub-cube, D_q = 1) and mu = 1 / sum_c ||Psi^dagger X_c||_{2,1} (rows over
  the sub-cube's channels).  Sub-cube c holds channels c, c + C, ... (Eq. 3).
* Noise statistics and l2 bounds from a model image (Sec. 3.3 (i), Sec. 5.1
  and the pre-processing paragraph of Sec. 5): with the residual visibilities
  r_{l,b} = Theta_l (y_{l,b} - Phi_{l,b} x0_l) of a model cube x0, the noise
  level of block (l, b) is sigma_l times the standard deviation of r_{l,b}
  (complex sample standard deviation, mean removed, M_{l,b} - 1 degrees of
  freedom) and its l2 bound is ||r_{l,b}||_2.  With data reduction the bound
  of channel l is ||y'_l - Phi'_l x0_l||_2 (Sec. 5.2, with the model
  visibilities Phi_l x0_l), and its noise level eps'_l / sqrt(M'_l).
"""
from __future__ import annotations

import numpy as np


def psf_peak_factors(op, ny: int, nx: int) -> np.ndarray:
    """eta_l for every channel of ``op`` (a nufft.Operator)."""
    d = np.zeros((ny, nx))
    d[ny // 2, nx // 2] = 1.0
    out = []
    for l in range(op.L):
        psf = np.real(op.adjoint(op.forward(d, l), l))
        out.append(1.0 / psf[ny // 2, nx // 2])
    return np.array(out)


def residual(op, yw, X: np.ndarray, eta: np.ndarray) -> np.ndarray:
    """r_l = eta_l Re Phi_l^dagger (y_l - Phi_l x_l); X may be None (dirty image)."""
    out = []
    for l in range(op.L):
        r = yw[l] if X is None else yw[l] - op.forward(X[l], l)
        out.append(eta[l] * np.real(op.adjoint(r, l)))
    return np.stack(out)


def default_regularisation(Xd: np.ndarray, C: int, facets, sara) -> tuple:
    """(mu, mu_bar) from the dirty cube Xd (L, ny, nx)."""
    L = Xd.shape[0]
    nuc = 0.0
    l21 = 0.0
    for c in range(C):
        ch = list(range(c, L, C))
        for (y0, y1, x0, x1) in facets:
            Z = Xd[ch, y0:y1, x0:x1].reshape(len(ch), -1)
            nuc += float(np.linalg.svd(Z, compute_uv=False).sum())
        A = np.stack([sara.analysis(Xd[l]) for l in ch])
        l21 += float(np.sqrt((A ** 2).sum(axis=0)).sum())
    return 1.0 / l21, 1.0 / nuc


def noise_from_model(op, yw, sigma, block_offsets, X0: np.ndarray) -> tuple:
    """(sigma_hat (L, B), eps (L, B)) from the model cube X0 (L, ny, nx); yw the
    whitened data per channel, sigma the per-channel whitening."""
    bo = np.asarray(block_offsets)
    L, B = bo.shape[0], bo.shape[1] - 1
    sig = np.zeros((L, B))
    eps = np.zeros((L, B))
    for l in range(L):
        r = yw[l] - op.forward(X0[l], l)
        for b in range(B):
            rb = r[bo[l, b]:bo[l, b + 1]]
            eps[l, b] = np.linalg.norm(rb)
            if len(rb) > 1:
                sig[l, b] = sigma[l] * np.sqrt(np.sum(np.abs(rb - rb.mean()) ** 2) / (len(rb) - 1))
    return sig, eps


def reduced_bounds(red, X0: np.ndarray) -> tuple:
    """(sigma_hat (L,), eps' (L,)) of the reduced data (``reduction.Reduced``)."""
    eps = np.array([np.linalg.norm(red.y[l] - red.forward(X0[l], l)) for l in range(red.L)])
    m = np.array([red.m_red(l) for l in range(red.L)], dtype=np.float64)
    return np.where(m > 0, eps / np.sqrt(np.maximum(m, 1.0)), 0.0), eps
