"""Oracle proximal steps of the PDFB iteration (Eq. 2, Sec. 2.2.2-2.2.3).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

Every dual update has the Moreau form u+ = z - s prox_{g/s}(z/s) with
z = u + s L xbar (s the dual step), which for the three terms of Eq. 3 reads:

* l2 ball (data fidelity, Eq. 2):   u+ = (z - s y)(1 - min(1, s eps / ||z - s y||))
* weighted l21 (joint sparsity):    u+_r = z_r min(1, mu w_r / ||z_r||)   (row r over channels)
* weighted nuclear norm (facet):    u+ = z - SVT(z, mu_bar w_i)   (threshold per singular value)
"""
from __future__ import annotations

import math

import numpy as np


def eps_blocks(M_l: int, block_sizes) -> np.ndarray:
    """eps_{l,b} = sqrt(eps_l^2 M_{l,b} / M_l), eps_l^2 = M_l + 2 sqrt(M_l) (Eq. 2)."""
    e2 = M_l + 2.0 * math.sqrt(M_l)
    return np.sqrt(e2 * np.asarray(block_sizes, dtype=np.float64) / M_l)


def proj_l2ball(z: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """Projection onto B(y, eps) = {z : ||z - y|| <= eps}."""
    r = z - y
    nr = np.linalg.norm(r)
    if nr <= eps:
        return z.copy()
    return y + r * (eps / nr)


def l2ball_dual(v: np.ndarray, phix: np.ndarray, y: np.ndarray, eps: float, s: float) -> np.ndarray:
    """Data dual update of one block: z = v + s Phi xbar, u+ = z - s proj_B(z / s)."""
    z = v + s * phix
    return z - s * proj_l2ball(z / s, y, eps)


def l21_dual(W: np.ndarray, A: np.ndarray, s: float, mu: float, weights: np.ndarray) -> np.ndarray:
    """W, A: (L_c, n_coef); rows are the columns (one coefficient across channels).
    z = W + s A; u+ = z - s prox_{(mu/s)||.||_{2,1,w}}(z/s)."""
    z = W + s * A
    nrm = np.sqrt(np.sum(z * z, axis=0))
    thr = mu * weights
    with np.errstate(divide="ignore", invalid="ignore"):
        shrink = np.where(nrm > thr, 1.0 - thr / nrm, 0.0)     # prox of (mu/s) w ||.|| at z/s, times s
    return z - z * shrink[None, :]


def svt(Z: np.ndarray, thr: np.ndarray) -> np.ndarray:
    """Weighted singular-value soft-thresholding of a (p x L) matrix; thr[i]
    pairs with the i-th largest singular value."""
    U, S, Vt = np.linalg.svd(Z, full_matrices=False)
    Sp = np.maximum(S - thr[: len(S)], 0.0)
    return (U * Sp[None, :]) @ Vt


def nuclear_dual(P: np.ndarray, Xq: np.ndarray, s: float, mu_bar: float, weights: np.ndarray) -> np.ndarray:
    """P, Xq: (L_c, wy, wx) facet dual and facet of xbar.  z = P + s Xq;
    u+ = z - s prox_{(mu_bar/s)||.||_{*,w}}(z/s) = z - SVT(z, mu_bar w)."""
    L = P.shape[0]
    Z = (P + s * Xq).reshape(L, -1).T              # pixels x channels
    out = Z - svt(Z, mu_bar * weights)
    return out.T.reshape(P.shape)


def l21_weights(A: np.ndarray, upsilon: float) -> np.ndarray:
    """Log-sum reweighting of the l21 rows (Sec. 2.2.3; Candes et al. 2008): the
    weight of row r is upsilon / (upsilon + ||A_r||_2), where A is (L_c, n_coef)
    and row r is column r, one coefficient across the sub-cube's channels."""
    return upsilon / (upsilon + np.sqrt(np.sum(A * A, axis=0)))


def nuclear_weights(Z: np.ndarray, upsilon_bar: float, L: int) -> np.ndarray:
    """Log-sum reweighting of one facet's singular values (Sec. 2.2.3): Z is the
    (pixels x L) facet matrix; weight i is upsilon_bar / (upsilon_bar + sigma_i)
    with sigma_i the i-th largest singular value, and 1 beyond the rank bound
    min(pixels, L).  The weights come out non-decreasing, as the weighted SVT
    of ``svt`` expects."""
    S = np.linalg.svd(Z, compute_uv=False)          # descending
    w = np.ones(L)
    w[: len(S)] = upsilon_bar / (upsilon_bar + S)
    return w


def nuclear_facets(ny: int, nx: int, qy: int, qx: int, overlap: float):
    """Facet windows [(y0, y1, x0, x1)] of the faceted low-rankness prior:
    tiles at floor(i n / Q) extended on their low side by ceil(overlap * tile),
    clipped at 0 (row-major facet order)."""
    def axis(n, Q):
        b = [(i * n) // Q for i in range(Q + 1)]
        out = []
        for i in range(Q):
            ext = int(math.ceil(overlap * (b[i + 1] - b[i])))
            out.append((max(0, b[i] - ext), b[i + 1]))
        return out
    return [(y0, y1, x0, x1) for (y0, y1) in axis(ny, qy) for (x0, x1) in axis(nx, qx)]


def facet_coverage(ny: int, nx: int, facets) -> np.ndarray:
    cov = np.zeros((ny, nx))
    for y0, y1, x0, x1 in facets:
        cov[y0:y1, x0:x1] += 1.0
    return cov
