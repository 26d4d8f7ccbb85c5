"""Oracle SARA dictionary and its exact faceted form (Sec. 2.2.2, spatial faceting).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

Readings taken where the paper is silent:

* Psi^dagger = (1/3) [I; W_db1; ...; W_db8]: the Dirac basis and eight
  Daubechies bases (p = 1..8 vanishing moments, 2p taps), each a J-level
  separable 2-D decimated transform (J = 4 by default).  The normalisation
  1/sqrt(9) = 1/3 makes Psi Psi^dagger = I, so ||Psi|| = 1.
* One level along one axis keeps every non-zero sample of the decimated full
  convolution with zero extension: c[k] = sum_i f[i] a[2k+1-i],
  k = 0..floor((n+F-1)/2)-1.  With orthonormal filters this map is an
  isometry (W^T W = I).  The low-pass filter h is the minimum-phase
  (extremal-phase) spectral factor of Daubechies' polynomial; the high-pass
  is g[k] = (-1)^k h[F-1-k].
* 2-D: axis 1 (x) then axis 0 (y); per level the detail subbands are stored
  (y-filter, x-filter) = (lo, hi), (hi, lo), (hi, hi), each row-major, and
  the (lo, lo) band of the last level follows.  The coefficient vector of one
  channel is [Dirac; db1; ...; db8], all scaled by 1/3.
* Faceting: tiles split each axis at floor(i n / Q).  A level-(j+1)
  coefficient k belongs to the facet whose level-j range holds index 2k+1
  (the highest input it touches), so facet ranges map b -> ceil((b-1)/2) and
  the last facet keeps the border coefficients.  A facet reads a window that
  starts far enough below its tile (aligned to 2^J) and ends at its tile's
  upper edge; analysis keeps the owned coefficients, synthesis overlap-adds.
"""
from __future__ import annotations

import math
from math import comb

import numpy as np

N_BASES = 9        # Dirac + db1..db8
SARA_SCALE = 1.0 / 3.0


# ---------------------------------------------------------------------------
# Daubechies filters by spectral factorisation (Daubechies 1988)
# ---------------------------------------------------------------------------

def daubechies(p: int) -> np.ndarray:
    """Low-pass filter of db_p (2p taps), sum = sqrt(2), minimum phase.

    |m0|^2 = cos^{2p}(w/2) P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k.
    Each root y_k of P gives z + 1/z = 2 - 4 y_k; the root of modulus < 1 is a
    zero of H(z) = sum h[n] z^{-n}; the other p zeros sit at z = -1.
    """
    coef = [comb(p - 1 + k, k) for k in range(p)]        # ascending powers of y
    zeros = []
    if p > 1:
        ys = np.roots(coef[::-1])
        for yk in ys:
            b = 2.0 - 4.0 * yk
            disc = np.sqrt(b * b - 4.0 + 0j)
            z1, z2 = (b + disc) / 2.0, (b - disc) / 2.0
            zeros.append(z1 if abs(z1) < 1.0 else z2)
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, [1.0, 1.0])
    for z in zeros:
        poly = np.convolve(poly, [1.0, -z])
    h = np.real(poly)
    return h * (math.sqrt(2.0) / h.sum())


def highpass(h: np.ndarray) -> np.ndarray:
    F = len(h)
    return np.array([(-1) ** k * h[F - 1 - k] for k in range(F)])


# ---------------------------------------------------------------------------
# One level, one axis
# ---------------------------------------------------------------------------

def out_len(n: int, F: int) -> int:
    return (n + F - 1) // 2


def analysis_axis(a: np.ndarray, f: np.ndarray, axis: int) -> np.ndarray:
    """c[k] = sum_i f[i] a[2k+1-i] along ``axis`` (zero outside [0, n))."""
    a = np.moveaxis(a, axis, -1)
    n, F = a.shape[-1], len(f)
    m = out_len(n, F)
    k = np.arange(m)
    out = np.zeros(a.shape[:-1] + (m,), dtype=a.dtype)
    for i in range(F):
        idx = 2 * k + 1 - i
        ok = (idx >= 0) & (idx < n)
        out[..., ok] += f[i] * a[..., idx[ok]]
    return np.moveaxis(out, -1, axis)


def synthesis_axis(c: np.ndarray, f: np.ndarray, n: int, axis: int) -> np.ndarray:
    """Adjoint of ``analysis_axis``: a[2k+1-i] += f[i] c[k], kept on [0, n)."""
    c = np.moveaxis(c, axis, -1)
    m, F = c.shape[-1], len(f)
    k = np.arange(m)
    out = np.zeros(c.shape[:-1] + (n,), dtype=c.dtype)
    for i in range(F):
        idx = 2 * k + 1 - i
        ok = (idx >= 0) & (idx < n)
        out[..., idx[ok]] += f[i] * c[..., ok]
    return np.moveaxis(out, -1, axis)


# ---------------------------------------------------------------------------
# Multi-level 2-D transform of one basis
# ---------------------------------------------------------------------------

def level_shapes(ny: int, nx: int, F: int, levels: int):
    """[(n_y^j, n_x^j)] for j = 0..levels."""
    shapes = [(ny, nx)]
    for _ in range(levels):
        a, b = shapes[-1]
        shapes.append((out_len(a, F), out_len(b, F)))
    return shapes


def dwt2(a: np.ndarray, h: np.ndarray, levels: int):
    """Multi-level analysis of the last two axes: list of per-level
    (lh, hl, hh) detail triplets and the final ll band."""
    g = highpass(h)
    details = []
    for _ in range(levels):
        lo_x = analysis_axis(a, h, -1)
        hi_x = analysis_axis(a, g, -1)
        ll = analysis_axis(lo_x, h, -2)
        lh = analysis_axis(hi_x, h, -2)       # y lo, x hi
        hl = analysis_axis(lo_x, g, -2)       # y hi, x lo
        hh = analysis_axis(hi_x, g, -2)
        details.append((lh, hl, hh))
        a = ll
    return details, a


def idwt2(details, ll: np.ndarray, h: np.ndarray, ny: int, nx: int) -> np.ndarray:
    """Adjoint of ``dwt2`` (exact inverse on the range)."""
    g = highpass(h)
    F = len(h)
    shapes = level_shapes(ny, nx, F, len(details))
    a = ll
    for j in range(len(details) - 1, -1, -1):
        lh, hl, hh = details[j]
        n0, n1 = shapes[j]
        lo_x = synthesis_axis(a, h, n0, -2) + synthesis_axis(hl, g, n0, -2)
        hi_x = synthesis_axis(lh, h, n0, -2) + synthesis_axis(hh, g, n0, -2)
        a = synthesis_axis(lo_x, h, n1, -1) + synthesis_axis(hi_x, g, n1, -1)
    return a


def flatten_basis(details, ll) -> np.ndarray:
    parts = []
    for lh, hl, hh in details:
        for band in (lh, hl, hh):
            parts.append(band.reshape(band.shape[:-2] + (-1,)))
    parts.append(ll.reshape(ll.shape[:-2] + (-1,)))
    return np.concatenate(parts, axis=-1)


def unflatten_basis(vec: np.ndarray, ny: int, nx: int, F: int, levels: int):
    shapes = level_shapes(ny, nx, F, levels)
    lead = vec.shape[:-1]
    pos = 0
    details = []
    for j in range(1, levels + 1):
        my, mx = shapes[j]
        trip = []
        for _ in range(3):
            trip.append(vec[..., pos: pos + my * mx].reshape(lead + (my, mx)))
            pos += my * mx
        details.append(tuple(trip))
    my, mx = shapes[levels]
    ll = vec[..., pos: pos + my * mx].reshape(lead + (my, mx))
    pos += my * mx
    assert pos == vec.shape[-1]
    return details, ll


def basis_size(ny: int, nx: int, F: int, levels: int) -> int:
    shapes = level_shapes(ny, nx, F, levels)
    return sum(3 * a * b for a, b in shapes[1:]) + shapes[-1][0] * shapes[-1][1]


# ---------------------------------------------------------------------------
# SARA: Psi^dagger and Psi
# ---------------------------------------------------------------------------

class Sara:
    """Psi^dagger x = (1/3)[x; W_db1 x; ...; W_db8 x] for images (..., ny, nx)."""

    def __init__(self, ny: int, nx: int, levels: int = 4, n_db: int = 8):
        self.ny, self.nx, self.levels = ny, nx, levels
        self.filters = [daubechies(p) for p in range(1, n_db + 1)]
        self.sizes = [ny * nx] + [basis_size(ny, nx, len(h), levels) for h in self.filters]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        self.n_coef = int(self.offsets[-1])

    def analysis(self, x: np.ndarray) -> np.ndarray:
        lead = x.shape[:-2]
        parts = [x.reshape(lead + (-1,))]
        for h in self.filters:
            parts.append(flatten_basis(*dwt2(x, h, self.levels)))
        return SARA_SCALE * np.concatenate(parts, axis=-1)

    def synthesis(self, c: np.ndarray) -> np.ndarray:
        lead = c.shape[:-1]
        o = self.offsets
        out = c[..., o[0]:o[1]].reshape(lead + (self.ny, self.nx)).copy()
        for b, h in enumerate(self.filters, start=1):
            det, ll = unflatten_basis(c[..., o[b]:o[b + 1]], self.ny, self.nx, len(h), self.levels)
            out += idwt2(det, ll, h, self.ny, self.nx)
        return SARA_SCALE * out


# ---------------------------------------------------------------------------
# Exact faceted SARA (Prusa 2012, Ch. 4, as used in Sec. 2.2.2)
# ---------------------------------------------------------------------------

def tile_bounds(n: int, Q: int) -> list:
    return [(i * n) // Q for i in range(Q + 1)]


def owner_bounds(n: int, Q: int, F: int, levels: int) -> list:
    """Per level j = 0..levels, the facet boundaries B^j_0..B^j_Q along one axis."""
    b = tile_bounds(n, Q)
    out = [b]
    n_j = n
    for _ in range(levels):
        n_j = out_len(n_j, F)
        prev = out[-1]
        nb = [0] + [-(-(prev[i] - 1) // 2) for i in range(1, Q)] + [n_j]
        out.append(nb)
    return out


def facet_window(n: int, Q: int, i: int, F: int, levels: int) -> tuple:
    """[s, e) pixel window read by facet i: its tile extended downwards by
    F * 2^levels samples, start aligned to a multiple of 2^levels."""
    b = tile_bounds(n, Q)
    step = 1 << levels
    s = max(0, b[i] - F * step)
    s = (s // step) * step
    return s, b[i + 1]


class FacetedSara(Sara):
    """Psi^dagger and Psi computed facet by facet on a Qy x Qx tiling."""

    def __init__(self, ny, nx, qy, qx, levels=4, n_db=8):
        super().__init__(ny, nx, levels, n_db)
        self.qy, self.qx = qy, qx

    def _facet_basis_analysis(self, x, h):
        F, J = len(h), self.levels
        gshapes = level_shapes(self.ny, self.nx, F, J)
        obY = owner_bounds(self.ny, self.qy, F, J)
        obX = owner_bounds(self.nx, self.qx, F, J)
        lead = x.shape[:-2]
        gdet = [tuple(np.zeros(lead + gshapes[j]) for _ in range(3)) for j in range(1, J + 1)]
        gll = np.zeros(lead + gshapes[J])
        for iy in range(self.qy):
            sy, ey = facet_window(self.ny, self.qy, iy, F, J)
            for ix in range(self.qx):
                sx, ex = facet_window(self.nx, self.qx, ix, F, J)
                det, ll = dwt2(x[..., sy:ey, sx:ex], h, J)
                for j in range(1, J + 1):
                    oy, ox = sy >> j, sx >> j
                    y0, y1 = obY[j][iy], obY[j][iy + 1]
                    x0, x1 = obX[j][ix], obX[j][ix + 1]
                    for band in range(3):
                        gdet[j - 1][band][..., y0:y1, x0:x1] = \
                            det[j - 1][band][..., y0 - oy:y1 - oy, x0 - ox:x1 - ox]
                    if j == J:
                        gll[..., y0:y1, x0:x1] = ll[..., y0 - oy:y1 - oy, x0 - ox:x1 - ox]
        return gdet, gll

    def analysis(self, x):
        lead = x.shape[:-2]
        parts = [x.reshape(lead + (-1,))]
        for h in self.filters:
            parts.append(flatten_basis(*self._facet_basis_analysis(x, h)))
        return SARA_SCALE * np.concatenate(parts, axis=-1)

    def synthesis(self, c):
        lead = c.shape[:-1]
        o = self.offsets
        out = c[..., o[0]:o[1]].reshape(lead + (self.ny, self.nx)).copy()
        for b, h in enumerate(self.filters, start=1):
            F, J = len(h), self.levels
            gdet, gll = unflatten_basis(c[..., o[b]:o[b + 1]], self.ny, self.nx, F, J)
            obY = owner_bounds(self.ny, self.qy, F, J)
            obX = owner_bounds(self.nx, self.qx, F, J)
            for iy in range(self.qy):
                sy, ey = facet_window(self.ny, self.qy, iy, F, J)
                for ix in range(self.qx):
                    sx, ex = facet_window(self.nx, self.qx, ix, F, J)
                    lsh = level_shapes(ey - sy, ex - sx, F, J)
                    det = []
                    for j in range(1, J + 1):
                        oy, ox = sy >> j, sx >> j
                        y0, y1 = obY[j][iy], obY[j][iy + 1]
                        x0, x1 = obX[j][ix], obX[j][ix + 1]
                        trip = []
                        for band in range(3):
                            loc = np.zeros(lead + lsh[j])
                            loc[..., y0 - oy:y1 - oy, x0 - ox:x1 - ox] = gdet[j - 1][band][..., y0:y1, x0:x1]
                            trip.append(loc)
                        det.append(tuple(trip))
                        if j == J:
                            ll = np.zeros(lead + lsh[J])
                            ll[..., y0 - oy:y1 - oy, x0 - ox:x1 - ox] = gll[..., y0:y1, x0:x1]
                    out[..., sy:ey, sx:ex] += idwt2(det, ll, h, ey - sy, ex - sx)
        return SARA_SCALE * out
