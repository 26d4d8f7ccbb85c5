"""Oracle measurement operator Phi_l = Theta_l G_l F Z (Sec. 2.1, Eq. 1).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

Conventions (the paper leaves them open; these are the readings used):

* pixel n = (n1, n2), n_d in [-N_d/2, N_d/2); array index i_d = n_d + N_d/2;
  axis 0 is y (rows, n1), axis 1 is x (columns, n2).
* the exact operator is (A x)_m = sum_n x_n c_m(n) exp(-i (w1 n1 + w2 n2)),
  omega_m = (w1, w2) in radians per pixel, c_m the w-term chirp
  exp(i pi w_m dl^2 (n1^2 + n2^2)) of the small-field approximation (Sec. 3.2).
* Z: multiply by s_1(n1) s_2(n2) and place at grid index (n mod K_d),
  K_d = 2 N_d (2x oversampling per dimension).
* F: unnormalised K1 x K2 DFT, exp(-2 pi i k n / K).
* G: row m holds, per dimension, the J = 7 Kaiser-Bessel samples
  phi(kappa - k) at the J integers k nearest kappa = omega K / (2 pi),
  discretely convolved with the truncated w-kernel; the 2-D row is the outer
  product of the two 1-D rows; columns wrap modulo K.
* phi(t) = I0(beta sqrt(1 - (2t/J)^2)) / I0(beta), |t| <= J/2, with
  beta = pi sqrt((J/os)^2 (os - 1/2)^2 - 0.8), os = 2 (Beatty et al. 2005);
  s_d(n) = 1 / phi_hat(n / K_d), phi_hat the continuous Fourier transform.
* Theta_l: natural weighting, G rows and y divided by sigma_l.
* w-projection: w is quantised to planes w_p = p * w_max / (P - 1); the
  kernel of a plane is the K-point DFT of the chirp exp(i pi w_p dl^2 psi(n)),
  psi(n) = n^2 on the image and smoothly extended over the padding
  (``chirp_phase``), truncated to 2h+1 taps, h = round(4 |p| / (P - 1)), and
  renormalised to unit sum (h = 0 gives the plain NUFFT row).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass(frozen=True)
class Geometry:
    ny: int
    nx: int
    J: int = 7
    oversample: float = 2.0
    w_max: float = 0.0
    n_wplanes: int = 64
    pixel_size: float = 0.0

    @property
    def K1(self) -> int:
        return int(round(self.oversample * self.ny))

    @property
    def K2(self) -> int:
        return int(round(self.oversample * self.nx))

    @property
    def beta(self) -> float:
        J, os_ = self.J, self.oversample
        return math.pi * math.sqrt((J / os_) ** 2 * (os_ - 0.5) ** 2 - 0.8)


def kb(t, J: int, beta: float):
    """Kaiser-Bessel kernel phi(t), zero outside |t| <= J/2."""
    t = np.asarray(t, dtype=np.float64)
    r = 1.0 - (2.0 * t / J) ** 2
    out = np.zeros_like(t)
    ok = r >= 0
    out[ok] = np.i0(beta * np.sqrt(r[ok])) / np.i0(beta)
    return out


def kb_hat(nu, J: int, beta: float):
    """Continuous Fourier transform of phi at frequency nu (cycles per cell):
    J sinh(sqrt(beta^2 - (pi J nu)^2)) / (sqrt(.) I0(beta)), sin form past the
    zero of the square root (Jackson et al. 1991)."""
    nu = np.asarray(nu, dtype=np.float64)
    z2 = beta * beta - (math.pi * J * nu) ** 2
    out = np.empty_like(nu)
    pos = z2 > 0
    z = np.sqrt(np.abs(z2))
    out[pos] = np.sinh(z[pos]) / z[pos]
    neg = z2 < 0
    out[neg] = np.sin(z[neg]) / z[neg]
    out[z2 == 0] = 1.0
    return J * out / np.i0(beta)


def scaling(N: int, K: int, J: int, beta: float) -> np.ndarray:
    """Diagonal of Z's scaling along one axis, indexed by i = n + N/2."""
    n = np.arange(N) - N // 2
    return 1.0 / kb_hat(n / K, J, beta)


def wplane(w: np.ndarray, geom: Geometry):
    """Plane index p, plane w_p and kernel half-width h of each visibility."""
    w = np.asarray(w, dtype=np.float64)
    if geom.w_max <= 0.0:
        z = np.zeros(w.shape, dtype=np.int64)
        return z, np.zeros(w.shape), z
    P1 = geom.n_wplanes - 1
    dw = geom.w_max / P1
    p = np.floor(np.abs(w) / dw + 0.5).astype(np.int64)
    p = np.minimum(p, P1) * np.where(w < 0, -1, 1)
    wp = p * dw
    h = (8 * np.abs(p) + P1) // (2 * P1)           # round(4 |p| / P1) in integers
    return p, wp, h


def chirp_phase(N: int, K: int) -> np.ndarray:
    """psi(n) for n = -K/2..K/2-1: n^2 on the image support |n| <= N/2; on the
    zero-padded part its slope falls linearly from N to 0 at |n| = K/2, so the
    extended chirp is smooth across the periodic wrap of the grid."""
    n = np.abs(np.arange(K, dtype=np.float64) - K // 2)
    hN, hK = N / 2.0, K / 2.0
    out = n * n
    pad = n > hN
    t = n[pad]
    out[pad] = hN * hN + N / (hK - hN) * (hK * (t - hN) - 0.5 * (t * t - hN * hN))
    return out


def wkernel(wp: float, N: int, K: int, pixel_size: float, j_lo: int, j_hi: int) -> np.ndarray:
    """DFT coefficients chat(j) = (1/K) sum_n exp(i pi a psi(n)) exp(-2 pi i j n / K),
    a = w_p dl^2, n over the whole K grid, for j = j_lo..j_hi.  On the image
    support the chirp equals the w-term exp(i pi w dl^2 n^2); elsewhere the
    image is zero, so any extension gives the same exact (untruncated) row."""
    n = np.arange(K, dtype=np.float64) - K // 2
    chirp = np.exp(1j * math.pi * wp * pixel_size ** 2 * chirp_phase(N, K))
    j = np.arange(j_lo, j_hi + 1, dtype=np.float64)
    return (np.exp(-2j * math.pi * np.outer(j, n) / K) @ chirp) / K


def _rows_1d(kappa: np.ndarray, K: int, J: int, beta: float, ck: np.ndarray, j_lo: int):
    """1-D rows: first column c = p0 - j_hi (p0 the first KB tap) and values
    g(t) = sum_j chat(j) phi(kappa - (c + t + j)), t = 0..J+S-2."""
    p0 = np.floor(kappa - J / 2.0).astype(np.int64) + 1
    taps = kb(kappa[:, None] - (p0[:, None] + np.arange(J)[None, :]), J, beta)  # (m, J)
    S = len(ck)
    T = J + S - 1
    g = np.zeros((len(kappa), T), dtype=np.complex128)
    # Tap i sits at column p0 + i; kernel entry jj stands for j = j_lo + jj and
    # moves it to column k = p0 + i - j, i.e. offset t = i - jj + S - 1 from
    # the corner c = p0 - (S - 1) - j_lo.
    for jj in range(S):
        for i in range(J):
            g[:, i - jj + (S - 1)] += ck[jj] * taps[:, i]
    corner = p0 - (S - 1) - j_lo
    return corner, g


def g_rows(omega: np.ndarray, w: np.ndarray, geom: Geometry, full_wkernel: bool = False):
    """Rows of G for visibilities (omega (M,2), w (M,)), before whitening.

    Returns a list of (index array, corner1, corner2, g1, g2): for visibilities
    ``idx`` sharing one w-plane, row value at grid (corner1 + t1, corner2 + t2)
    (mod K) is g1[:, t1] * g2[:, t2].
    """
    K1, K2, J, beta = geom.K1, geom.K2, geom.J, geom.beta
    kap1 = omega[:, 0] * K1 / (2.0 * math.pi)
    kap2 = omega[:, 1] * K2 / (2.0 * math.pi)
    p, wp, h = wplane(w, geom)
    out = []
    for pv in np.unique(p):
        idx = np.nonzero(p == pv)[0]
        wpv = float(wp[idx[0]])
        hv = int(h[idx[0]])
        ks = []
        for N, K in ((geom.ny, K1), (geom.nx, K2)):
            if full_wkernel:
                j_lo, j_hi = -(K // 2), K - K // 2 - 1
                ck = wkernel(wpv, N, K, geom.pixel_size, j_lo, j_hi)
            else:
                j_lo, j_hi = -hv, hv
                ck = wkernel(wpv, N, K, geom.pixel_size, j_lo, j_hi) if hv > 0 else np.ones(1, complex)
                ck = ck / ck.sum()
            ks.append((ck, j_lo))
        c1, g1 = _rows_1d(kap1[idx], K1, J, beta, *ks[0])
        c2, g2 = _rows_1d(kap2[idx], K2, J, beta, *ks[1])
        out.append((idx, c1, c2, g1, g2))
    return out


DDE_TAPS = 5            # DDE kernels: S x S taps in grid units, centred (offsets -2..2)


def dde_convolve(box: np.ndarray, dde: np.ndarray) -> np.ndarray:
    """Full 2-D convolution of row boxes (n, T1, T2) with DDE kernels (n, S, S):
    out[a + j1, b + j2] += D[j1, j2] box[a, b] (Sec. 3.1: the row of G is the
    convolution of the DDE Fourier kernel with the interpolation kernel)."""
    n, T1, T2 = box.shape
    S = dde.shape[1]
    out = np.zeros((n, T1 + S - 1, T2 + S - 1), dtype=np.complex128)
    for j1 in range(S):
        for j2 in range(S):
            out[:, j1:j1 + T1, j2:j2 + T2] += dde[:, j1, j2, None, None] * box
    return out


def build_G(omega: np.ndarray, w: np.ndarray, sigma: float, geom: Geometry,
            full_wkernel: bool = False, dde: np.ndarray | None = None) -> sp.csr_matrix:
    """Whitened degridding matrix Theta G (M x K1*K2, complex128, CSR).  With
    ``dde`` (M, S, S) every row is further convolved with its visibility's DDE
    kernel (centred: the box grows by (S-1)/2 on each side)."""
    M = omega.shape[0]
    K1, K2 = geom.K1, geom.K2
    rows, cols, vals = [], [], []
    for idx, c1, c2, g1, g2 in g_rows(omega, w, geom, full_wkernel):
        box = g1[:, :, None] * g2[:, None, :]
        if dde is not None:
            box = dde_convolve(box, dde[idx])
            h = (dde.shape[1] - 1) // 2
            c1, c2 = c1 - h, c2 - h
        T1, T2 = box.shape[1], box.shape[2]
        k1 = (c1[:, None] + np.arange(T1)[None, :]) % K1
        k2 = (c2[:, None] + np.arange(T2)[None, :]) % K2
        col = (k1[:, :, None] * K2 + k2[:, None, :]).reshape(len(idx), -1)
        val = box.reshape(len(idx), -1)
        rows.append(np.repeat(idx, T1 * T2))
        cols.append(col.ravel())
        vals.append(val.ravel())
    G = sp.coo_matrix((np.concatenate(vals) / sigma, (np.concatenate(rows), np.concatenate(cols))),
                      shape=(M, K1 * K2)).tocsr()
    G.sum_duplicates()
    return G


class Operator:
    """Phi_l for every channel of a problem: G matrices, scaling, FFT."""

    def __init__(self, omega, w, sigma, geom: Geometry, full_wkernel: bool = False, dde=None):
        self.geom = geom
        self.L = omega.shape[0]
        self.G = [build_G(omega[l], w[l], float(sigma[l]), geom, full_wkernel,
                          None if dde is None else dde[l]) for l in range(self.L)]
        self.s1 = scaling(geom.ny, geom.K1, geom.J, geom.beta)
        self.s2 = scaling(geom.nx, geom.K2, geom.J, geom.beta)
        self.i1 = (np.arange(geom.ny) - geom.ny // 2) % geom.K1
        self.i2 = (np.arange(geom.nx) - geom.nx // 2) % geom.K2

    def fzx(self, x: np.ndarray) -> np.ndarray:
        """F Z x for one channel image (ny, nx), real or complex -> (K1, K2) complex grid."""
        g = np.zeros((self.geom.K1, self.geom.K2), dtype=np.complex128)
        g[np.ix_(self.i1, self.i2)] = x * self.s1[:, None] * self.s2[None, :]
        return np.fft.fft2(g)

    def zf_adj(self, grid: np.ndarray) -> np.ndarray:
        """Re(Z^T F^H grid): adjoint of fzx restricted to real images."""
        K1, K2 = self.geom.K1, self.geom.K2
        img = np.fft.ifft2(grid) * (K1 * K2)
        return np.real(img[np.ix_(self.i1, self.i2)]) * self.s1[:, None] * self.s2[None, :]

    def forward(self, x: np.ndarray, l: int) -> np.ndarray:
        return self.G[l] @ self.fzx(x).ravel()

    def adjoint(self, v: np.ndarray, l: int) -> np.ndarray:
        grid = (self.G[l].conj().T @ v).reshape(self.geom.K1, self.geom.K2)
        return self.zf_adj(grid)

    def forward_all(self, X: np.ndarray) -> list:
        return [self.forward(X[l], l) for l in range(self.L)]

    def adjoint_all(self, V: list) -> np.ndarray:
        return np.stack([self.adjoint(V[l], l) for l in range(self.L)])

    def norm2_eigsh(self, l: int, tol: float = 1e-12) -> float:
        """||Phi_l||^2 as the largest eigenvalue of Re(Phi_l^H Phi_l), by ARPACK's
        implicitly restarted Lanczos (scipy ``eigsh``) on the FP64 operator."""
        from scipy.sparse.linalg import LinearOperator, eigsh
        ny, nx = self.geom.ny, self.geom.nx
        n = ny * nx

        def mv(x):
            return np.asarray(self.adjoint(self.forward(np.asarray(x).reshape(ny, nx), l), l)).ravel()

        A = LinearOperator((n, n), matvec=mv, dtype=np.float64)
        v0 = np.random.default_rng(0).standard_normal(n)
        return float(eigsh(A, k=1, which="LA", tol=tol, v0=v0, return_eigenvectors=False)[0])

    def norm2(self, l: int, n_iter: int = 200, tol: float = 1e-10, seed: int = 0) -> float:
        """||Phi_l||^2 by power iteration on Re(Phi_l^H Phi_l)."""
        rng = np.random.default_rng(seed)
        x = rng.standard_normal((self.geom.ny, self.geom.nx))
        x /= np.linalg.norm(x)
        lam = 0.0
        for _ in range(n_iter):
            y = self.adjoint(self.forward(x, l), l)
            lam_new = float(np.vdot(x, y).real)
            x = y / np.linalg.norm(y)
            if abs(lam_new - lam) <= tol * abs(lam_new):
                return lam_new
            lam = lam_new
        return lam


def nudft(x: np.ndarray, omega: np.ndarray, w: np.ndarray | None = None,
          pixel_size: float = 0.0) -> np.ndarray:
    """Brute-force direct transform sum_n x_n exp(i pi w dl^2 |n|^2) exp(-i omega . n)."""
    ny, nx = x.shape
    n1 = np.arange(ny) - ny // 2
    n2 = np.arange(nx) - nx // 2
    N1, N2 = np.meshgrid(n1, n2, indexing="ij")
    n1f, n2f, xf = N1.ravel(), N2.ravel(), x.ravel()
    out = np.empty(omega.shape[0], dtype=np.complex128)
    for m in range(omega.shape[0]):
        ph = -(omega[m, 0] * n1f + omega[m, 1] * n2f)
        if w is not None:
            ph = ph + math.pi * w[m] * pixel_size ** 2 * (n1f ** 2 + n2f ** 2)
        out[m] = np.sum(xf * np.exp(1j * ph))
    return out
