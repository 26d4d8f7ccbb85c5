"""Pins of the oracle measurement operator (Sec. 2.1, Eq. 1; Sec. 3.2) to
things other than itself: a brute-force direct Fourier transform, quadrature,
dense linear algebra and exact special cases."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import nufft as nf


def _uv(M, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, (M, 2))


@pytest.mark.parametrize("ny,nx", [(32, 32), (24, 40), (18, 30)])
def test_nufft_matches_direct_transform(ny, nx):
    """Phi (w = 0) against sum_n x_n exp(-i omega.n): the 7-tap KB NUFFT with
    2x oversampling approximates the direct transform to ~1e-6."""
    geom = nf.Geometry(ny, nx)
    om = _uv(250, 1)
    op = nf.Operator(om[None], np.zeros((1, 250)), np.ones(1), geom)
    x = np.random.default_rng(2).standard_normal((ny, nx))
    a = op.forward(x, 0)
    b = nf.nudft(x, om)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


def test_full_wkernel_matches_direct_transform_with_wterm():
    """With the untruncated w-kernel the row equals the NUFFT of x times the
    chirp exp(i pi w dl^2 |n|^2) exactly, so it matches the direct transform
    with the w-phase to the NUFFT accuracy (Sec. 3.2)."""
    ny, nx = 32, 24
    geom = nf.Geometry(ny, nx, w_max=2000.0, n_wplanes=16, pixel_size=math.sqrt(2 / 2000) / 32)
    M = 150
    om = _uv(M, 3)
    w = np.random.default_rng(4).uniform(-2000, 2000, M)
    _, wp, _ = nf.wplane(w, geom)
    x = np.random.default_rng(5).standard_normal((ny, nx))
    op = nf.Operator(om[None], w[None], np.ones(1), geom, full_wkernel=True)
    b = nf.nudft(x, om, wp, geom.pixel_size)
    assert np.linalg.norm(op.forward(x, 0) - b) / np.linalg.norm(b) < 1e-5
    # the truncated (7..15 taps) kernel is an approximation: reported, and it
    # must at least beat ignoring the w-term
    opt = nf.Operator(om[None], w[None], np.ones(1), geom)
    err_t = np.linalg.norm(opt.forward(x, 0) - b) / np.linalg.norm(b)
    err_0 = np.linalg.norm(nf.nudft(x, om) - b) / np.linalg.norm(b)
    assert err_t < 0.5 * err_0
    T = np.diff(opt.G[0].indptr)
    assert set(np.unique(T)) <= {49, 81, 121, 169, 225}


def test_w_zero_rows_equal_plain_kb_rows():
    geom0 = nf.Geometry(32, 32)
    geomw = nf.Geometry(32, 32, w_max=2000.0, n_wplanes=16, pixel_size=1e-3)
    om = _uv(100, 6)
    G0 = nf.build_G(om, np.zeros(100), 1.0, geom0)
    Gw = nf.build_G(om, np.zeros(100), 1.0, geomw)
    assert abs(G0 - Gw).max() == 0.0
    assert np.all(np.diff(G0.indptr) == 49)


def test_wplane_support_rule():
    geom = nf.Geometry(64, 64, w_max=2000.0, n_wplanes=64, pixel_size=1e-4)
    w = np.array([0.0, 15.0, 16.5, 300.0, 1000.0, 1999.0, 2000.0, -2000.0, 5000.0])
    p, wp, h = nf.wplane(w, geom)
    dw = 2000.0 / 63
    assert list(p) == [0, 0, 1, 9, 32, 63, 63, -63, 63]
    np.testing.assert_allclose(wp, p * dw)
    # h = round(4 |p| / 63)
    assert list(h) == [int(math.floor(4 * abs(q) / 63 + 0.5)) for q in p]


def test_kb_hat_is_fourier_transform_of_kb():
    """Closed-form phi_hat against numerical quadrature of phi."""
    geom = nf.Geometry(64, 64)
    J, beta = geom.J, geom.beta
    for nu in [0.0, 0.05, 0.2, 0.37, 0.5]:
        val, _ = integrate.quad(lambda t: nf.kb(np.array([t]), J, beta)[0] * math.cos(2 * math.pi * nu * t),
                                -J / 2, J / 2, epsabs=1e-13, epsrel=1e-13, limit=200)
        assert abs(nf.kb_hat(np.array([nu]), J, beta)[0] - val) < 1e-10 * max(1.0, abs(val))


def test_beta_value():
    # beta = pi sqrt((J/2)^2 (3/2)^2 - 0.8) for J = 7, oversampling 2
    assert abs(nf.Geometry(8, 8).beta - math.pi * math.sqrt(3.5 ** 2 * 1.5 ** 2 - 0.8)) < 1e-15


def test_adjoint_identity():
    geom = nf.Geometry(40, 24, w_max=2000.0, n_wplanes=8, pixel_size=1e-3)
    M = 300
    om = _uv(M, 7)
    w = np.random.default_rng(8).uniform(0, 2000, M)
    op = nf.Operator(om[None], w[None], np.array([0.7]), geom)
    rng = np.random.default_rng(9)
    x = rng.standard_normal((40, 24))
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    lhs = np.vdot(v, op.forward(x, 0)).real
    rhs = np.vdot(op.adjoint(v, 0), x).real
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_power_iteration_matches_dense_svd():
    """||Phi||^2 by power iteration against the largest singular value of the
    explicit real matrix [Re Phi; Im Phi]."""
    ny, nx, M = 12, 16, 60
    geom = nf.Geometry(ny, nx)
    om = _uv(M, 10)
    op = nf.Operator(om[None], np.zeros((1, M)), np.array([1.3]), geom)
    cols = []
    for k in range(ny * nx):
        e = np.zeros(ny * nx)
        e[k] = 1.0
        cols.append(op.forward(e.reshape(ny, nx), 0))
    A = np.array(cols).T
    Ar = np.vstack([A.real, A.imag])
    smax = np.linalg.svd(Ar, compute_uv=False)[0]
    # real images pair the singular values, so the gap is small: iterate long
    assert abs(op.norm2(0, n_iter=20000, tol=0.0) - smax ** 2) < 1e-8 * smax ** 2
    # the Lanczos (ARPACK) estimate reaches the same value directly
    assert abs(op.norm2_eigsh(0) - smax ** 2) < 1e-10 * smax ** 2


def test_psf_peaks_at_phase_centre():
    """Phi^H Phi delta (the dirty beam) is maximal at the phase centre, where
    it equals ||Phi delta||^2 (Sec. 5.3 normalisation)."""
    ny, nx = 32, 32
    geom = nf.Geometry(ny, nx)
    om = _uv(400, 11)
    op = nf.Operator(om[None], np.zeros((1, 400)), np.ones(1), geom)
    d = np.zeros((ny, nx))
    d[ny // 2, nx // 2] = 1.0
    psf = op.adjoint(op.forward(d, 0), 0)
    assert np.unravel_index(np.argmax(psf), psf.shape) == (ny // 2, nx // 2)
    assert abs(psf.max() - np.linalg.norm(op.forward(d, 0)) ** 2) < 1e-9 * psf.max()
    # and the direct transform of delta has unit modulus at every uv point
    assert np.allclose(np.abs(op.forward(d, 0)), 1.0, atol=1e-5)


def test_dde_rows_equal_image_modulation():
    """A row convolved with a centred 5x5 DDE kernel D_m (Sec. 3.1) and applied to
    F Z x equals the plain row applied to F Z (d_m x), with the image-domain
    modulation d_m(n) = sum_delta D_m[delta + 2] exp(-2 pi i (delta1 n1 / K1 + delta2 n2 / K2)):
    a convolution in the grid is a product in the image.  A centred delta
    kernel leaves G unchanged; the DDE operator keeps the adjoint identity."""
    ny, nx, M = 12, 16, 25
    geom = nf.Geometry(ny, nx)
    om = _uv(M, 21)
    rng = np.random.default_rng(7)
    dde = rng.standard_normal((M, 5, 5)) + 1j * rng.standard_normal((M, 5, 5))
    op = nf.Operator(om[None], np.zeros((1, M)), np.array([1.3]), geom)
    opd = nf.Operator(om[None], np.zeros((1, M)), np.array([1.3]), geom, dde=dde[None])
    x = rng.standard_normal((ny, nx))
    got = opd.forward(x, 0)
    n1 = (np.arange(ny) - ny // 2)[:, None]
    n2 = (np.arange(nx) - nx // 2)[None, :]
    for m in range(M):
        d = sum(dde[m, a, b] * np.exp(-2j * np.pi * ((a - 2) * n1 / geom.K1 + (b - 2) * n2 / geom.K2))
                for a in range(5) for b in range(5))
        ref = op.forward(d * x, 0)[m]
        assert abs(got[m] - ref) < 1e-12 * max(1.0, abs(ref))
    delta = np.zeros((1, M, 5, 5), dtype=np.complex128)
    delta[:, :, 2, 2] = 1.0
    op1 = nf.Operator(om[None], np.zeros((1, M)), np.array([1.3]), geom, dde=delta)
    assert abs(op1.G[0] - op.G[0]).max() < 1e-15
    v = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    assert abs(np.vdot(v, opd.forward(x, 0)).real - np.vdot(opd.adjoint(v, 0), x).real) < 1e-12 * np.linalg.norm(v) * np.linalg.norm(got)
