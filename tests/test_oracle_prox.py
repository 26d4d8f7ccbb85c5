"""Pins of the oracle proximal steps (Eq. 2; Sec. 2.2.2) to closed forms,
variational characterisations and dense SVDs."""
import math
import os

import numpy as np
import pytest
from scipy import optimize

from oracle import prox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_eps_golden():
    with open(os.path.join(GOLDEN, "l2ball_radius.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            M, Mb, e2 = line.split()
            got = prox.eps_blocks(int(M), [int(Mb)])[0] ** 2
            assert abs(got - float(e2)) < 1e-9 * float(e2)


def test_l2ball_projection_characterisation():
    rng = np.random.default_rng(0)
    y = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    eps = 1.5
    z_in = y + 0.1 * (rng.standard_normal(20) + 1j * rng.standard_normal(20))
    assert np.array_equal(prox.proj_l2ball(z_in, y, eps), z_in)
    z = y + 3.0 * (rng.standard_normal(20) + 1j * rng.standard_normal(20))
    p = prox.proj_l2ball(z, y, eps)
    assert abs(np.linalg.norm(p - y) - eps) < 1e-12
    np.testing.assert_allclose(prox.proj_l2ball(p, y, eps), p, atol=1e-14)     # idempotent
    for _ in range(200):                   # obtuse angle with every point of the ball
        q = y + eps * rng.uniform() * (lambda u: u / np.linalg.norm(u))(rng.standard_normal(20) + 1j * rng.standard_normal(20))
        assert np.vdot(z - p, q - p).real <= 1e-10


def test_l2ball_dual_moreau():
    """u+ = z - s proj(z/s) satisfies z = u+ + s proj(z/s) and u+ lies in the
    normal cone: <u+, q - proj> <= 0 for q in the ball."""
    rng = np.random.default_rng(1)
    y = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    v = rng.standard_normal(30) + 1j * rng.standard_normal(30)
    phix = 5 * (rng.standard_normal(30) + 1j * rng.standard_normal(30))
    s, eps = 0.3, 2.0
    u = prox.l2ball_dual(v, phix, y, eps, s)
    p = prox.proj_l2ball((v + s * phix) / s, y, eps)
    np.testing.assert_allclose(u + s * p, v + s * phix, atol=1e-13)
    for _ in range(100):
        d = rng.standard_normal(30) + 1j * rng.standard_normal(30)
        q = y + eps * rng.uniform() * d / np.linalg.norm(d)
        assert np.vdot(u, q - p).real <= 1e-9


def test_l21_dual_against_numerical_prox():
    """Row prox of lam ||.||_2 by direct minimisation vs the closed form used."""
    rng = np.random.default_rng(2)
    Lc, n = 4, 6
    W = rng.standard_normal((Lc, n))
    A = rng.standard_normal((Lc, n))
    wts = rng.uniform(0.2, 1.0, n)
    mu, s = 0.8, 0.7
    U = prox.l21_dual(W, A, s, mu, wts)
    z = W + s * A
    for r in range(n):
        lam = mu * wts[r] / s
        f = lambda t: 0.5 * np.sum((t - z[:, r] / s) ** 2) + lam * np.linalg.norm(t)
        res = optimize.minimize(f, z[:, r] / s, method="Nelder-Mead",
                                options=dict(xatol=1e-12, fatol=1e-14, maxiter=40000))
        np.testing.assert_allclose(U[:, r], z[:, r] - s * res.x, atol=2e-5)
        assert np.linalg.norm(U[:, r]) <= mu * wts[r] + 1e-12


def test_svt_properties():
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((50, 6))
    S = np.linalg.svd(Z, compute_uv=False)
    np.testing.assert_allclose(prox.svt(Z, np.zeros(6)), Z, atol=1e-12)
    thr = np.full(6, 0.5 * (S[2] + S[3]))
    R = prox.svt(Z, thr)
    assert np.linalg.matrix_rank(R, tol=1e-9) == 3
    np.testing.assert_allclose(np.linalg.svd(R, compute_uv=False)[:3], S[:3] - thr[:3], atol=1e-12)
    # Gram route (eigendecomposition of Z^T Z, the route the GPU takes) agrees in FP64
    lam, V = np.linalg.eigh(Z.T @ Z)
    order = np.argsort(lam)[::-1]
    lam, V = lam[order], V[:, order]
    sig = np.sqrt(np.maximum(lam, 0))
    fac = np.maximum(sig - thr, 0) / sig
    np.testing.assert_allclose(Z @ V @ np.diag(fac) @ V.T, R, atol=1e-12)
    # unitary invariance: SVT(Q Z) = Q SVT(Z)
    Qm, _ = np.linalg.qr(rng.standard_normal((50, 50)))
    np.testing.assert_allclose(prox.svt(Qm @ Z, thr), Qm @ R, atol=1e-11)


def test_svt_rank_one_closed_form():
    u = np.array([3.0, 4.0, 0.0]) / 5.0
    v = np.array([1.0, 0.0])
    Z = 7.0 * np.outer(u, v)
    np.testing.assert_allclose(prox.svt(Z, np.array([2.0, 2.0])), 5.0 * np.outer(u, v), atol=1e-14)
    np.testing.assert_allclose(prox.svt(Z, np.array([9.0, 9.0])), 0.0, atol=1e-14)


def test_nuclear_facets_cover_and_overlap():
    f = prox.nuclear_facets(128, 128, 2, 2, 0.1)
    assert f == [(0, 64, 0, 64), (0, 64, 57, 128), (57, 128, 0, 64), (57, 128, 57, 128)]
    cov = prox.facet_coverage(128, 128, f)
    assert cov.min() == 1 and cov.max() == 4
    f2 = prox.nuclear_facets(1024, 1024, 4, 4, 0.1)
    assert (f2[5][1] - f2[5][0]) == 282
