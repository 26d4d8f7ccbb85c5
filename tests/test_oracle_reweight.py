"""Pins of the oracle's log-sum reweighting (Sec. 2.2.3) on cubes whose weights
have closed forms, and mutation checks: a plausible mistake planted in the
oracle's weight rules (CPU only) fails one of the pins.

The rules: the l21 weight of coefficient row r is upsilon / (upsilon +
||(Psi^dagger X)_r||_2), the row running over the channels of a sub-cube; the
weight of the i-th largest singular value of facet q is upsilon_bar /
(upsilon_bar + sigma_i(S_q X)), 1 past the rank bound.

* A cube X_l = c_l u (one image u, channel gains c) has rank one on every
  facet: sigma_0 = ||u_q|| ||c||, all other singular values 0, so the nuclear
  weights are [upsilon_bar / (upsilon_bar + ||u_q|| ||c||), 1, ..., 1]; its
  analysis rows are c_l (Psi^dagger u)_r, with norm ||c|| |(Psi^dagger u)_r|,
  and on the Dirac block (the first ny nx coefficients, (1/3) I) that is
  ||c|| u_n / 3, with no transform at all.
* A cube X_l = a_l u + b_l v with u and v on disjoint pixel sets (so
  orthogonal on every facet) and a orthogonal to b has the two singular values
  ||u_q|| ||a|| and ||v_q|| ||b|| on facet q; their order differs from facet to
  facet, which fixes the pairing of weights with singular values.
"""
import numpy as np
import pytest

from oracle import pdfb, prox
from paper_2209_07604_gb300 import synth

UPS, UPS_BAR = 0.5, 0.7          # weights well inside (0, 1) for the values below


def _fhs(L, C, ny=32, nx=48, qy=2, qx=2, overlap=0.2):
    P = synth.make_problem("tiny", L=L, C=C, ny=ny, nx=nx, qy=qy, qx=qx, overlap=overlap)
    steps = pdfb.Steps(tau=0.33, sigma0=0.25, sigma1=1.0, sigma2=1e-3)
    return pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, C, P.qy, P.qx, P.overlap,
                    mu=0.02, mu_bar=0.3, upsilon=UPS, upsilon_bar=UPS_BAR, steps=steps)


def _image(ny, nx, seed, lo=0.5, hi=3.0):
    return np.random.default_rng(seed).uniform(lo, hi, (ny, nx))


def test_rank_one_cube_weights():
    o = _fhs(L=6, C=2)
    ny, nx = o.ny, o.nx
    u = _image(ny, nx, 1)
    gains = np.array([1.3, 0.4, 2.1, 0.9, 0.6, 1.7])
    o.X = gains[:, None, None] * u[None]
    o.reweight()
    a = o.sara.analysis(u[None])[0]
    N = ny * nx
    for c, ch in enumerate(o.chans):
        gc = np.linalg.norm(gains[ch])
        # Dirac block: closed form without any transform
        np.testing.assert_allclose(o.w21[c][:N], UPS / (UPS + gc * u.ravel() / 3.0), rtol=1e-12)
        # all rows: ||c|| |(Psi^dagger u)_r|
        np.testing.assert_allclose(o.w21[c], UPS / (UPS + gc * np.abs(a)), rtol=1e-12)
        for q, (y0, y1, x0, x1) in enumerate(o.facets):
            s0 = np.linalg.norm(u[y0:y1, x0:x1]) * gc
            expect = np.ones(len(ch))
            expect[0] = UPS_BAR / (UPS_BAR + s0)
            np.testing.assert_allclose(o.wnuc[c][q], expect, rtol=1e-10)


def test_rank_two_cube_weight_order():
    """Two singular values per facet whose order changes between facets: the
    smaller weight goes with the larger singular value on each facet."""
    o = _fhs(L=3, C=1, ny=40, nx=40, qy=2, qx=2, overlap=0.1)
    ny, nx = o.ny, o.nx
    yy, xx = np.mgrid[0:ny, 0:nx]
    even = (yy + xx) % 2 == 0
    # u bright on the left half, v bright on the right half: the order of
    # ||u_q|| ||a|| and ||v_q|| ||b|| flips between the facet columns
    u = np.where(even, np.where(xx < nx // 2, 3.0, 0.3), 0.0)
    v = np.where(~even, np.where(xx < nx // 2, 0.3, 3.0), 0.0)
    a = np.array([1.0, 2.0, 2.0]) / 3.0 * 1.2
    b = np.array([2.0, 1.0, -2.0]) / 3.0 * 0.9
    assert abs(a @ b) < 1e-15
    o.X = a[:, None, None] * u[None] + b[:, None, None] * v[None]
    o.reweight()
    orders = set()
    for q, (y0, y1, x0, x1) in enumerate(o.facets):
        su = np.linalg.norm(u[y0:y1, x0:x1]) * np.linalg.norm(a)
        sv = np.linalg.norm(v[y0:y1, x0:x1]) * np.linalg.norm(b)
        s = sorted([su, sv], reverse=True)
        orders.add(su > sv)
        expect = np.array([UPS_BAR / (UPS_BAR + s[0]), UPS_BAR / (UPS_BAR + s[1]), 1.0])
        np.testing.assert_allclose(o.wnuc[0][q], expect, rtol=1e-10)
        assert np.all(np.diff(o.wnuc[0][q]) >= 0)
    assert orders == {True, False}, "the construction must flip the order between facets"
    # Dirac rows of a rank-two cube: sqrt((a_l u_n)^2 + (b_l v_n)^2 summed over l) / 3, u v = 0
    N = ny * nx
    rn = np.sqrt((a @ a) * u.ravel() ** 2 + (b @ b) * v.ravel() ** 2) / 3.0
    np.testing.assert_allclose(o.w21[0][:N], UPS / (UPS + rn), rtol=1e-12)


def test_zero_cube_gives_unit_weights():
    o = _fhs(L=4, C=2)
    o.X[:] = 0.0
    o.reweight()
    for c in range(2):
        np.testing.assert_array_equal(o.w21[c], 1.0)
        for q in range(len(o.facets)):
            np.testing.assert_array_equal(o.wnuc[c][q], 1.0)


# ---------------------------------------------------------------------------
# Mistakes planted in the oracle's weight rules: each must fail a pin above.
# ---------------------------------------------------------------------------

def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_mutation_squared_row_norm(monkeypatch):
    monkeypatch.setattr(prox, "l21_weights", lambda A, ups: ups / (ups + np.sum(A * A, axis=0)))
    assert _fails(test_rank_one_cube_weights)


def test_mutation_relative_upsilon(monkeypatch):
    def rel_ups(A, ups):
        n = np.sqrt(np.sum(A * A, axis=0))
        u = ups * n.max()
        return u / (u + n)
    monkeypatch.setattr(prox, "l21_weights", rel_ups)
    assert _fails(test_rank_one_cube_weights)


def test_mutation_norm_over_coefficients_not_channels(monkeypatch):
    monkeypatch.setattr(prox, "l21_weights",
                        lambda A, ups: np.broadcast_to(ups / (ups + np.sqrt(np.sum(A * A, axis=1))).mean(),
                                                       A.shape[1:]).copy())
    assert _fails(test_rank_one_cube_weights)


def test_mutation_ascending_pairing(monkeypatch):
    def ascending(Z, ups, L):
        S = np.sort(np.linalg.svd(Z, compute_uv=False))
        w = np.ones(L)
        w[: len(S)] = ups / (ups + S)
        return w
    monkeypatch.setattr(prox, "nuclear_weights", ascending)
    assert _fails(test_rank_two_cube_weight_order)


def test_mutation_squared_singular_values(monkeypatch):
    def squared(Z, ups, L):
        S = np.linalg.svd(Z, compute_uv=False)
        w = np.ones(L)
        w[: len(S)] = ups / (ups + S * S)
        return w
    monkeypatch.setattr(prox, "nuclear_weights", squared)
    assert _fails(test_rank_one_cube_weights)
