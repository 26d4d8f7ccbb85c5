"""Pins of the oracle PDFB iteration (Eq. 2-3, Sec. 2.2.3) and mutation
checks showing that a plausible mistake planted in the oracle fails a pin."""
import math

import numpy as np
import pytest

from oracle import nufft as nf
from oracle import pdfb, prox, wavelets as wv
from paper_2209_07604_gb300 import synth

import test_oracle_nufft as tn
import test_oracle_prox as tp
import test_oracle_sara as ts


def _feasible_problem(seed=0, ny=16, nx=16, L=2, M=300):
    """Data made with the oracle's own Phi plus unit complex noise, so the
    feasible set of Eq. 2 contains the truth."""
    rng = np.random.default_rng(seed)
    om = rng.uniform(-math.pi, math.pi, (L, M, 2)) * 0.6
    w = np.zeros((L, M))
    op = nf.Operator(om, w, np.ones(L), nf.Geometry(ny, nx))
    xt = np.zeros((L, ny, nx))
    xt[:, 5:9, 6:11] = 1.0
    xt[1] *= 0.5
    y = np.stack([op.forward(xt[l], l) for l in range(L)])
    y = y + (rng.standard_normal((L, M)) + 1j * rng.standard_normal((L, M))) / math.sqrt(2)
    bo = np.array([[0, M // 2, M]] * L)
    return om, w, y, bo, xt


def test_unregularised_run_reaches_the_l2_balls():
    om, w, y, bo, xt = _feasible_problem()
    o = pdfb.FHS(om, w, y, np.ones(2), bo, 16, 16, 1, 2, 2, 0.2, mu=0, mu_bar=0)
    o.run(400)
    assert np.all(o.residual_norms() <= o.eps * (1 + 1e-3))
    assert o.X.min() >= 0.0


def test_iterates_settle():
    """Fixed point of the iteration: successive changes shrink by orders."""
    om, w, y, bo, xt = _feasible_problem(1)
    o = pdfb.FHS(om, w, y, np.ones(2), bo, 16, 16, 1, 2, 2, 0.2, mu=0.05, mu_bar=0.5)
    rels = o.run(300)
    assert rels[-1] < 1e-3 * rels[5]


def _tiny(C=2, L=4):
    P = synth.make_problem("tiny", L=L, C=C)
    return P


def test_subcubes_are_independent_problems():
    """Eq. 3: solving C channel-interleaved sub-cubes jointly equals C separate solves."""
    P = _tiny()
    steps = pdfb.Steps(tau=0.33, sigma0=0.25, sigma1=1.0, sigma2=1e-3)
    kw = dict(mu=0.02, mu_bar=0.3, steps=steps)
    joint = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 2, P.qy, P.qx, P.overlap, **kw)
    joint.run(6, 1)
    for c in range(2):
        ch = list(range(c, 4, 2))
        sep = pdfb.FHS(P.omega[ch], P.w[ch], P.y[ch], P.sigma[ch], P.block_offsets[ch], P.ny, P.nx, 1,
                       P.qy, P.qx, P.overlap, **kw)
        sep.run(6, 1)
        np.testing.assert_allclose(joint.X[ch], sep.X, rtol=0, atol=1e-12 * np.abs(sep.X).max())


def test_faceted_sara_inside_pdfb_equals_global():
    P = _tiny(C=1, L=2)
    steps = pdfb.Steps(tau=0.33, sigma0=0.25, sigma1=1.0, sigma2=1e-3)
    kw = dict(mu=0.02, mu_bar=0.3, steps=steps)
    a = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, P.qy, P.qx, P.overlap, **kw)
    b = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, P.qy, P.qx, P.overlap,
                 faceted_sara=True, sara_q=(2, 3), **kw)
    a.run(5)
    b.run(5)
    np.testing.assert_allclose(a.X, b.X, rtol=0, atol=1e-12 * np.abs(a.X).max())


def test_hypersara_special_case_single_facet():
    """(C, Q) = (1, 1): the nuclear dual is the global SVT of the whole cube."""
    P = _tiny(C=1, L=2)
    steps = pdfb.Steps(tau=0.33, sigma0=1.0, sigma1=1.0, sigma2=1e-3)
    o = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, 1, 1, 0.0,
                 mu=0.0, mu_bar=0.4, steps=steps)
    assert o.facets == [(0, P.ny, 0, P.nx)]
    o.run(3)
    Xold = o.X.copy()
    Pold = o.P[0][0].copy()
    o.step()
    Xb = 2 * o.X - Xold
    Z = (Pold + Xb).reshape(2, -1).T
    U, S, Vt = np.linalg.svd(Z, full_matrices=False)
    expect = Z - (U * np.maximum(S - 0.4, 0)) @ Vt
    np.testing.assert_allclose(o.P[0][0].reshape(2, -1).T, expect, atol=1e-12)


def test_first_iteration_closed_form():
    """From x = 0 and zero duals: x+ = 0, xbar = 0, so v_{l,b} = -s y (1 - min(1, eps/||y||)),
    W = 0, P = 0."""
    P = _tiny(C=1, L=2)
    steps = pdfb.Steps(tau=0.33, sigma0=0.25, sigma1=1.0, sigma2=2e-3)
    o = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, P.qy, P.qx, P.overlap,
                 mu=0.1, mu_bar=0.1, steps=steps)
    o.step()
    assert np.all(o.X == 0)
    for l in range(2):
        for b in range(P.B):
            s0, s1 = P.block_offsets[l, b], P.block_offsets[l, b + 1]
            yb = P.y[l, s0:s1] / P.sigma[l]
            expect = -2e-3 * yb * (1 - min(1.0, o.eps[l, b] / np.linalg.norm(yb)))
            np.testing.assert_allclose(o.v[l][s0:s1], expect, atol=1e-15)
    assert np.all(o.W[0] == 0)


# ---------------------------------------------------------------------------
# Plant a mistake in the oracle (CPU only) and check that a pin catches it.
# ---------------------------------------------------------------------------

def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def test_mutation_dropped_scaling(monkeypatch):
    monkeypatch.setattr(nf, "scaling", lambda N, K, J, beta: np.ones(N))
    assert _fails(tn.test_nufft_matches_direct_transform, 32, 32)


def test_mutation_fft_sign(monkeypatch):
    def wrong(self, x):
        g = np.zeros((self.geom.K1, self.geom.K2), dtype=np.complex128)
        g[np.ix_(self.i1, self.i2)] = x * self.s1[:, None] * self.s2[None, :]
        return np.fft.ifft2(g) * g.size
    monkeypatch.setattr(nf.Operator, "fzx", wrong)
    assert _fails(tn.test_nufft_matches_direct_transform, 32, 32)


def test_mutation_wkernel_sign(monkeypatch):
    orig = nf.wkernel
    monkeypatch.setattr(nf, "wkernel", lambda wp, N, K, ps, lo, hi: orig(-wp, N, K, ps, lo, hi))
    assert _fails(tn.test_full_wkernel_matches_direct_transform_with_wterm)


def test_mutation_highpass_without_alternation(monkeypatch):
    monkeypatch.setattr(wv, "highpass", lambda h: h[::-1].copy())
    assert _fails(ts.test_parseval_and_adjoint, 64, 48)


def test_mutation_decimation_phase(monkeypatch):
    orig = wv.analysis_axis

    def shifted(a, f, axis):
        a2 = np.moveaxis(a, axis, -1)
        n, F = a2.shape[-1], len(f)
        m = wv.out_len(n, F)
        k = np.arange(m)
        out = np.zeros(a2.shape[:-1] + (m,))
        for i in range(F):
            idx = 2 * k - i                      # even phase instead of 2k+1-i
            ok = (idx >= 0) & (idx < n)
            out[..., ok] += f[i] * a2[..., idx[ok]]
        return np.moveaxis(out, -1, axis)
    monkeypatch.setattr(wv, "analysis_axis", shifted)
    assert _fails(ts.test_haar_level_by_hand)
    assert _fails(ts.test_parseval_and_adjoint, 37, 53)


def test_mutation_sara_scale(monkeypatch):
    monkeypatch.setattr(wv, "SARA_SCALE", 1.0)
    assert _fails(ts.test_parseval_and_adjoint, 16, 16)


def test_mutation_facet_window_too_short(monkeypatch):
    def short(n, Q, i, F, levels):
        b = wv.tile_bounds(n, Q)
        step = 1 << levels
        return (max(0, b[i] - 2 * step) // step) * step, b[i + 1]
    monkeypatch.setattr(wv, "facet_window", short)
    assert _fails(ts.test_faceted_equals_global, 128, 128, 2, 2)


def test_mutation_eps_not_squared(monkeypatch):
    monkeypatch.setattr(prox, "eps_blocks", lambda M, bs: (M + 2.0 * math.sqrt(M)) * np.asarray(bs, float) / M)
    assert _fails(tp.test_eps_golden)


def test_mutation_l21_threshold_scaled_by_step(monkeypatch):
    orig = prox.l21_dual
    monkeypatch.setattr(prox, "l21_dual", lambda W, A, s, mu, wts: orig(W, A, s, mu / s, wts))
    assert _fails(tp.test_l21_dual_against_numerical_prox)


def test_mutation_svt_hard_threshold(monkeypatch):
    def wrong(Z, thr):
        U, S, Vt = np.linalg.svd(Z, full_matrices=False)
        return (U * np.where(S > thr[: len(S)], S, 0.0)[None, :]) @ Vt     # hard instead of soft
    monkeypatch.setattr(prox, "svt", wrong)
    assert _fails(tp.test_svt_properties)


def test_mutation_ball_radius_ignores_step(monkeypatch):
    orig = prox.l2ball_dual
    monkeypatch.setattr(prox, "l2ball_dual", lambda v, phix, y, eps, s: orig(v, phix, y, eps * s, s))
    assert _fails(test_first_iteration_closed_form)
