"""Pins of the oracle's dirty image, residual and regularisation defaults
(oracle/defaults.py) against what the definitions fix on their own: a point
source at the phase centre images to exactly its amplitude there and leaves
a zero residual; cubes whose sub-cubes repeat one image per channel have
closed-form facet nuclear norms and l21 norms."""
import numpy as np

from oracle import defaults as od
from oracle import nufft as nf
from paper_2209_07604_gb300 import synth
from oracle import prox, wavelets


def _op(L=2, ny=16, nx=24, M=300, seed=3):
    rng = np.random.default_rng(seed)
    om = rng.uniform(-np.pi, np.pi, size=(L, M, 2)) * 0.6
    sigma = 1.0 + 0.5 * np.arange(L)
    return nf.Operator(om, np.zeros((L, M)), sigma, nf.Geometry(ny, nx)), ny, nx


def test_point_source_dirty_image_and_zero_residual():
    op, ny, nx = _op()
    eta = od.psf_peak_factors(op, ny, nx)
    a = 2.5
    X = np.zeros((op.L, ny, nx))
    X[:, ny // 2, nx // 2] = a
    yw = [op.forward(X[l], l) for l in range(op.L)]
    dirty = od.residual(op, yw, None, eta)
    for l in range(op.L):
        assert abs(dirty[l, ny // 2, nx // 2] - a) < 1e-12 * a
        assert np.unravel_index(np.argmax(dirty[l]), (ny, nx)) == (ny // 2, nx // 2)
    r = od.residual(op, yw, X, eta)
    assert np.abs(r).max() < 1e-12 * a
    # eta is the inverse PSF peak, i.e. 1 / ||Phi_l delta||^2
    d = np.zeros((ny, nx))
    d[ny // 2, nx // 2] = 1.0
    for l in range(op.L):
        assert abs(eta[l] * np.linalg.norm(op.forward(d, l)) ** 2 - 1.0) < 1e-12


def test_default_regularisation_closed_forms():
    ny, nx, L, C = 20, 28, 4, 2
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal((ny, nx)), rng.standard_normal((ny, nx))
    Xd = np.stack([u, v, u, v])                          # sub-cube 0: channels 0, 2; sub-cube 1: 1, 3
    facets = prox.nuclear_facets(ny, nx, 2, 2, 0.2)
    sara = wavelets.Sara(ny, nx, 2)
    mu, mu_bar = od.default_regularisation(Xd, C, facets, sara)
    nuc = sum(np.sqrt(2.0) * (np.linalg.norm(u[y0:y1, x0:x1]) + np.linalg.norm(v[y0:y1, x0:x1]))
              for (y0, y1, x0, x1) in facets)
    l21 = np.sqrt(2.0) * (np.abs(sara.analysis(u)).sum() + np.abs(sara.analysis(v)).sum())
    assert abs(mu_bar - 1.0 / nuc) < 1e-12 / nuc
    assert abs(mu - 1.0 / l21) < 1e-12 / l21
    mu2, mu_bar2 = od.default_regularisation(2.0 * Xd, C, facets, sara)
    assert abs(mu2 - mu / 2) < 1e-12 * mu and abs(mu_bar2 - mu_bar / 2) < 1e-12 * mu_bar


def test_noise_from_true_model_recovers_the_added_noise():
    """Data made as Phi x_true + s n (whitened, n i.i.d. CN(0, 1)): the residual
    of the true model is exactly s n, so the block bounds are ||s n_b|| and the
    noise levels estimate sigma_l s (4 standard errors); the reduced bound is
    ||Gamma_l (s n_l)|| (Sec. 3.3, 3.4, 5.1)."""
    from oracle import reduction as ored
    P = synth.make_problem("tiny")
    geom = nf.Geometry(P.ny, P.nx)
    op = nf.Operator(P.omega, P.w, P.sigma, geom)
    x = np.clip(synth.random_image((P.L, P.ny, P.nx), 21), 0, None)
    rng = np.random.default_rng(22)
    s = 3.0
    n = [(rng.standard_normal(P.M) + 1j * rng.standard_normal(P.M)) / np.sqrt(2.0) for _ in range(P.L)]
    yw = [op.forward(x[l], l) + s * n[l] for l in range(P.L)]
    sig, eps = od.noise_from_model(op, yw, P.sigma, P.block_offsets, x)
    for l in range(P.L):
        for b in range(P.B):
            nb = n[l][P.block_offsets[l, b]:P.block_offsets[l, b + 1]]
            assert abs(eps[l, b] - s * np.linalg.norm(nb)) < 1e-9 * eps[l, b]
            assert abs(sig[l, b] / (P.sigma[l] * s) - 1.0) < 4.0 / (2.0 * np.sqrt(len(nb)))
    red = ored.Reduced(op, yw)
    _, epr = od.reduced_bounds(red, x)
    for l in range(P.L):
        ref = np.linalg.norm(red.gamma(s * n[l], l))
        assert abs(epr[l] - ref) < 1e-9 * ref
