"""Pins of the oracle's visibility-gridding data reduction (Sec. 3.4,
Eqs. 4-5) against what the definitions fix: dense brute force on a tiny
problem, the whitening property of Lambda (Gamma Gamma^H has a unit
diagonal), the reduced residual equals the gridded residual for any image,
the adjoint identity, the exact mean and variance of ||Gamma n||^2 for
Gaussian noise (the basis of the default bound), noise-free data lying in the
reduced model, and a PDFB run with the reduced data term reaching its l2
ball."""
import numpy as np
import pytest

from paper_2209_07604_gb300 import synth
from oracle import nufft as onf, pdfb as opdfb, reduction as ored


def _setup(name="tiny", **over):
    P = synth.make_problem(name, **over)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    yw = [P.y[l] / P.sigma[l] for l in range(P.L)]
    return P, op, yw, ored.Reduced(op, yw)


def test_dense_brute_force():
    P, op, yw, red = _setup()
    for l in range(P.L):
        Gd = op.G[l].toarray()
        Hd = Gd.conj().T @ Gd
        touched = np.unique(np.nonzero(Gd)[1])             # grid cells any row reaches
        np.testing.assert_array_equal(red.rows[l], touched)
        d = np.real(np.diag(Hd))[touched]
        np.testing.assert_allclose(red.lam[l], 1.0 / np.sqrt(d), rtol=1e-13)
        np.testing.assert_allclose(red.Hr[l].toarray(), Hd[touched], rtol=0, atol=1e-13 * np.abs(Hd).max())
        ref_y = (1.0 / np.sqrt(d)) * (Gd.conj().T @ yw[l])[touched]
        np.testing.assert_allclose(red.y[l], ref_y, rtol=1e-12, atol=1e-12 * np.abs(ref_y).max())


def test_whitening_unit_diagonal():
    """Lambda whitens: Gamma Gamma^H = Lambda H Lambda has ones on its diagonal."""
    P, op, yw, red = _setup()
    Gd = op.G[0].toarray()
    Gam = red.lam[0][:, None] * Gd.conj().T[red.rows[0]]
    np.testing.assert_allclose(np.real(np.diag(Gam @ Gam.conj().T)), 1.0, rtol=1e-12)
    assert red.m_red(0) < op.geom.K1 * op.geom.K2


def test_reduced_residual_is_gridded_residual():
    """y' - Phi' x = Gamma (y - Phi x) for any x (Eq. 4 applied to the model)."""
    P, op, yw, red = _setup("mid_w")
    x = synth.random_image((P.ny, P.nx), 3)
    for l in (0, P.L - 1):
        lhs = red.y[l] - red.forward(x, l)
        rhs = red.gamma(yw[l] - op.forward(x, l), l)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11 * np.abs(rhs).max())


def test_adjoint_identity():
    P, op, yw, red = _setup("mid_w")
    x = synth.random_image((P.ny, P.nx), 4)
    rng = np.random.default_rng(5)
    v = rng.standard_normal(red.m_red(1)) + 1j * rng.standard_normal(red.m_red(1))
    lhs = np.vdot(v, red.forward(x, 1)).real
    rhs = float(np.sum(x * red.adjoint(v, 1)))
    assert abs(lhs - rhs) <= 1e-11 * np.linalg.norm(v) * np.linalg.norm(red.forward(x, 1))


def test_gridded_noise_norm_statistics():
    """For n with i.i.d. CN(0, 1) entries, E||Gamma n||^2 = trace(Gamma Gamma^H) = M'
    and Var = ||Gamma Gamma^H||_F^2; the sample mean of 400 draws lies within 4
    standard errors of M'."""
    P, op, yw, red = _setup()
    Gd = op.G[0].toarray()
    Gam = red.lam[0][:, None] * Gd.conj().T[red.rows[0]]
    A = Gam @ Gam.conj().T
    M = Gd.shape[0]
    rng = np.random.default_rng(11)
    n = (rng.standard_normal((400, M)) + 1j * rng.standard_normal((400, M))) / np.sqrt(2.0)
    q = np.sum(np.abs(n @ Gam.T) ** 2, axis=1)
    se = np.sqrt(np.sum(np.abs(A) ** 2) / 400)
    assert abs(q.mean() - red.m_red(0)) < 4 * se
    np.testing.assert_allclose(red.eps_default()[0] ** 2, red.m_red(0) + 2 * np.sqrt(red.m_red(0)))


def test_norm_by_lanczos_matches_power_iteration():
    P, op, yw, red = _setup()
    a = red.norm2_eigsh(0)
    b = red.norm2(0, n_iter=5000, tol=1e-13)
    assert abs(a - b) < 1e-6 * a


def test_noise_free_data_lies_in_the_reduced_model():
    P, op, _, _ = _setup()
    x = synth.random_image((P.L, P.ny, P.nx), 8)
    yw = [op.forward(x[l], l) for l in range(P.L)]
    red = ored.Reduced(op, yw)
    for l in range(P.L):
        r = red.y[l] - red.forward(x[l], l)
        assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(red.y[l])


def test_reduced_pdfb_reaches_its_ball():
    """Data term alone (mu = mu_bar = 0): the PDFB iterate of the reduced problem
    ends inside (up to 1 %) the l2 ball around y' of radius eps' = 1.2 ||Gamma n||,
    starting from x = 0, which lies far outside it."""
    P = synth.make_problem("tiny")
    geom = onf.Geometry(P.ny, P.nx)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    ywn = [P.y[l] / P.sigma[l] for l in range(P.L)]
    red = ored.Reduced(op, ywn)
    x0 = np.clip(synth.random_image((P.L, P.ny, P.nx), 9), 0, None)
    rng = np.random.default_rng(12)
    noise = [0.3 * (rng.standard_normal(P.M) + 1j * rng.standard_normal(P.M)) for _ in range(P.L)]
    y = np.stack([(op.forward(x0[l], l) + noise[l]) * P.sigma[l] for l in range(P.L)])
    eps = np.array([1.2 * np.linalg.norm(red.gamma(noise[l], l)) for l in range(P.L)])
    ref = opdfb.FHS(P.omega, P.w, y, P.sigma, P.block_offsets, P.ny, P.nx, 1, 1, 1, 0.0, mu=0.0, mu_bar=0.0,
                    eps=eps, reduction=True)
    assert np.all(ref.residual_norms()[:, 0] > 3 * eps)
    ref.run(600)
    assert np.all(ref.residual_norms()[:, 0] <= 1.01 * eps)
    assert ref.X.min() >= 0.0
