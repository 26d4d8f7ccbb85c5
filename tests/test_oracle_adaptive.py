"""Pins of the oracle's adaptive noise estimation (Sec. 3.3 (ii), reading in
oracle/adaptive.py) against the noise statistics of synthetic data
y = Phi x + s n: the bound rule at the true model against its closed form,
the recovery of an effective noise level 2.5 times the nominal one from the
nominal bounds, and the stop rule."""
import numpy as np
import pytest

from paper_2209_07604_gb300 import synth
from oracle import adaptive as oad, nufft as onf, pdfb as opdfb


S_EFF = 2.5


def _data(s, seed=44, M=6000):
    P = synth.make_problem("tiny", M=M)
    op = onf.Operator(P.omega, P.w, P.sigma, onf.Geometry(P.ny, P.nx))
    x = np.clip(synth.random_image((P.L, P.ny, P.nx), 43), 0, None)
    rng = np.random.default_rng(seed)
    n = (rng.standard_normal((P.L, P.M)) + 1j * rng.standard_normal((P.L, P.M))) / np.sqrt(2.0)
    y = np.stack([(op.forward(x[l], l) + s * n[l]) * P.sigma[l] for l in range(P.L)])
    ref = opdfb.FHS(P.omega, P.w, y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=0.05, mu_bar=0.5)
    noise = np.array([[np.linalg.norm(s * n[l][P.block_offsets[l, b]:P.block_offsets[l, b + 1]])
                       for b in range(P.B)] for l in range(P.L)])
    return P, x, ref, noise


def test_unit_bounds_are_the_default_bounds():
    P, _, ref, _ = _data(S_EFF)
    np.testing.assert_allclose(oad.unit_bounds(ref), ref.eps, rtol=0, atol=0)
    M = P.M
    np.testing.assert_allclose(oad.unit_bounds(ref) ** 2, (M + 2 * np.sqrt(M)) * 0.5, rtol=1e-14)


def test_bound_rule_at_the_true_model():
    """At x = x_true the whitened residual is s n: the re-estimated bound is
    s eps0_{l,b} within four standard errors of the sample standard deviation
    (1 / (2 sqrt(M_b)) relative), in every channel whatever its sigma_l."""
    P, x, ref, _ = _data(S_EFF)
    eps = oad.updated_bounds(ref, P.sigma, x)
    eps0 = oad.unit_bounds(ref)
    Mb = np.diff(P.block_offsets, axis=1).astype(np.float64)
    assert np.all(np.abs(eps / (S_EFF * eps0) - 1.0) < 4.0 / (2.0 * np.sqrt(Mb)) + 1e-3)
    sig, rho, s = oad.estimate(ref, P.sigma, x)
    np.testing.assert_allclose(s, sig / P.sigma[:, None], rtol=1e-14)
    # and rho is the norm of s n itself
    assert np.all(np.abs(rho / (S_EFF * np.sqrt(Mb)) - 1.0) < 4.0 / (2.0 * np.sqrt(Mb)) + 1e-3)


def test_recovers_an_effective_noise_level_above_the_nominal_one():
    """Nominal bounds (unit whitened noise) on data whose noise is 2.5 times
    larger: the bounds cannot hold, the iterate settles with its residual near
    the noise, the bounds are re-estimated and then hold.  The fixed bounds end
    near ||s n_b|| (from 0.4 ||s n_b|| at the start), the regularisation is
    restored, and every check before the last found a violated bound."""
    P, _, ref, noise = _data(S_EFF)
    assert np.all(ref.eps < 0.45 * noise)
    r = oad.adaptive_noise(ref, P.sigma, max_iter=400, check_every=10, settle_tol=3.5e-3)
    assert r.satisfied and r.n_updates >= 1
    assert np.all(r.eps / noise > 0.9) and np.all(r.eps / noise < 1.3)
    assert ref.mu == 0.05 and ref.mu_bar == 0.5
    np.testing.assert_array_equal(ref.eps, r.eps)
    it, rho, eps = r.checks[-1]
    assert it == r.iterations and np.all(rho <= eps)
    for it, rho, eps in r.checks[:-1]:
        assert np.any(rho > eps)
    # the noise level of the final iterate's residual, against the true one
    assert np.all(np.abs(r.sigma_hat / (P.sigma[:, None] * S_EFF) - 1.0) < 0.3)


def test_no_check_before_the_iterate_settles():
    """A tolerance the iterate never reaches: no check acts, the bounds stay
    nominal and the phase ends after max_iter iterations."""
    P, _, ref, _ = _data(S_EFF)
    eps0 = ref.eps.copy()
    r = oad.adaptive_noise(ref, P.sigma, max_iter=25, check_every=10, settle_tol=1e-9)
    assert r.iterations == 25 and r.n_updates == 0 and not r.satisfied and not r.checks
    np.testing.assert_array_equal(r.eps, eps0)


def test_the_phase_starts_the_run():
    P, _, ref, _ = _data(S_EFF)
    ref.step()
    with pytest.raises(ValueError):
        oad.adaptive_noise(ref, P.sigma, max_iter=10)


def test_every_check_acts_with_an_infinite_tolerance():
    """settle_tol = inf: a check every check_every iterations; the first one
    (residual far above the nominal bounds) re-estimates them."""
    P, _, ref, _ = _data(S_EFF)
    r = oad.adaptive_noise(ref, P.sigma, max_iter=40, check_every=20, settle_tol=np.inf)
    assert r.checks[0][0] == 20 and r.n_updates >= 1
    assert np.any(r.checks[0][1] > r.checks[0][2])
    assert len(r.checks) == r.n_updates + (1 if r.satisfied else 0)


def _pin_holds(P, ref, eps):
    Mb = np.diff(P.block_offsets, axis=1).astype(np.float64)
    return bool(np.all(np.abs(eps / (S_EFF * oad.unit_bounds(ref)) - 1.0) < 4.0 / (2.0 * np.sqrt(Mb)) + 1e-3))


def test_mutations_of_the_bound_rule_fail_the_pin():
    """Plausible mistakes in the bound rule, planted on the CPU: the noise level
    left unwhitened (sigma_hat instead of sigma_hat / sigma_l), the variance in
    place of the standard deviation, and the residual norm in place of the
    noise level: each fails the closed-form pin that the rule itself passes."""
    P, x, ref, _ = _data(S_EFF)
    sig, rho, s = oad.estimate(ref, P.sigma, x)
    eps0 = oad.unit_bounds(ref)
    assert _pin_holds(P, ref, s * eps0)
    assert not _pin_holds(P, ref, sig * eps0)
    assert not _pin_holds(P, ref, s ** 2 * eps0)
    assert not _pin_holds(P, ref, rho * eps0)


def test_bound_rule_with_data_reduction_at_the_true_model():
    """Gridded data (Sec. 3.4): at x = x_true the reduced residual is exactly
    Gamma_l (s n_l), and the re-estimated bound is s eps0'_l within four
    standard errors. ||Gamma_l n_l||^2 has mean trace(A) = M'_l and variance
    ||A||_F^2 with A = Lambda_l H_l Lambda_l, for circular complex Gaussian
    noise of unit variance."""
    P = synth.make_problem("tiny", M=6000)
    op = onf.Operator(P.omega, P.w, P.sigma, onf.Geometry(P.ny, P.nx))
    x = np.clip(synth.random_image((P.L, P.ny, P.nx), 43), 0, None)
    rng = np.random.default_rng(44)
    n = (rng.standard_normal((P.L, P.M)) + 1j * rng.standard_normal((P.L, P.M))) / np.sqrt(2.0)
    y = np.stack([(op.forward(x[l], l) + S_EFF * n[l]) * P.sigma[l] for l in range(P.L)])
    ref = opdfb.FHS(P.omega, P.w, y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=0.0, mu_bar=0.0, reduction=True)
    red = ref.red
    np.testing.assert_array_equal(oad.unit_bounds(ref).ravel(), red.eps_default())
    sig, rho, s = oad.estimate(ref, P.sigma, x)
    eps = oad.updated_bounds(ref, P.sigma, x)
    for l in range(P.L):
        m = red.m_red(l)
        gn = np.linalg.norm(red.gamma(S_EFF * n[l], l))
        assert abs(rho[l, 0] - gn) <= 1e-9 * gn
        A = red.Hr[l][:, red.rows[l]].multiply(np.outer(red.lam[l], red.lam[l]))
        assert abs(np.real(A.diagonal()).sum() - m) < 1e-9 * m
        se = 0.5 * np.sqrt(np.real(A.multiply(A.conj()).sum())) / m
        assert abs(eps[l, 0] / (S_EFF * red.eps_default()[l]) - 1.0) < 4.0 * se + 1e-3
        assert abs(s[l, 0] / S_EFF - 1.0) < 4.0 * se + 1e-3
