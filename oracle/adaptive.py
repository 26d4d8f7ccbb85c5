"""Oracle adaptive estimation of the effective noise level (Sec. 3.3 (ii)).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

Sec. 3.3 (ii) gives the strategy in outline only: the PDFB iteration starts
with its image priors inactive, the noise estimates and the parameters that
follow from them (the l2 bounds) are updated while it runs, and once the l2
bounds hold they are fixed and the full problem is solved.  The update rules
are left to the cited works, so the schedule below is a reading, built from
the two rules this paper does state:

* estimator (Sec. 3.3 (i)): the noise level of block (l, b) is the standard
  deviation of the residual visibilities Theta_l (y_{l,b} - Phi_{l,b} x) of
  an image x, here the current iterate (``defaults.noise_from_model``; with
  data reduction ``defaults.reduced_bounds``);
* bound for a noise level (Eq. 2 with the chi-square reading of the default):
  eps_{l,b} = s_{l,b} eps0_{l,b}, where eps0 is the bound for unit whitened
  noise (``prox.eps_blocks``; ``Reduced.eps_default``) and s_{l,b} the
  estimated whitened noise level (sigma_hat_{l,b} / sigma_l; with data
  reduction sigma_hat'_l, already whitened).

Schedule: mu = mu_bar = 0 (priors inactive) and the bounds the problem was
built with.  Every ``check_every`` iterations, and only once the iterate has
settled (relative change of the last iteration below ``settle_tol``), a check
takes the residual norms rho_{l,b} of the current iterate: if every block has
rho_{l,b} <= eps_{l,b} the bounds hold and are fixed (the phase ends);
otherwise every bound is re-estimated as above and the iteration goes on.
The phase also ends after ``max_iter`` iterations.  mu and mu_bar are then
restored; the regularisation defaults of this package do not depend on the
noise level (dirty-image reading), so the bounds are the only parameters the
estimate moves.

Pinned by ``tests/test_oracle_adaptive.py``: the bound rule at the true
model against the closed form of the noise statistics, the recovery of an
effective noise level 2.5 times the nominal one, and the stop rule.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import defaults, prox


@dataclass
class AdaptiveResult:
    sigma_hat: np.ndarray          # noise levels of the final iterate's residual
    eps: np.ndarray                # bounds in force at the end (fixed)
    iterations: int
    n_updates: int
    satisfied: bool                # the last check found every bound satisfied
    checks: list = field(default_factory=list)   # (iteration, rho, eps before the check)


def unit_bounds(fhs) -> np.ndarray:
    """eps0: the l2 bounds of unit-variance whitened noise, shape of fhs.eps."""
    if getattr(fhs, "red", None) is not None and fhs.data is fhs.red:
        return fhs.red.eps_default().reshape(fhs.eps.shape)
    return np.stack([prox.eps_blocks(len(fhs.yw[l]), np.diff(fhs.bo[l])) for l in range(fhs.L)])


def estimate(fhs, sigma, X) -> tuple:
    """(sigma_hat, rho, s): the Sec. 3.3 (i) estimator on the image X, the residual
    norms and the whitened noise levels, each shaped like fhs.eps."""
    if getattr(fhs, "red", None) is not None and fhs.data is fhs.red:
        sig, rho = defaults.reduced_bounds(fhs.red, X)
        sig, rho = sig.reshape(fhs.eps.shape), rho.reshape(fhs.eps.shape)
        return sig, rho, sig
    sig, rho = defaults.noise_from_model(fhs.op, fhs.yw, sigma, fhs.bo, X)
    return sig, rho, sig / np.asarray(sigma, dtype=np.float64)[:, None]


def updated_bounds(fhs, sigma, X) -> np.ndarray:
    """The re-estimated bounds s_{l,b} eps0_{l,b} for the image X."""
    return estimate(fhs, sigma, X)[2] * unit_bounds(fhs)


def adaptive_noise(fhs, sigma, max_iter: int, check_every: int = 10, settle_tol: float = 1e-3) -> AdaptiveResult:
    """Run the adaptive phase on the oracle problem ``fhs`` (``pdfb.FHS``, fresh:
    no iteration done) with the channel whitening ``sigma``."""
    if fhs.n_done != 0:
        raise ValueError("the adaptive phase starts the run: the problem has iterated already")
    mu, mu_bar = fhs.mu, fhs.mu_bar
    fhs.mu, fhs.mu_bar = 0.0, 0.0
    eps0 = unit_bounds(fhs)
    it, n_up, sat, checks = 0, 0, False, []
    try:
        while it < max_iter:
            n = min(check_every, max_iter - it)
            rel = float("inf")
            for _ in range(n):
                rel = fhs.step()
            it += n
            if not rel < settle_tol:
                continue
            _, rho, s = estimate(fhs, sigma, fhs.X)
            checks.append((it, rho.copy(), fhs.eps.copy()))
            if np.all(rho <= fhs.eps):
                sat = True
                break
            fhs.eps = s * eps0
            n_up += 1
    finally:
        fhs.mu, fhs.mu_bar = mu, mu_bar
    sig = estimate(fhs, sigma, fhs.X)[0]
    return AdaptiveResult(sigma_hat=sig, eps=fhs.eps.copy(), iterations=it, n_updates=n_up, satisfied=sat,
                          checks=checks)
