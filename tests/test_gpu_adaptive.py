"""Adaptive noise estimation (Sec. 3.3 (ii); the schedule is the reading in
oracle/adaptive.py) through the C ABI against the oracle on data whose
effective noise is 2.5 times the nominal one: the counts of the phase, the
re-estimated bounds and noise levels, the iterate, the iteration after the
phase with the priors restored, data reduction, and the argument and state
errors."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth
from oracle import adaptive as oad, nufft as onf, pdfb as opdfb

S_EFF = 2.5
TOL = 1e-4




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _pair(name, M, mu, mu_bar, dr=0):
    P = synth.make_problem(name, M=M)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    x = np.clip(synth.random_image((P.L, P.ny, P.nx), 43), 0, None)
    rng = np.random.default_rng(44)
    n = (rng.standard_normal((P.L, P.M)) + 1j * rng.standard_normal((P.L, P.M))) / np.sqrt(2.0)
    y = np.stack([(op.forward(x[l], l) + S_EFF * n[l]) * P.sigma[l] for l in range(P.L)])
    prob = fhs.Problem(fhs.default_params(ny=P.ny, nx=P.nx, n_channels=P.L, n_subcubes=P.C, n_blocks=P.B,
                                          qy=P.qy, qx=P.qx, facet_overlap=P.overlap, w_max=P.w_max,
                                          pixel_size=P.pixel_size, mu=mu, mu_bar=mu_bar, data_reduction=dr),
                       P.omega.reshape(-1, 2), P.w.reshape(-1), y.reshape(-1), P.sigma,
                       np.arange(P.L + 1, dtype=np.int64) * P.M, P.block_offsets)
    i = prob.info
    ref = opdfb.FHS(P.omega, P.w, y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=mu, mu_bar=mu_bar, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size,
                    steps=opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=i.sigma2),
                    reduction=bool(dr))
    return P, prob, ref


def _compare(P, prob, ref, max_iter, check_every):
    sig, eps, res = prob.adaptive_noise(max_iter, check_every, np.inf)
    r = oad.adaptive_noise(ref, P.sigma, max_iter, check_every, np.inf)
    # every decision of the oracle's checks is far from its threshold
    for _, rho, e in r.checks:
        assert np.all(np.abs(rho / e - 1.0) > 1e-3)
    assert res == dict(iterations=r.iterations, n_checks=len(r.checks), n_updates=r.n_updates,
                       satisfied=int(r.satisfied))
    assert r.n_updates >= 1
    assert rel(eps, r.eps.ravel()) < TOL
    assert rel(sig, r.sigma_hat.ravel()) < TOL
    torch.cuda.synchronize()
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL
    i = fhs.fhs_get_info(prob.handle)
    assert i.iteration == r.iterations and i.mu == ref.mu and i.mu_bar == ref.mu_bar
    return r


@pytest.mark.parametrize("graphs", [True, False])
def test_adaptive_phase_matches_oracle(graphs):
    """With graphs the calls run on a side stream, where the iteration is
    captured once and replayed: the phase must capture it again without the
    priors, and again with them after."""
    P, prob, ref = _pair("tiny", 6000, 0.05, 0.5)
    fhs.fhs_use_graphs(prob.handle, graphs)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side if graphs else torch.cuda.current_stream()):
        r = _compare(P, prob, ref, 30, 10)
        assert r.satisfied
        # the bounds moved up from the nominal ones towards the effective noise
        assert np.all(r.eps > 2.0 * oad.unit_bounds(ref))
        # the iteration after the phase: priors active again, bounds fixed
        prob.step(6)
        ref.run(6)
        torch.cuda.synchronize()
        assert rel(prob.image().cpu().numpy(), ref.X) < TOL
        v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
        assert rel(v, np.stack(ref.v)) < TOL
        assert np.any(prob.get_state(fhs.STATE_DUAL_SARA).cpu().numpy())
    torch.cuda.synchronize()
    prob.close()


def test_adaptive_phase_with_data_reduction():
    P, prob, ref = _pair("tiny", 6000, 0.0, 0.0, dr=1)
    r = _compare(P, prob, ref, 30, 10)
    assert r.eps.size == P.L
    prob.close()


def test_adaptive_phase_errors_and_zero_iterations():
    P, prob, ref = _pair("tiny", 3000, 0.05, 0.5)
    for args in [(-1, 10, 1e-3), (10, 0, 1e-3), (10, 10, 0.0), (10, 10, float("nan"))]:
        with pytest.raises(fhs.FhsError) as e:
            prob.adaptive_noise(*args)
        assert e.value.status == fhs.FHS_ERR_ARG
    # no iteration: the bounds stay, the noise levels are those of the data (x = 0)
    sig, eps, res = prob.adaptive_noise(0, 10, 1e-3)
    assert res == dict(iterations=0, n_checks=0, n_updates=0, satisfied=0)
    np.testing.assert_allclose(eps, oad.unit_bounds(ref).ravel(), rtol=1e-12)
    s0, _, _ = oad.estimate(ref, P.sigma, np.zeros((P.L, P.ny, P.nx)))
    assert rel(sig, s0.ravel()) < 1e-5
    prob.step(1)
    with pytest.raises(fhs.FhsError) as e:
        prob.adaptive_noise(10, 10, 1e-3)
    assert e.value.status == fhs.FHS_ERR_STATE
    prob.close()
