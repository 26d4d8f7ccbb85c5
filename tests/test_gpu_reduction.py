"""Visibility-gridding data reduction (Sec. 3.4, Eqs. 4-5) on the GPU against
the oracle's explicit sparse H: gridded point counts, ||Phi'_l||^2, the
reduced residual and dirty image (which exercise Lambda, y' and both passes
over G), PDFB iterates and the reduced dual, the dirty-image defaults of mu
and mu_bar, checkpoint/resume of the reduced dual, and DDE rows with data
reduction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth
from oracle import defaults as od, nufft as onf, pdfb as opdfb, prox as oprox, reduction as ored
from oracle import wavelets as owav

TOL_OP = 1e-5
TOL_IMG = 1e-4




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _oracle_red(P, dde=None):
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom, dde=dde)
    return ored.Reduced(op, [P.y[l] / P.sigma[l] for l in range(P.L)])


@pytest.mark.parametrize("name", ["tiny", "mid_w"])
def test_reduced_residual_dirty_image_and_norms(name):
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, data_reduction=1)
    red = _oracle_red(P)
    assert prob.info.n_red == sum(red.m_red(l) for l in range(P.L))
    # sigma2 = 1 / max_l ||Phi'_l||^2
    ref = max(red.norm2_eigsh(l) for l in range(P.L))
    assert abs(prob.info.phi_norm2_max - ref) < 1e-4 * ref
    eta = od.psf_peak_factors(red, P.ny, P.nx)
    assert rel(prob.residual().cpu().numpy(), od.residual(red, red.y, None, eta)) < TOL_OP
    x = synth.random_image((P.L, P.ny, P.nx), 13)
    got = prob.residual(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel(got, od.residual(red, red.y, x, eta)) < TOL_OP
    prob.close()


def _reduced_dual(prob, P, red):
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    on = [v[l][red.rows[l]] for l in range(P.L)]
    off = [np.delete(v[l], red.rows[l]) for l in range(P.L)]
    return on, off


@pytest.mark.parametrize("name,n_iter,n_reweight,mu,mu_bar", [("tiny", 12, 0, 0.02, 0.3),
                                                              ("mid_w", 12, 1, 0.05, 0.5)])
def test_reduced_pdfb_iterates(name, n_iter, n_reweight, mu, mu_bar):
    P = synth.make_problem(name)
    red = _oracle_red(P)
    sigma2 = 1.0 / (1.02 * max(red.norm2_eigsh(l) for l in range(P.L)))
    prob = fhs.Problem.from_synth(P, mu=mu, mu_bar=mu_bar, sigma2=sigma2, data_reduction=1)
    i = prob.info
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=mu, mu_bar=mu_bar, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size,
                    steps=opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=sigma2), reduction=True)
    ref.run(n_iter, n_reweight)
    per = n_iter // (n_reweight + 1)
    for r in range(n_reweight + 1):
        prob.step(per if r < n_reweight else n_iter - per * n_reweight)
        if r < n_reweight:
            prob.reweight()
    torch.cuda.synchronize()
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    on, off = _reduced_dual(prob, P, red)
    for l in range(P.L):
        assert rel(on[l], ref.v[l]) < TOL_IMG
        assert not np.any(off[l])
    prob.close()


def test_reduced_default_regularisation():
    P = synth.make_problem("small_128")
    prob = fhs.Problem.from_synth(P, mu=-1.0, mu_bar=-1.0, data_reduction=1)
    red = _oracle_red(P)
    eta = od.psf_peak_factors(red, P.ny, P.nx)
    dirty = od.residual(red, red.y, None, eta)
    mu, mu_bar = od.default_regularisation(dirty, P.C, oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap),
                                           owav.Sara(P.ny, P.nx, 4))
    assert abs(prob.info.mu - mu) < 1e-4 * mu and abs(prob.info.mu_bar - mu_bar) < 1e-4 * mu_bar
    prob.step(3)
    assert torch.isfinite(prob.image()).all()
    prob.close()


def test_reduced_eps_given_and_checkpoint_resume():
    """eps' given per channel (half the default) is the ball radius of the oracle
    run it matches; set_state of the reduced dual resumes the iteration."""
    P = synth.make_problem("mid_w")
    red = _oracle_red(P)
    eps = 0.5 * red.eps_default()
    prob = fhs.Problem(fhs.default_params(ny=P.ny, nx=P.nx, n_channels=P.L, n_subcubes=P.C, n_blocks=P.B,
                                          qy=P.qy, qx=P.qx, facet_overlap=P.overlap, w_max=P.w_max,
                                          pixel_size=P.pixel_size, mu=0.05, mu_bar=0.5, data_reduction=1),
                       P.omega.reshape(-1, 2), P.w.reshape(-1), P.y.reshape(-1), P.sigma,
                       np.arange(P.L + 1, dtype=np.int64) * P.M, P.block_offsets, eps)
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=0.05, mu_bar=0.5, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size, eps=eps,
                    steps=opdfb.Steps(tau=prob.info.tau, sigma0=prob.info.sigma0, sigma1=prob.info.sigma1,
                                      sigma2=prob.info.sigma2), reduction=True)
    prob.step(6)
    ref.run(6)
    torch.cuda.synchronize()
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    parts = [fhs.STATE_IMAGE, fhs.STATE_DUAL_DATA, fhs.STATE_DUAL_SARA, fhs.STATE_DUAL_NUCLEAR,
             fhs.STATE_WEIGHTS_SARA, fhs.STATE_WEIGHTS_NUC]
    saved = {k: prob.get_state(k).clone() for k in parts}
    assert saved[fhs.STATE_DUAL_DATA].numel() == 2 * P.L * 4 * P.ny * P.nx
    prob.step(4)
    Xa = prob.image().cpu().numpy()
    prob.params.sigma2 = prob.info.sigma2          # the step set-up chose from ||Phi'||^2
    other = fhs.Problem(prob.params, P.omega.reshape(-1, 2), P.w.reshape(-1), P.y.reshape(-1), P.sigma,
                        np.arange(P.L + 1, dtype=np.int64) * P.M, P.block_offsets, eps)
    for k in parts:
        other.set_state(k, saved[k])
    other.step(4)
    assert rel(other.image().cpu().numpy(), Xa) < 1e-5
    prob.close()
    other.close()


def test_reduced_with_dde_rows():
    P = synth.make_problem("tiny")
    dde = synth.random_dde(P.L, P.M, 31)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0, data_reduction=1, dde=dde)
    red = _oracle_red(P, dde)
    assert prob.info.n_red == sum(red.m_red(l) for l in range(P.L))
    eta = od.psf_peak_factors(red, P.ny, P.nx)
    x = synth.random_image((P.L, P.ny, P.nx), 14)
    got = prob.residual(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel(got, od.residual(red, red.y, x, eta)) < TOL_OP
    prob.close()
