"""Noise levels and l2 bounds from a model cube (Sec. 3.3 (i), Sec. 5) on the
GPU against the oracle, with and without data reduction, and the iteration
after the bounds are applied."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth
from oracle import defaults as od, nufft as onf, pdfb as opdfb, reduction as ored




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _model(P, seed):
    return np.clip(synth.random_image((P.L, P.ny, P.nx), seed), 0, None)


@pytest.mark.parametrize("name", ["tiny", "mid_w"])
def test_noise_from_model_matches_oracle(name):
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    x0 = _model(P, 41)
    sig, eps = prob.noise_from_model(torch.tensor(x0, dtype=torch.float32, device="cuda"), apply=True)
    yw = [P.y[l] / P.sigma[l] for l in range(P.L)]
    rs, re = od.noise_from_model(op, yw, P.sigma, P.block_offsets, x0)
    np.testing.assert_allclose(eps, re.ravel(), rtol=1e-5)
    np.testing.assert_allclose(sig, rs.ravel(), rtol=1e-5)
    # the applied bounds are the ones the iteration uses
    i = prob.info
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=0.05, mu_bar=0.5, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size, eps=re,
                    steps=opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=i.sigma2))
    prob.step(6)
    ref.run(6)
    torch.cuda.synchronize()
    assert rel(prob.image().cpu().numpy(), ref.X) < 1e-4
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    assert rel(v, np.stack(ref.v)) < 1e-4
    prob.close()


def test_noise_from_model_with_data_reduction():
    P = synth.make_problem("mid_w")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1e-3, data_reduction=1)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    red = ored.Reduced(onf.Operator(P.omega, P.w, P.sigma, geom), [P.y[l] / P.sigma[l] for l in range(P.L)])
    x0 = _model(P, 42)
    sig, eps = prob.noise_from_model(torch.tensor(x0, dtype=torch.float32, device="cuda"))
    rs, re = od.reduced_bounds(red, x0)
    np.testing.assert_allclose(eps, re, rtol=1e-5)
    np.testing.assert_allclose(sig, rs, rtol=1e-5)
    prob.close()


def test_noise_from_true_model_on_gpu():
    """Whitened data Phi x + s n with s = 2.5: the model x gives bounds ||s n_b||
    and noise levels sigma_l s within 4 standard errors."""
    P = synth.make_problem("small_128")
    geom = onf.Geometry(P.ny, P.nx)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    x = _model(P, 43)
    rng = np.random.default_rng(44)
    s = 2.5
    n = (rng.standard_normal((P.L, P.M)) + 1j * rng.standard_normal((P.L, P.M))) / np.sqrt(2.0)
    y = np.stack([(op.forward(x[l], l) + s * n[l]) * P.sigma[l] for l in range(P.L)])
    prob = fhs.Problem(fhs.default_params(ny=P.ny, nx=P.nx, n_channels=P.L, n_subcubes=P.C, n_blocks=P.B,
                                          qy=P.qy, qx=P.qx, facet_overlap=P.overlap, mu=0.0, mu_bar=0.0,
                                          sigma2=1.0),
                       P.omega.reshape(-1, 2), P.w.reshape(-1), y.reshape(-1), P.sigma,
                       np.arange(P.L + 1, dtype=np.int64) * P.M, P.block_offsets)
    sig, eps = prob.noise_from_model(torch.tensor(x, dtype=torch.float32, device="cuda"))
    for l in range(P.L):
        for b in range(P.B):
            nb = n[l][P.block_offsets[l, b]:P.block_offsets[l, b + 1]]
            k = l * P.B + b
            # FP32 operator: the residual of the true model is s n up to ~1e-6 of ||y||
            assert abs(eps[k] - s * np.linalg.norm(nb)) < 2e-3 * eps[k]
            assert abs(sig[k] / (P.sigma[l] * s) - 1.0) < 4.0 / (2.0 * np.sqrt(len(nb))) + 2e-3
    prob.close()
