"""Mixed precision of the nuclear dual step: the facet Gram on the tensor cores
(tcgen05, TF32 or BF16 inputs, FP32 accumulation in tensor memory) against the
FP64 oracle, with the FP32 and FP64 CUDA-core Grams beside it.  Each case
reports the relative error of the image and of the nuclear dual after a fixed
number of iterations.  The bounds follow from the rounding: TF32 keeps 10
mantissa bits and BF16 7, so Gram entries carry relative errors of order 2^-11
and 2^-8; any Gram in FP32 arithmetic resolves the singular values of Z only
down to about sqrt(eps) of the largest, and the SVT weights of the ones near
the threshold inherit that.  Every mode is held to the 1e-4 image tolerance
after the fixed iteration count; the nuclear dual itself, which carries the
SVT of the singular values nearest the threshold, is held to 1e-4 with the
FP64 Gram and to the rounding bounds below with the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth
from oracle import nufft as onf, pdfb as opdfb

# error bounds after the runs below: the image (every precision) and the nuclear dual (per precision)
BOUND_IMG = 1e-4
BOUND = {fhs.GRAM_FP64: 1e-4, fhs.GRAM_FP32: 1e-2, fhs.GRAM_TF32: 1e-2, fhs.GRAM_BF16: 3e-2}
NAMES = {fhs.GRAM_FP64: "fp64", fhs.GRAM_FP32: "fp32", fhs.GRAM_TF32: "tf32", fhs.GRAM_BF16: "bf16"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()




_REF = {}


def _reference(name, n_iter, mu, mu_bar, **over):
    key = (name, n_iter, mu, mu_bar, tuple(sorted(over.items())))
    if key not in _REF:
        P = synth.make_problem(name, **over)
        geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
        op = onf.Operator(P.omega[:1], P.w[:1], P.sigma[:1], geom)
        sigma2 = 1.0 / (1.02 * op.norm2(0, n_iter=60))
        probe = fhs.Problem.from_synth(P, mu=mu, mu_bar=mu_bar, sigma2=sigma2)
        i = probe.info
        steps = opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=sigma2)
        probe.close()
        ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                        mu=mu, mu_bar=mu_bar, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size, steps=steps)
        ref.run(n_iter, 0)
        _REF[key] = (P, sigma2, ref)
    return _REF[key]


def _errors(name, n_iter, mu, mu_bar, precision, **over):
    P, sigma2, ref = _reference(name, n_iter, mu, mu_bar, **over)
    prob = fhs.Problem.from_synth(P, mu=mu, mu_bar=mu_bar, sigma2=sigma2, gram_precision=precision)
    prob.step(n_iter)
    torch.cuda.synchronize()
    fhs.fhs_device_status(prob.handle)          # no bounded wait gave up
    e_img = rel(prob.image().cpu().numpy(), ref.X)
    Pn = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy()
    Pref = np.concatenate([ref.P[c][q].ravel() for c in range(P.C) for q in range(len(ref.facets))])
    e_nuc = rel(Pn, Pref)
    prob.close()
    print("gram %s on %s (L=%d, C=%d): image rel err %.2e, nuclear dual rel err %.2e"
          % (NAMES[precision], name, P.L, P.C, e_img, e_nuc))
    return e_img, e_nuc


@pytest.mark.parametrize("precision", [fhs.GRAM_FP64, fhs.GRAM_FP32, fhs.GRAM_TF32, fhs.GRAM_BF16])
def test_gram_precision_mid_w(precision):
    e_img, e_nuc = _errors("mid_w", 20, 0.05, 0.5, precision)
    assert e_img < BOUND_IMG and e_nuc < BOUND[precision]


@pytest.mark.parametrize("precision", [fhs.GRAM_FP64, fhs.GRAM_FP32, fhs.GRAM_TF32, fhs.GRAM_BF16])
def test_gram_precision_32_channels(precision):
    """32 channels per sub-cube: the full N = 32 of the tensor-core tile."""
    e_img, e_nuc = _errors("tiny", 8, 0.02, 0.3, precision, L=32, C=1)
    assert e_img < BOUND_IMG and e_nuc < BOUND[precision]


def test_tensor_gram_close_to_fp32_gram():
    """Same problem, FP32 Gram vs TF32 Gram: the difference is at the TF32
    rounding level, far below what a wrong operand layout would give."""
    P, sigma2, _ = _reference("mid_w", 20, 0.05, 0.5)
    out = {}
    for prec in (fhs.GRAM_FP32, fhs.GRAM_TF32):
        prob = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=sigma2, gram_precision=prec)
        prob.step(30)
        out[prec] = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy().astype(np.float64)
        fhs.fhs_device_status(prob.handle)
        prob.close()
    assert np.linalg.norm(out[fhs.GRAM_FP32]) > 0
    assert rel(out[fhs.GRAM_TF32], out[fhs.GRAM_FP32]) < 3e-3
