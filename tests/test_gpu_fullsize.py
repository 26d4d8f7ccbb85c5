"""Parity at the benchmark size (1024x1024, 16 channels, 16e6 visibilities,
w-projection, 4 blocks, 4x4 facets, 2 sub-cubes), in the launch
configuration bench.py times, on outputs the FP64 oracle can compute one by
one and on properties that hold at any size.

* Phi: sampled visibilities of two channels against the oracle's G rows
  applied to its own FFT of the zero-padded, scaled image.
* Phi^H: the adjoint of a vector that is non-zero on sampled visibilities only
  (every G row, bin and channel of the full problem is still traversed),
  against the oracle's gridding of those rows, on every pixel.
* First PDFB iteration: the data dual in closed form (x = 0, Eq. 2).
* After more iterations: x >= 0, every l21 dual row inside its ball of
  radius mu w, every nuclear dual facet with singular values <= mu_bar w.
* Reweighting: nuclear weights against numpy's SVD of each facet of x, l21
  weights against the library's own analysis of x.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from paper_2209_07604_gb300 import synth
from oracle import nufft as onf, prox as oprox

MU, MU_BAR = 1e-2, 1e-1        # the regularisation bench.py uses


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()
    P = synth.make_problem("vla_1024")
    prob = fhs.Problem.from_synth(P, mu=MU, mu_bar=MU_BAR)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    yield P, prob, geom
    prob.close()


def _oracle_rows(P, geom, l, idx):
    return onf.build_G(P.omega[l, idx], P.w[l, idx], float(P.sigma[l]), geom)


def test_phi_sampled_visibilities(full):
    P, prob, geom = full
    x = synth.random_image((P.L, P.ny, P.nx), 31)
    vis = prob.measure(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().reshape(P.L, -1)
    rng = np.random.default_rng(5)
    op_s = onf.scaling(P.ny, geom.K1, geom.J, geom.beta), onf.scaling(P.nx, geom.K2, geom.J, geom.beta)
    for l in (0, P.L - 1):
        idx = np.sort(rng.choice(P.M, 3000, replace=False))
        G = _oracle_rows(P, geom, l, idx)
        g = np.zeros((geom.K1, geom.K2), dtype=np.complex128)
        i1 = (np.arange(P.ny) - P.ny // 2) % geom.K1
        i2 = (np.arange(P.nx) - P.nx // 2) % geom.K2
        g[np.ix_(i1, i2)] = x[l] * op_s[0][:, None] * op_s[1][None, :]
        ref = G @ np.fft.fft2(g).ravel()
        got = vis[l, idx]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_phi_adjoint_of_sampled_visibilities(full):
    P, prob, geom = full
    rng = np.random.default_rng(6)
    v = np.zeros((P.L, P.M), dtype=np.complex128)
    picks = {}
    for l in range(P.L):
        idx = np.sort(rng.choice(P.M, 400, replace=False))
        v[l, idx] = synth.random_vis(400, 100 + l)
        picks[l] = idx
    img = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    for l in (1, P.L // 2):
        G = _oracle_rows(P, geom, l, picks[l])
        grid = (G.conj().T @ v[l, picks[l]]).reshape(geom.K1, geom.K2)
        s1 = onf.scaling(P.ny, geom.K1, geom.J, geom.beta)
        s2 = onf.scaling(P.nx, geom.K2, geom.J, geom.beta)
        full_img = np.fft.ifft2(grid) * grid.size
        i1 = (np.arange(P.ny) - P.ny // 2) % geom.K1
        i2 = (np.arange(P.nx) - P.nx // 2) % geom.K2
        ref = np.real(full_img[np.ix_(i1, i2)]) * s1[:, None] * s2[None, :]
        assert np.linalg.norm(img[l] - ref) / np.linalg.norm(ref) < 1e-5


def test_adjoint_identity_full(full):
    P, prob, geom = full
    x = synth.random_image((P.L, P.ny, P.nx), 41, nonneg=False)
    v = synth.random_vis(P.L * P.M, 42)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    vt = torch.tensor(v, dtype=torch.complex64, device="cuda")
    phix = prob.measure(xt).cpu().numpy().astype(np.complex128)
    phtv = prob.adjoint(vt).cpu().numpy().astype(np.float64)
    lhs = np.vdot(v, phix).real
    rhs = float(np.sum(phtv * x))
    assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(v) * np.linalg.norm(phix)


def test_pdfb_full_size_properties(full):
    P, prob, geom = full
    info = prob.info
    prob.step(1)
    # first iteration: x+ = 0, v_b = -s y_b (1 - min(1, eps_b / ||y_b||)) (whitened y)
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    s2 = info.sigma2
    for l in (0, 7, 15):
        for b in range(P.B):
            a, e = P.block_offsets[l, b], P.block_offsets[l, b + 1]
            yb = P.y[l, a:e] / P.sigma[l]
            eps = oprox.eps_blocks(P.M, [e - a])[0]
            ref = -s2 * yb * (1.0 - min(1.0, eps / np.linalg.norm(yb)))
            assert np.linalg.norm(v[l, a:e] - ref) / np.linalg.norm(ref) < 1e-5
    assert float(prob.image().abs().max()) == 0.0
    prob.step(4)
    X = prob.image()
    assert torch.isfinite(X).all() and float(X.min()) >= 0.0
    # l21 dual rows (over the channels of each sub-cube) inside radius mu (weights 1)
    W = prob.get_state(fhs.STATE_DUAL_SARA).reshape(P.L, -1)
    for c in range(P.C):
        rows = torch.sqrt((W[c::P.C].double() ** 2).sum(0))
        assert float(rows.max()) <= MU * (1 + 1e-5)
    # nuclear dual facets: singular values clipped at mu_bar
    Pn = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy().astype(np.float64)
    facets = oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap)
    Lc = P.L // P.C
    off = 0
    for c in range(P.C):
        for (y0, y1, x0, x1) in facets:
            n = Lc * (y1 - y0) * (x1 - x0)
            Z = Pn[off:off + n].reshape(Lc, -1).T
            off += n
            assert np.linalg.svd(Z, compute_uv=False)[0] <= MU_BAR * (1 + 1e-4)
    assert off == Pn.size


def test_reweight_full_size(full):
    P, prob, geom = full
    prob.reweight()
    X = prob.image().cpu().numpy().astype(np.float64)
    wn = prob.get_state(fhs.STATE_WEIGHTS_NUC).cpu().numpy().reshape(P.C, -1, P.L // P.C)
    facets = oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap)
    ups = 1e-3
    for c in range(P.C):
        for q, (y0, y1, x0, x1) in enumerate(facets):
            S = np.linalg.svd(X[c::P.C, y0:y1, x0:x1].reshape(P.L // P.C, -1).T, compute_uv=False)
            np.testing.assert_allclose(wn[c, q], ups / (ups + S), rtol=1e-4, atol=1e-6)
    coef = prob.sara_analysis(prob.image()).double()
    w21 = prob.get_state(fhs.STATE_WEIGHTS_SARA).reshape(P.C, -1).double()
    for c in range(P.C):
        rows = torch.sqrt((coef[c::P.C] ** 2).sum(0))
        ref = ups / (ups + rows)
        assert float((w21[c] - ref).abs().max()) < 1e-5
