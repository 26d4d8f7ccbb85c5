"""GPU parity of libfhs against the FP64 oracle, through the C ABI.

Tolerances: Phi / Phi^H and the SARA transforms run in FP32 with FP32
accumulation over at most a few hundred terms, so the relative error of a
whole output vector is bounded by ~sqrt(terms) * 2^-24 * (condition of the
sum) ~ 1e-6; the parity bound is 1e-5 (relative, 2-norm).  A PDFB iterate is
a non-expansive map of FP32-rounded operators, so after k iterations the
image error stays at a few 1e-6; the bound is 1e-4.  Every comparison takes
the larger of the relative 2-norm error and the element-wise error
max|a - b| / max|b| (tests/parity.py), so each bound holds element by element
on the array's own scale too.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel, rel2
from paper_2209_07604_gb300 import synth
from oracle import nufft as onf, pdfb as opdfb, prox as oprox, wavelets as owv

TOL_OP = 1e-5
TOL_IMG = 1e-4




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _oracle(P, mu, mu_bar, sigma2, n_wplanes=64, **kw):
    return opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                     mu=mu, mu_bar=mu_bar, w_max=P.w_max, n_wplanes=n_wplanes, pixel_size=P.pixel_size,
                     steps=kw.pop("steps", None), **kw)


def _steps_from(prob, sigma2):
    i = prob.info
    return opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=sigma2)


@pytest.mark.parametrize("name", ["tiny", "small_128", "mid_w"])
def test_measure_and_adjoint(name):
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    x = synth.random_image((P.L, P.ny, P.nx), 1)
    vis = prob.measure(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().reshape(P.L, -1)
    ref = np.stack(op.forward_all(x))
    assert rel(vis, ref) < TOL_OP
    v = synth.random_vis((P.L, P.M), 2)
    img = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    ref_img = op.adjoint_all(list(v))
    assert rel(img, ref_img) < TOL_OP
    # adjoint identity of the GPU pair itself, on the Cauchy-Schwarz scale
    # ||v|| ||Phi x|| (the sum itself cancels heavily)
    lhs = np.vdot(v.reshape(-1), vis.reshape(-1).astype(np.complex128)).real
    rhs = float(np.sum(img.astype(np.float64) * x))
    assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(v) * np.linalg.norm(vis)
    prob.close()


def test_nnz_and_row_lengths_match_oracle():
    P = synth.make_problem("mid_w")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    nnz = sum(onf.build_G(P.omega[l], P.w[l], 1.0, geom).nnz for l in range(P.L))
    assert prob.info.nnz == nnz
    prob.close()


@pytest.mark.parametrize("ny,nx,levels", [(128, 128, 4), (96, 160, 4), (48, 32, 2), (64, 64, 1)])
def test_sara_analysis_synthesis(ny, nx, levels):
    P = synth.make_problem("tiny")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0, ny=ny, nx=nx, wavelet_levels=levels)
    S = owv.Sara(ny, nx, levels)
    assert prob.info.n_coef == S.n_coef
    x = synth.random_image((P.L, ny, nx), 3, nonneg=False)
    c = prob.sara_analysis(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel(c, S.analysis(x)) < TOL_OP
    z = synth.random_image((P.L, S.n_coef), 4, nonneg=False)
    xs = prob.sara_synthesis(torch.tensor(z, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel(xs, S.synthesis(z)) < TOL_OP
    prob.close()


def test_operator_norms():
    """||Phi_l||^2 by the GPU Lanczos estimate against the largest singular
    value of the explicit FP64 matrix (tiny problem), and against ARPACK's
    Lanczos on the FP64 oracle operator at the parity sizes (with and without
    w-terms)."""
    P = synth.make_problem("tiny")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    gpu = prob.operator_norms(200)
    for l in range(P.L):
        cols = []
        for k in range(P.ny * P.nx):
            e = np.zeros(P.ny * P.nx)
            e[k] = 1.0
            cols.append(op.forward(e.reshape(P.ny, P.nx), l))
        A = np.array(cols).T
        smax = np.linalg.svd(np.vstack([A.real, A.imag]), compute_uv=False)[0]
        assert abs(gpu[l] - smax ** 2) < 1e-5 * smax ** 2
    prob.close()
    for name in ("small_128", "mid_w"):
        P = synth.make_problem(name)
        prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
        op = onf.Operator(P.omega, P.w, P.sigma, onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64,
                                                               pixel_size=P.pixel_size))
        gpu = prob.operator_norms(80)
        refs = [op.norm2_eigsh(l) for l in range(P.L)]
        for l in range(P.L):
            assert abs(gpu[l] - refs[l]) < 1e-5 * refs[l], (name, l, gpu[l], refs[l])
        prob.close()
        # the data step chosen at set-up (sigma2 <= 0): 1 / max_l ||Phi_l||^2
        prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0)
        assert abs(prob.info.sigma2 * max(refs) - 1.0) < 1e-5
        prob.close()


def _run_pair(name, n_iter, n_reweight, mu, mu_bar, gram_precision=0, **over):
    P = synth.make_problem(name, **over)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega[:1], P.w[:1], P.sigma[:1], geom)
    sigma2 = 1.0 / (1.02 * op.norm2(0, n_iter=60))
    prob = fhs.Problem.from_synth(P, mu=mu, mu_bar=mu_bar, sigma2=sigma2, gram_precision=gram_precision)
    ref = _oracle(P, mu, mu_bar, sigma2, steps=_steps_from(prob, sigma2))
    ref.run(n_iter, n_reweight)
    per = n_iter // (n_reweight + 1)
    for r in range(n_reweight + 1):
        k = per if r < n_reweight else n_iter - per * n_reweight
        prob.step(k)
        if r < n_reweight:
            prob.reweight()
    torch.cuda.synchronize()
    return P, prob, ref


@pytest.mark.parametrize("name,n_iter,n_reweight,mu,mu_bar", [
    ("tiny", 10, 0, 0.02, 0.3),
    ("small_128", 50, 0, 0.05, 1.0),
    ("mid_w", 20, 1, 0.05, 0.5),
])
def test_pdfb_iterates(name, n_iter, n_reweight, mu, mu_bar):
    P, prob, ref = _run_pair(name, n_iter, n_reweight, mu, mu_bar)
    img = prob.image().cpu().numpy()
    assert rel(img, ref.X) < TOL_IMG
    # duals
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    assert rel(v, np.stack(ref.v)) < TOL_IMG
    W = prob.get_state(fhs.STATE_DUAL_SARA).cpu().numpy().reshape(P.L, -1)
    Wref = np.zeros_like(W, dtype=np.float64)
    for c, ch in enumerate(ref.chans):
        Wref[ch] = ref.W[c]
    assert rel(W, Wref) < TOL_IMG
    Pn = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy()
    Pref = np.concatenate([ref.P[c][q].ravel() for c in range(P.C) for q in range(len(ref.facets))])
    assert rel(Pn, Pref) < TOL_IMG
    if n_reweight:
        w21 = prob.get_state(fhs.STATE_WEIGHTS_SARA).cpu().numpy().reshape(P.C, -1)
        assert rel(w21, np.stack(ref.w21)) < TOL_IMG
        wn = prob.get_state(fhs.STATE_WEIGHTS_NUC).cpu().numpy()
        wref = np.concatenate([ref.wnuc[c][q] for c in range(P.C) for q in range(len(ref.facets))])
        assert rel(wn, wref) < TOL_IMG
    prob.close()


@pytest.mark.parametrize("L", [17, 32])
def test_pdfb_iterates_many_channels_per_subcube(L):
    """L_c in (16, 32]: the shared-memory Gram (FP64 mode, which resolves the
    small singular values that the SVT weights see), the 32 x 32 FP64 Jacobi
    and the 32-channel apply (odd L_c pads the Jacobi to an even size).  The
    FP32, TF32 and BF16 Grams at this size are measured against the oracle in
    the mixed-precision tests."""
    P, prob, ref = _run_pair("tiny", 8, 1, 0.02, 0.3, L=L, C=1, gram_precision=fhs.GRAM_FP64)
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    Pn = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy()
    Pref = np.concatenate([ref.P[c][q].ravel() for c in range(P.C) for q in range(len(ref.facets))])
    assert rel(Pn, Pref) < TOL_IMG
    wn = prob.get_state(fhs.STATE_WEIGHTS_NUC).cpu().numpy()
    wref = np.concatenate([ref.wnuc[c][q] for c in range(P.C) for q in range(len(ref.facets))])
    assert rel(wn, wref) < TOL_IMG
    prob.close()


@pytest.mark.parametrize("name", ["tiny", "mid_w"])
def test_residual_and_dirty_image(name):
    """eta_l Re Phi_l^H (y_l - Phi_l x_l) (Sec. 5.3) against the oracle, for x = 0
    (the dirty image) and for a random x; eta from the oracle's PSF peak."""
    from oracle import defaults as od
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    eta = od.psf_peak_factors(op, P.ny, P.nx)
    yw = [P.y[l] / P.sigma[l] for l in range(P.L)]
    assert rel(prob.residual().cpu().numpy(), od.residual(op, yw, None, eta)) < TOL_OP
    x = synth.random_image((P.L, P.ny, P.nx), 12)
    got = prob.residual(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert rel(got, od.residual(op, yw, x, eta)) < TOL_OP
    prob.close()


@pytest.mark.parametrize("name", ["small_128", "mid_w"])
def test_default_regularisation(name):
    """mu, mu_bar < 0 select 1 / ||Psi^dagger X||_{2,1} and 1 / sum_q ||S_q X||_* of the
    dirty cube X, summed over sub-cubes, against the oracle; the iteration then runs."""
    from oracle import defaults as od
    from oracle import wavelets as owav
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=-1.0, mu_bar=-1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    eta = od.psf_peak_factors(op, P.ny, P.nx)
    dirty = od.residual(op, [P.y[l] / P.sigma[l] for l in range(P.L)], None, eta)
    mu, mu_bar = od.default_regularisation(dirty, P.C, oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap),
                                           owav.Sara(P.ny, P.nx, 4))
    info = prob.info
    assert abs(info.mu - mu) < 1e-4 * mu and abs(info.mu_bar - mu_bar) < 1e-4 * mu_bar
    prob.step(3)
    assert torch.isfinite(prob.image()).all()
    prob.close()


def test_relative_change_and_nonnegativity():
    P = synth.make_problem("tiny")
    prob = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    prob.step(3)
    Xa = prob.image().cpu().numpy().astype(np.float64)
    r = prob.step(1, want_rel=True)
    Xb = prob.image().cpu().numpy().astype(np.float64)
    assert abs(r - np.linalg.norm(Xb - Xa) / np.linalg.norm(Xb)) < 1e-5 * r
    assert Xb.min() >= 0.0
    prob.close()


def test_checkpoint_resume():
    P = synth.make_problem("mid_w")
    prob = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-7)
    prob.step(4)
    prob.reweight()
    prob.step(2)
    parts = [fhs.STATE_IMAGE, fhs.STATE_DUAL_DATA, fhs.STATE_DUAL_SARA, fhs.STATE_DUAL_NUCLEAR,
             fhs.STATE_WEIGHTS_SARA, fhs.STATE_WEIGHTS_NUC]
    saved = {k: prob.get_state(k).clone() for k in parts}
    prob.step(5)
    Xa = prob.image().cpu().numpy()
    other = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-7)
    for k in parts:
        other.set_state(k, saved[k])
    other.step(5)
    Xb = other.image().cpu().numpy()
    assert rel(Xb, Xa) < 1e-5
    prob.close()
    other.close()


def test_solve_matches_step_schedule():
    P = synth.make_problem("tiny")
    a = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    n = a.solve(12, 0.0, n_reweight=1, check_every=4)
    assert n == 12
    b = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    b.step(6)
    b.reweight()
    b.step(6)
    assert rel(a.image().cpu().numpy(), b.image().cpu().numpy()) < 1e-5
    a.close()
    b.close()


def test_empty_block_and_uneven_channels():
    """A block with no visibilities (eps = 0, factor 1) and channels with
    different visibility counts, against the oracle."""
    P = synth.make_problem("tiny", L=2, C=1)
    M = P.M
    cut = M - 200
    omega = np.concatenate([P.omega[0], P.omega[1, :cut]])
    w = np.concatenate([P.w[0], P.w[1, :cut]])
    y = np.concatenate([P.y[0], P.y[1, :cut]])
    vo = np.array([0, M, M + cut], dtype=np.int64)
    bo = np.array([[0, M // 2, M], [0, 0, cut]], dtype=np.int64)
    params = fhs.default_params(ny=P.ny, nx=P.nx, n_channels=2, n_subcubes=1, n_blocks=2, qy=P.qy, qx=P.qx,
                                facet_overlap=P.overlap, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    prob = fhs.Problem(params, omega, w, y, P.sigma, vo, bo)
    prob.step(6)
    X = prob.image().cpu().numpy()
    # oracle per channel: channel 1 with its truncated data, blocks [0,0) and [0,cut)
    geom = onf.Geometry(P.ny, P.nx)
    from oracle import prox as oprox
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, P.qy, P.qx, P.overlap,
                    mu=0.02, mu_bar=0.3, steps=_steps_from(prob, 5e-6))
    ref.op.G[1] = onf.build_G(P.omega[1, :cut], P.w[1, :cut], P.sigma[1], geom)
    ref.yw[1] = P.y[1, :cut] / P.sigma[1]
    ref.v[1] = np.zeros(cut, dtype=np.complex128)
    ref.bo = np.array([[0, M // 2, M], [0, 0, cut]])
    ref.eps = np.stack([oprox.eps_blocks(M, [M // 2, M - M // 2]), oprox.eps_blocks(cut, [0, cut])])
    ref.run(6)
    assert rel(X, ref.X) < TOL_IMG
    prob.close()


@pytest.mark.parametrize("name,over,n_iter,mu,mu_bar", [
    ("small_128", {}, 20, 0.0, 0.0),                          # data fidelity only
    ("tiny", dict(qy=1, qx=1, overlap=0.0), 8, 0.02, 0.3),     # (C, Q) = (1, 1): HyperSARA
    ("tiny", dict(L=2, C=2), 8, 0.02, 0.3),                    # one channel per sub-cube
    ("tiny", dict(L=3, C=1, B=1), 8, 0.02, 0.3),               # odd L_c, one block
])
def test_pdfb_degenerate_cases(name, over, n_iter, mu, mu_bar):
    P, prob, ref = _run_pair(name, n_iter, 0, mu, mu_bar, **over)
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    assert rel(v, np.stack(ref.v)) < TOL_IMG
    prob.close()


def test_empty_channel():
    """A channel without visibilities: its data term is zero (Phi_l has no
    rows, eps = 0); the priors still couple it to the other channel."""
    import scipy.sparse as sp
    P = synth.make_problem("tiny", L=2, C=1)
    M = P.M
    omega = P.omega[0]
    w = P.w[0]
    y = P.y[0]
    vo = np.array([0, M, M], dtype=np.int64)
    bo = np.array([[0, M // 2, M], [0, 0, 0]], dtype=np.int64)
    params = fhs.default_params(ny=P.ny, nx=P.nx, n_channels=2, n_subcubes=1, n_blocks=2, qy=P.qy, qx=P.qx,
                                facet_overlap=P.overlap, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    prob = fhs.Problem(params, omega, w, y, P.sigma, vo, bo)
    prob.step(6)
    X = prob.image().cpu().numpy()
    from oracle import prox as oprox
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, 1, P.qy, P.qx, P.overlap,
                    mu=0.02, mu_bar=0.3, steps=_steps_from(prob, 5e-6))
    geom = onf.Geometry(P.ny, P.nx)
    ref.op.G[1] = sp.csr_matrix((0, geom.K1 * geom.K2), dtype=np.complex128)
    ref.yw[1] = np.zeros(0, dtype=np.complex128)
    ref.v[1] = np.zeros(0, dtype=np.complex128)
    ref.bo = np.array([[0, M // 2, M], [0, 0, 0]])
    ref.eps = np.stack([oprox.eps_blocks(M, [M // 2, M - M // 2]), np.zeros(2)])
    ref.run(6)
    assert rel(X, ref.X) < TOL_IMG
    prob.close()


@pytest.mark.parametrize("name", ["tiny", "small_128", "mid_w"])
def test_adjoint_precision_of_fixed_point_scatter(name):
    """Phi^H accumulates dense bins in 32-bit fixed point (quantum 2^-21 of each
    bin's bound on its contributions); against the FP64 oracle its relative
    2-norm error stays within 5e-6, half the operator tolerance, and every
    pixel within the operator tolerance on the image's scale (the roundings
    of the cells a pixel gathers do not average out pixel by pixel)."""
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    v = synth.random_vis((P.L, P.M), 2)
    img = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    ref = op.adjoint_all(list(v))
    assert rel2(img, ref) < 5e-6 and rel(img, ref) < TOL_OP
    yw = [P.y[l] / P.sigma[l] for l in range(P.L)]
    img = prob.adjoint(torch.tensor(np.concatenate(yw).astype(np.complex64), device="cuda")).cpu().numpy()
    ref = op.adjoint_all(yw)
    assert rel2(img, ref) < 5e-6 and rel(img, ref) < TOL_OP
    prob.close()


@pytest.mark.parametrize("scale", [1e-20, 1e20])
def test_adjoint_scales_linearly_across_the_fixed_point_range(scale):
    """Phi^H (s v) = s Phi^H v for scales that send the bins' bounds far from 1:
    the fixed-point windows rescale per bin (2^(21 - e))."""
    P = synth.make_problem("small_128")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    v = synth.random_vis((P.L, P.M), 3).reshape(-1)
    ref = prob.adjoint(torch.tensor(v, dtype=torch.complex64, device="cuda")).cpu().numpy().astype(np.float64)
    got = prob.adjoint(torch.tensor(v * scale, dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert np.all(np.isfinite(got))
    # two independent fixed-point roundings (s is not a power of two), each within 5e-6 of exact
    # in 2-norm and within the operator tolerance pixel by pixel
    assert rel2(got / scale, ref) < 5e-6 and rel(got / scale, ref) < TOL_OP
    prob.close()


def test_adjoint_with_a_non_finite_visibility():
    """A NaN visibility sends its bin to the FP32 atomics (no fixed-point
    conversion of a non-finite value): its channel's image is NaN, as with
    floating-point accumulation, and the other channels are unchanged."""
    P = synth.make_problem("small_128")
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    v = synth.random_vis((P.L, P.M), 4)
    ref = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    v[1, P.M // 3] = np.nan
    got = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert np.isnan(got[1]).any()
    for l in (0, 2, 3):
        np.testing.assert_array_equal(np.isfinite(got[l]), True)
        # the same fixed-point sums; only the order of the FP32 window flushes into the grid differs
        assert rel2(got[l], ref[l]) < 1e-6 and rel(got[l], ref[l]) < TOL_OP
    prob.close()


def test_measure_adjoint_and_iterates_with_negative_w():
    """w < 0 takes the negative w-planes (-P1..-1) of the kernel table: half of
    the visibilities get their w negated, against the oracle's planes of the
    same sign; operators, then PDFB iterates with a reweighting."""
    P = synth.make_problem("mid_w")
    P.w = P.w * np.where(np.arange(P.M) % 2 == 0, -1.0, 1.0)[None, :]
    assert (P.w < 0).mean() > 0.4
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom)
    x = synth.random_image((P.L, P.ny, P.nx), 31)
    vis = prob.measure(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().reshape(P.L, -1)
    assert rel(vis, np.stack(op.forward_all(x))) < TOL_OP
    v = synth.random_vis((P.L, P.M), 32)
    img = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert rel(img, op.adjoint_all(list(v))) < TOL_OP
    prob.close()
    sigma2 = 1.0 / (1.02 * onf.Operator(P.omega[:1], P.w[:1], P.sigma[:1], geom).norm2(0, n_iter=60))
    prob = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=sigma2)
    ref = _oracle(P, 0.05, 0.5, sigma2, steps=_steps_from(prob, sigma2))
    ref.run(12, 1)
    prob.step(6)
    prob.reweight()
    prob.step(6)
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    vg = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    assert rel(vg, np.stack(ref.v)) < TOL_IMG
    prob.close()


def test_reweight_closed_forms():
    """The library's reweighting on cubes whose weights have closed forms
    (Sec. 2.2.3): X_l = c_l u has rank one on every facet, so facet q's
    weights are [ub / (ub + ||u_q|| ||c||), 1, ...]; its l21 weights on the
    Dirac block are u / (u + ||c|| u_n / 3).  Set as the image by the state
    transfer, then reweighted; FP64 arithmetic on the GPU, single-precision
    image."""
    ups, ups_bar = 0.5, 0.7
    P = synth.make_problem("mid_w")
    prob = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-7, upsilon=ups, upsilon_bar=ups_bar)
    rng = np.random.default_rng(5)
    u = rng.uniform(0.5, 3.0, (P.ny, P.nx)).astype(np.float32)
    gains = np.array([1.3, 0.4, 2.1, 0.9], dtype=np.float32)[:P.L]
    X = (gains[:, None, None] * u[None]).astype(np.float32)
    prob.set_state(fhs.STATE_IMAGE, torch.tensor(X.ravel(), device="cuda"))
    prob.reweight()
    torch.cuda.synchronize()
    facets = oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap)
    wn = prob.get_state(fhs.STATE_WEIGHTS_NUC).cpu().numpy().reshape(P.C, len(facets), -1)
    w21 = prob.get_state(fhs.STATE_WEIGHTS_SARA).cpu().numpy().reshape(P.C, -1)
    u64, g64 = u.astype(np.float64), gains.astype(np.float64)
    N = P.ny * P.nx
    for c in range(P.C):
        ch = list(range(c, P.L, P.C))
        gc = np.linalg.norm(g64[ch])
        exp21 = ups / (ups + gc * u64.ravel() / 3.0)
        assert rel(w21[c, :N], exp21) < 1e-5
        for q, (y0, y1, x0, x1) in enumerate(facets):
            s0 = np.linalg.norm(u64[y0:y1, x0:x1]) * gc
            expect = np.ones(len(ch))
            expect[0] = ups_bar / (ups_bar + s0)
            assert rel(wn[c, q], expect) < 1e-5, (c, q, wn[c, q], expect)
    prob.close()


_GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


_GEOM_PROBLEMS = {}

# the nuclear dual under the tensor-core Grams: the bounds of the mixed-precision tests (TF32 keeps 10
# mantissa bits, BF16 7); every other part of the state is held to the image tolerance in every mode
_NUC_BOUND = {fhs.GRAM_FP32: TOL_IMG, fhs.GRAM_TF32: 1e-2, fhs.GRAM_BF16: 3e-2}


def _benchmark_geometry(side, precision):
    d = np.load(os.path.join(_GOLDEN, "fhs_%s_samples.npz" % side))
    if side not in _GEOM_PROBLEMS:
        _GEOM_PROBLEMS.clear()
        _GEOM_PROBLEMS[side] = synth.make_problem(str(d["workload"]), M=int(d["m_per_channel"]))
    P = _GEOM_PROBLEMS[side]
    prob = fhs.Problem.from_synth(P, mu=float(d["mu"]), mu_bar=float(d["mu_bar"]), sigma2=float(d["sigma2"]),
                                  gram_precision=precision)
    i = prob.info
    for k in ("tau", "sigma0", "sigma1"):
        assert abs(getattr(i, k) - float(d[k])) < 1e-12 * float(d[k]), k
    n_iter, n_rw = int(d["n_iter"]), int(d["n_reweight"])
    per = n_iter // (n_rw + 1)
    for r in range(n_rw + 1):
        prob.step(per if r < n_rw else n_iter - per * n_rw)
        if r < n_rw:
            prob.reweight()
    torch.cuda.synchronize()
    fhs.fhs_device_status(prob.handle)          # no bounded wait gave up
    X = prob.get_state(fhs.STATE_IMAGE).cpu().numpy()
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64)
    W = prob.get_state(fhs.STATE_DUAL_SARA).cpu().numpy()
    Pn = prob.get_state(fhs.STATE_DUAL_NUCLEAR).cpu().numpy()
    w21 = prob.get_state(fhs.STATE_WEIGHTS_SARA).cpu().numpy()
    wn = prob.get_state(fhs.STATE_WEIGHTS_NUC).cpu().numpy()
    prob.close()
    assert W.size == P.L * int(d["n_coef"])
    tol = {"X": TOL_IMG, "v": TOL_IMG, "W": TOL_IMG, "P": _NUC_BOUND[precision], "w21": TOL_IMG,
           "wnuc": TOL_IMG}
    errs = {}
    for name, arr in (("X", X), ("v", v), ("W", W), ("P", Pn), ("w21", w21)):
        got = arr[d[name + "_idx"]]
        errs[name] = rel(got, d[name])
        # the element-wise part on the scale of the whole array
        assert np.abs(got - d[name]).max() <= tol[name] * float(d[name + "_absmax"]), name
    errs["wnuc"] = rel(wn, d["wnuc"])
    print("benchmark geometry %s, %s Gram, %d iterations + %d reweighting:"
          % (side, {fhs.GRAM_FP32: "fp32", fhs.GRAM_TF32: "tf32", fhs.GRAM_BF16: "bf16"}[precision], n_iter, n_rw),
          {k: "%.1e" % e for k, e in errs.items()})
    for k, e in errs.items():
        assert e < tol[k], (k, e)


@pytest.mark.parametrize("side", ["1024", "2048"])
def test_pdfb_iterates_benchmark_geometry(side):
    """The geometry of the two imaging workloads at 3e4 visibilities per
    channel, against the FP64 oracle's run stored as seeded samples of the
    image, the three duals and the weights by tests/golden/make_fhs_samples.py
    (which calls only the oracle); every sample compared element by element.
    1024: 1024 x 1024, 16 channels in 2 sub-cubes, 4 x 4 facets with 10 %
    overlap, w-projection with 7..15 taps, 4 blocks; 10 PDFB iterations with
    one reweighting.  2048: 2048 x 2048, 32 channels in 4 sub-cubes, 8 x 8
    facets with 10 % overlap, 8 blocks; 6 iterations with one reweighting.
    The facet Gram is the default FP32 one."""
    _benchmark_geometry(side, fhs.GRAM_FP32)


@pytest.mark.parametrize("precision", [fhs.GRAM_TF32, fhs.GRAM_BF16])
def test_tensor_core_gram_benchmark_geometry(precision):
    """The 2048 x 2048, 32-channel geometry of the test above with the facet
    Gram on the tensor cores (TF32 or BF16 inputs): the per-result errors
    against the same oracle run, printed; the image, the data and SARA duals
    and the weights held to the image tolerance, the nuclear dual to the
    rounding bound of its input type."""
    _benchmark_geometry("2048", precision)
