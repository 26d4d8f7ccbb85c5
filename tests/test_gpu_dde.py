"""DDE kernels folded into G (Sec. 3.1) on the GPU, compared with the oracle's
rows (the 2-D convolution of each interpolation box with its DDE kernel):
Phi and Phi^H, the adjoint identity of the GPU pair, the centred delta kernel
(which leaves G unchanged), and PDFB iterates and duals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth
from oracle import nufft as onf, pdfb as opdfb

TOL_OP = 1e-5
TOL_IMG = 1e-4




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _problem(name):
    P = synth.make_problem(name)
    if P.w_max > 0:
        # w-kernels of at most 2 extra taps per side leave room for the 4 DDE taps
        P.w *= 0.5
    dde = synth.random_dde(P.L, P.M, 7604 + 17 * len(name))
    return P, dde


@pytest.mark.parametrize("name", ["tiny", "small_128", "mid_w"])
def test_dde_measure_and_adjoint(name):
    P, dde = _problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0, dde=dde)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega, P.w, P.sigma, geom, dde=dde)
    x = synth.random_image((P.L, P.ny, P.nx), 1)
    vis = prob.measure(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy().reshape(P.L, -1)
    assert rel(vis, np.stack(op.forward_all(x))) < TOL_OP
    v = synth.random_vis((P.L, P.M), 2)
    img = prob.adjoint(torch.tensor(v.reshape(-1), dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert rel(img, op.adjoint_all(list(v))) < TOL_OP
    lhs = np.vdot(v.reshape(-1), vis.reshape(-1).astype(np.complex128)).real
    rhs = float(np.sum(img.astype(np.float64) * x))
    assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(v) * np.linalg.norm(vis)
    # every row is stored as 5 separable terms of T + 4 taps per axis
    T = np.sqrt(prob.info.nnz / (P.L * P.M))
    assert prob.info.n_gfac == pytest.approx(2 * 5 * P.L * P.M * T, rel=0.2)
    prob.close()


def test_delta_dde_leaves_phi_unchanged():
    P = synth.make_problem("small_128")
    dde = np.zeros((P.L, P.M, 5, 5), dtype=np.complex128)
    dde[:, :, 2, 2] = 1.0
    a = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0)
    b = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0, dde=dde)
    x = torch.tensor(synth.random_image((P.L, P.ny, P.nx), 5), dtype=torch.float32, device="cuda")
    assert rel(b.measure(x).cpu().numpy(), a.measure(x).cpu().numpy()) < 1e-6
    v = torch.tensor(synth.random_vis(P.L * P.M, 6), dtype=torch.complex64, device="cuda")
    assert rel(b.adjoint(v).cpu().numpy(), a.adjoint(v).cpu().numpy()) < 1e-5
    a.close()
    b.close()


@pytest.mark.parametrize("name,n_iter,mu,mu_bar", [("tiny", 10, 0.02, 0.3), ("mid_w", 12, 0.05, 0.5)])
def test_dde_pdfb_iterates(name, n_iter, mu, mu_bar):
    P, dde = _problem(name)
    geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
    op = onf.Operator(P.omega[:1], P.w[:1], P.sigma[:1], geom, dde=dde[:1])
    sigma2 = 1.0 / (1.02 * op.norm2(0, n_iter=60))
    prob = fhs.Problem.from_synth(P, mu=mu, mu_bar=mu_bar, sigma2=sigma2, dde=dde)
    i = prob.info
    ref = opdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                    mu=mu, mu_bar=mu_bar, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size,
                    steps=opdfb.Steps(tau=i.tau, sigma0=i.sigma0, sigma1=i.sigma1, sigma2=sigma2), dde=dde)
    ref.run(n_iter, 0)
    prob.step(n_iter)
    torch.cuda.synchronize()
    assert rel(prob.image().cpu().numpy(), ref.X) < TOL_IMG
    v = prob.get_state(fhs.STATE_DUAL_DATA).cpu().numpy().view(np.complex64).reshape(P.L, -1)
    assert rel(v, np.stack(ref.v)) < TOL_IMG
    prob.close()
