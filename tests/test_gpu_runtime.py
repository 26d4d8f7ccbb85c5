"""Runtime pieces on the GPU: footprint estimate vs the bytes a problem holds,
CUDA-graph replay vs kernel-by-kernel launches, concurrent stepping of
several independent problems on their own streams vs stepping them alone, and
the measured choice of tile bins (the operators and the iteration unchanged)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


@pytest.mark.parametrize("name", ["tiny", "mid_w", "small_128"])
def test_estimate_matches_held_bytes(name):
    P = synth.make_problem(name)
    prob = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=1e-3)
    res, peak = fhs.fhs_estimate_bytes(prob.params, P.w.reshape(-1), P.L * P.M)
    held = prob.info.device_bytes
    assert held <= res <= held * 1.01 + (1 << 20)
    assert peak >= res
    prob.close()


def test_graph_replay_matches_plain_launches():
    P = synth.make_problem("mid_w")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-7)
        b = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-7)
        fhs.fhs_use_graphs(b.handle, False)
        n0a, n0b = fhs.fhs_kernel_launches(a.handle), fhs.fhs_kernel_launches(b.handle)
        a.step(7)
        b.step(7)
        a.reweight()
        b.reweight()
        a.step(5)
        b.step(5)
        s.synchronize()
        assert rel(a.image().cpu().numpy(), b.image().cpu().numpy()) < 1e-5
        assert fhs.fhs_kernel_launches(a.handle) - n0a == fhs.fhs_kernel_launches(b.handle) - n0b
        assert fhs.fhs_get_info(a.handle).iteration == 12
    a.close()
    b.close()


def test_batched_problems_match_alone():
    names = ["tiny", "mid_w", "small_128"]
    Ps = [synth.make_problem(n) for n in names]
    streams = [torch.cuda.Stream() for _ in names]
    batch = [fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-4) for P in Ps]
    rel_b = fhs.fhs_pdfb_step_batch([p.handle for p in batch], 9, streams, want_rel=True)
    alone = []
    for P in Ps:
        q = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-4)
        r = q.step(9, want_rel=True)
        alone.append((q, r))
    torch.cuda.synchronize()
    for k, (q, r) in enumerate(alone):
        assert rel(batch[k].image().cpu().numpy(), q.image().cpu().numpy()) < 1e-5
        assert abs(rel_b[k] - r) <= 1e-4 * r
        q.close()
        batch[k].close()


@pytest.mark.parametrize("name", ["mid_w", "small_128"])
def test_autotune_bins_changes_layout_only(name):
    """After fhs_autotune_bins, Phi, Phi^H and the PDFB iteration (resumed from a
    mid-run state, with its graph recaptured) agree with an untuned twin; the
    binning reported is one of the candidates."""
    P = synth.make_problem(name)
    a = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5)        # sigma2 from the set-up's norm estimate
    b = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=a.info.sigma2)
    a.step(3)
    b.step(3)
    dm, sp = b.autotune_bins()
    assert dm in (16, 32, 48, 96) and sp in (192, 288, 384)
    assert (b.info.bin_dense_min, b.info.bin_split) == (dm, sp)
    x = torch.tensor(synth.random_image((P.L, P.ny, P.nx), 3), dtype=torch.float32, device="cuda")
    va, vb = a.measure(x), b.measure(x)
    assert rel(vb.cpu().numpy(), va.cpu().numpy()) < 1e-6
    v = torch.tensor(synth.random_vis(P.L * P.M, 4), dtype=torch.complex64, device="cuda")
    assert rel(b.adjoint(v).cpu().numpy(), a.adjoint(v).cpu().numpy()) < 1e-5
    a.step(4)
    b.step(4)
    torch.cuda.synchronize()
    # the adjoint's summation order differs: iterates agree to the suite's 1e-4
    assert rel(b.image().cpu().numpy(), a.image().cpu().numpy()) < 1e-4
    for part in (fhs.STATE_DUAL_DATA, fhs.STATE_DUAL_SARA, fhs.STATE_DUAL_NUCLEAR):
        pa = a.get_state(part).cpu().numpy()
        pb = b.get_state(part).cpu().numpy()
        assert rel(pb, pa) < 1e-4, part
    a.close()
    b.close()


def test_device_wait_that_runs_out_is_reported():
    """Failure detection without a fault: a kernel waits, with the bounded wait
    of the pass over G's window copy, on an mbarrier that nothing arrives at.
    The wait gives up, the kernel records a timeout and returns, and every
    synchronising call that reads the flag reports FHS_ERR_TIMEOUT once; the
    problem stays usable afterwards."""
    import time
    P = synth.make_problem("tiny")
    prob = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    prob.step(2)
    fhs.fhs_device_status(prob.handle)                    # healthy
    t0 = time.perf_counter()
    fhs.fhs_debug_unsatisfied_wait(prob.handle, 1000)
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_device_status(prob.handle)
    assert time.perf_counter() - t0 < 30.0                 # the wait is bounded
    assert e.value.status == fhs.FHS_ERR_TIMEOUT
    assert "window copy" in str(e.value)
    fhs.fhs_device_status(prob.handle)                    # read once, then clear
    # the iteration's own synchronising calls read the same flag
    fhs.fhs_debug_unsatisfied_wait(prob.handle, 1000)
    with pytest.raises(fhs.FhsError) as e:
        prob.step(1, want_rel=True)
    assert e.value.status == fhs.FHS_ERR_TIMEOUT
    fhs.fhs_debug_unsatisfied_wait(prob.handle, 1000)
    with pytest.raises(fhs.FhsError) as e:
        prob.solve(4, 0.0, n_reweight=1, check_every=2)
    assert e.value.status == fhs.FHS_ERR_TIMEOUT
    fhs.fhs_debug_unsatisfied_wait(prob.handle, 1000)
    with pytest.raises(fhs.FhsError) as e:
        prob.noise_from_model(prob.image())
    assert e.value.status == fhs.FHS_ERR_TIMEOUT
    r = prob.step(1, want_rel=True)
    assert np.isfinite(r)
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_debug_unsatisfied_wait(prob.handle, 0)
    assert e.value.status == fhs.FHS_ERR_ARG
    prob.close()


def test_get_image_and_workspace_names():
    """fhs_get_image is the image part of the state transfer and
    fhs_workspace_bytes the footprint query under the boundary's names."""
    P = synth.make_problem("tiny")
    prob = fhs.Problem.from_synth(P, mu=0.02, mu_bar=0.3, sigma2=5e-6)
    prob.step(3)
    a = prob.get_state(fhs.STATE_IMAGE).cpu().numpy()
    x = torch.empty((P.L, P.ny, P.nx), dtype=torch.float32, device="cuda")
    fhs.fhs_get_image(prob.handle, x)
    np.testing.assert_array_equal(x.cpu().numpy().ravel(), a)
    assert fhs.fhs_workspace_bytes(prob.params, P.w.reshape(-1), P.L * P.M) == \
        fhs.fhs_estimate_bytes(prob.params, P.w.reshape(-1), P.L * P.M)
    prob.close()
