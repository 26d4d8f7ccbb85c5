"""Runtime pieces on the GPU: footprint estimate vs the bytes a problem holds,
CUDA-graph replay vs kernel-by-kernel launches, and concurrent stepping of
several independent problems on their own streams vs stepping them alone."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from paper_2209_07604_gb300 import synth


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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
        a = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-4)
        b = fhs.Problem.from_synth(P, mu=0.05, mu_bar=0.5, sigma2=1e-4)
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
