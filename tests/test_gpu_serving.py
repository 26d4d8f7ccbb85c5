"""Serving: requests of different sizes solved concurrently by the native
server give the same images as each request solved alone (within the FP32
tolerance of the parity tests; only the order of floating-point atomics
differs), admission respects the device-memory budget, and a request that
can never fit is refused at submission."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth

MIX = [("tiny", {}), ("mid_w", {}), ("small_128", {}), ("tiny", dict(L=3, C=1, trial=1))]
KW = dict(mu=0.05, mu_bar=0.5, max_iter=30, rel_tol=1e-3, n_reweight=1, check_every=5)




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def _alone(P):
    prob = fhs.Problem.from_synth(P, mu=KW["mu"], mu_bar=KW["mu_bar"])
    n = prob.solve(KW["max_iter"], KW["rel_tol"], KW["n_reweight"], KW["check_every"])
    img = prob.image().cpu().numpy()
    prob.close()
    return img, n


def test_mix_matches_alone():
    Ps = [synth.make_problem(n, **o) for n, o in MIX]
    sv = fhs.Server(hbm_budget_bytes=8 << 30, max_active=4, check_every=5)
    ids = [sv.submit_synth(P, **KW) for P in Ps]
    results = [sv.wait(i, shape=(P.L, P.ny, P.nx)) for i, P in zip(ids, Ps)]
    sv.close()
    for P, (img, res) in zip(Ps, results):
        assert res.state == fhs.REQ_DONE
        ref, n = _alone(P)
        assert res.iterations == n
        assert rel(img, ref) < 1e-5
    # the same request through a server on its own
    sv = fhs.Server(hbm_budget_bytes=8 << 30, max_active=4, check_every=5)
    img1, r1 = sv.wait(sv.submit_synth(Ps[1], **KW), shape=(Ps[1].L, Ps[1].ny, Ps[1].nx))
    sv.close()
    assert rel(img1, results[1][0]) < 1e-5


def test_admission_respects_budget():
    Ps = [synth.make_problem("small_128", trial=t) for t in range(4)]
    L, M = Ps[0].omega.shape[:2]
    params = fhs.default_params(ny=128, nx=128, n_channels=L, n_subcubes=1, n_blocks=2, qy=2, qx=2,
                                facet_overlap=0.1, mu=0.05, mu_bar=0.5)
    _, peak = fhs.fhs_estimate_bytes(params, None, L * M)
    budget = int(peak * 1.5)                       # room for one problem at a time
    sv = fhs.Server(hbm_budget_bytes=budget, max_active=8, check_every=5)
    ids = [sv.submit_synth(P, **KW) for P in Ps]
    seen = 0
    while True:
        act, q, used = sv.stats()
        assert used <= budget
        seen = max(seen, act)
        if act == 0 and q == 0:
            break
        time.sleep(0.002)
    res = [sv.wait(i)[1] for i in ids]
    sv.close()
    assert all(r.state == fhs.REQ_DONE for r in res)
    assert seen == 1
    # first-in first-out when only one fits: each starts after the previous ended
    for a, b in zip(res, res[1:]):
        assert b.t_start >= a.t_done - 1e-3


def test_request_larger_than_budget_is_refused():
    P = synth.make_problem("tiny")
    sv = fhs.Server(hbm_budget_bytes=1 << 20, max_active=2)
    with pytest.raises(fhs.FhsError) as e:
        sv.submit_synth(P, **KW)
    assert e.value.status == fhs.FHS_ERR_OOM
    sv.close()
