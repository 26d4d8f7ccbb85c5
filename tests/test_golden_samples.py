"""The stored oracle runs on the two benchmark geometries (tests/golden/
fhs_<side>_samples.npz, written by tests/golden/make_fhs_samples.py) agree
with the script that writes them: the workload, visibility count, iteration
and reweighting schedule and regularisation it names, step sizes that follow
the rules of the PDFB reading (tau = 0.99/3, sigma1 = 1, sigma0 = 1 / the
largest facet coverage of the geometry), and samples whose indices are
distinct, sorted and inside the arrays they were drawn from.  No GPU and no
oracle iteration: the files are read as they are."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_fhs_samples as mk  # noqa: E402
from oracle import prox  # noqa: E402
from paper_2209_07604_gb300 import synth  # noqa: E402


@pytest.mark.parametrize("side", sorted(mk.RUNS))
def test_stored_run_matches_its_script(side):
    d = np.load(mk.out_path(side))
    workload, m_per_channel, n_iter, n_reweight = mk.RUNS[side]
    assert str(d["workload"]) == workload
    assert int(d["m_per_channel"]) == m_per_channel
    assert int(d["n_iter"]) == n_iter and int(d["n_reweight"]) == n_reweight
    assert float(d["mu"]) == mk.MU and float(d["mu_bar"]) == mk.MU_BAR
    spec = synth.WORKLOADS[workload]
    ny, nx, L, C = spec["ny"], spec["nx"], spec["L"], spec["C"]
    facets = prox.nuclear_facets(ny, nx, spec["qy"], spec["qx"], spec["overlap"])
    cov = prox.facet_coverage(ny, nx, facets).max()
    assert abs(float(d["tau"]) - 0.99 / 3.0) < 1e-15
    assert float(d["sigma1"]) == 1.0
    assert abs(float(d["sigma0"]) - 1.0 / cov) < 1e-15
    assert 0.0 < float(d["sigma2"]) < 1.0
    assert int(d["lc"]) == L // C
    n_pix = L * ny * nx
    n_nuc = sum(L // C * (y1 - y0) * (x1 - x0) for (y0, y1, x0, x1) in facets) * C
    sizes = {"X": n_pix, "v": L * m_per_channel, "W": L * int(d["n_coef"]), "P": n_nuc,
             "w21": C * int(d["n_coef"])}
    for name, size in sizes.items():
        idx = d[name + "_idx"]
        assert idx.dtype == np.int64 and idx.size == d[name].size
        assert np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < size, name
        assert np.abs(d[name]).max() <= float(d[name + "_absmax"])
        assert np.isfinite(d[name]).all()
    wn = d["wnuc"]
    assert wn.size == C * len(facets) * (L // C)
    assert np.all((wn > 0) & (wn <= 1)), "log-sum weights lie in (0, 1]"
    assert np.all((d["w21"] > 0) & (d["w21"] <= 1))
