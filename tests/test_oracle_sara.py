"""Pins of the oracle SARA dictionary (Sec. 2.2.2): published closed-form
filters, filter identities, a hand-worked Haar level, level sizes, Parseval,
the adjoint, and exact agreement of the faceted transform with the global
one."""
import math
import os

import numpy as np
import pytest

from oracle import wavelets as wv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _closed_forms():
    env = {"r2": math.sqrt(2), "r3": math.sqrt(3), "r10": math.sqrt(10),
           "s": math.sqrt(5 + 2 * math.sqrt(10))}
    out = {}
    with open(os.path.join(GOLDEN, "daubechies_closed_form.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, rest = line.split(None, 1)
            out[int(name[2:])] = np.array([eval(e, {}, env) for e in rest.split(";")])
    return out


def test_daubechies_closed_forms():
    for p, h in _closed_forms().items():
        np.testing.assert_allclose(wv.daubechies(p), h, rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", range(1, 9))
def test_daubechies_identities(p):
    h = wv.daubechies(p)
    F = len(h)
    assert F == 2 * p
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    assert abs((h * h).sum() - 1.0) < 1e-13
    for m in range(1, p):
        assert abs(np.dot(h[: F - 2 * m], h[2 * m:])) < 1e-13
    g = wv.highpass(h)
    k = np.arange(F, dtype=np.float64)
    for j in range(p):            # p vanishing moments of the wavelet
        assert abs(np.sum(g * k ** j)) < 1e-12 * np.sum(np.abs(g) * k ** j) + 1e-13
    # minimum phase: the zeros of H(z) away from the p-fold zero at z = -1
    # (numerically split, so left out) lie strictly inside the unit circle
    r = np.roots(h)
    far = np.abs(r + 1.0) > 0.2
    assert far.sum() == p - 1
    assert np.all(np.abs(r[far]) < 1.0)


def test_haar_level_by_hand():
    a = np.array([[1.0, 3.0, -2.0, 5.0]])
    h = wv.daubechies(1)
    lo = wv.analysis_axis(a, h, -1)
    hi = wv.analysis_axis(a, wv.highpass(h), -1)
    r = 1 / math.sqrt(2)
    np.testing.assert_allclose(lo, [[4 * r, 3 * r]], atol=1e-15)
    np.testing.assert_allclose(hi, [[2 * r, 7 * r]], atol=1e-15)


def test_level_sizes_golden():
    with open(os.path.join(GOLDEN, "wavelet_sizes.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n0, F, *ns = map(int, line.split())
            got = [s[0] for s in wv.level_shapes(n0, n0, F, 4)[1:]]
            assert got == ns


@pytest.mark.parametrize("ny,nx", [(64, 48), (37, 53), (16, 16)])
def test_parseval_and_adjoint(ny, nx):
    S = wv.Sara(ny, nx)
    rng = np.random.default_rng(ny * nx)
    x = rng.standard_normal((2, ny, nx))
    c = S.analysis(x)
    assert abs(np.sum(c * c) - np.sum(x * x)) < 1e-12 * np.sum(x * x)
    np.testing.assert_allclose(S.synthesis(c), x, atol=1e-12)
    z = rng.standard_normal(c.shape)
    assert abs(np.vdot(c, z) - np.vdot(x, S.synthesis(z))) < 1e-11 * np.linalg.norm(z) * np.linalg.norm(x)


@pytest.mark.parametrize("ny,nx,qy,qx", [(64, 48, 2, 3), (128, 128, 2, 2), (37, 53, 3, 2), (96, 160, 3, 2)])
def test_faceted_equals_global(ny, nx, qy, qx):
    """Sec. 2.2.2: the wavelet dictionary decomposes exactly over overlapping facets."""
    S = wv.Sara(ny, nx)
    FS = wv.FacetedSara(ny, nx, qy, qx)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, ny, nx))
    c = S.analysis(x)
    cf = FS.analysis(x)
    assert np.abs(cf - c).max() <= 1e-13 * np.abs(c).max()
    z = rng.standard_normal(c.shape)
    assert np.abs(FS.synthesis(z) - S.synthesis(z)).max() <= 1e-12 * np.abs(z).max()
    # sum over facets of the l21 norm equals the global l21 norm (ownership partitions rows)
    assert S.n_coef == FS.n_coef
