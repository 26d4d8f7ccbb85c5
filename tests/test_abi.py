"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/fhs.h, rejects bad arguments before
touching the device, and computes its own Daubechies filters (compared with
the oracle's and with the published closed forms)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2209_07604_gb300 as fhs
from oracle import wavelets as wv

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_07604_gb300 import build
    build.build()
    return fhs.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fhs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fhs_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree(lib):
    decl = declared_symbols()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(lib, name), name
    assert sorted(fhs.EXPORTED) == decl


def test_library_filters_match_oracle(lib):
    for p in range(1, 9):
        np.testing.assert_allclose(fhs.fhs_daubechies_filter(p), wv.daubechies(p), rtol=0, atol=1e-13)


def test_bad_filter_order_is_rejected(lib):
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_daubechies_filter(9)
    assert e.value.status == fhs.FHS_ERR_ARG


def _args(L=2, M=10, B=2):
    om = np.zeros((L * M, 2))
    y = np.zeros((L * M, 2))
    sig = np.ones(L)
    vo = np.arange(L + 1, dtype=np.int64) * M
    bo = np.array([[0, M // 2, M]] * L, dtype=np.int64)
    return om, y, sig, vo, bo


@pytest.mark.parametrize("field,value", [("ny", 15), ("nx", 8), ("n_subcubes", 3), ("n_blocks", 0),
                                         ("facet_overlap", 1.0), ("wavelet_levels", 9), ("mu", float("nan")),
                                         ("upsilon", 0.0), ("qy", 0), ("data_reduction", 2)])
def test_invalid_params_rejected_without_device(lib, field, value):
    p = fhs.default_params(ny=32, nx=32, n_channels=2, n_subcubes=1, n_blocks=2, mu=0.1, mu_bar=0.1)
    setattr(p, field, value)
    om, y, sig, vo, bo = _args()
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_create_problem(p, om, None, y, sig, vo, bo)
    assert e.value.status == fhs.FHS_ERR_ARG
    assert lib.fhs_last_error().decode()


def test_invalid_inputs_rejected_without_device(lib):
    p = fhs.default_params(ny=32, nx=32, n_channels=2, n_subcubes=1, n_blocks=2)
    om, y, sig, vo, bo = _args()
    om[3, 0] = 4.0                                   # outside [-pi, pi)
    with pytest.raises(fhs.FhsError):
        fhs.fhs_create_problem(p, om, None, y, sig, vo, bo)
    om, y, sig, vo, bo = _args()
    bo[1, 2] = 9                                     # blocks must end at M_l
    with pytest.raises(fhs.FhsError):
        fhs.fhs_create_problem(p, om, None, y, sig, vo, bo)
    om, y, sig, vo, bo = _args()
    sig[0] = 0.0
    with pytest.raises(fhs.FhsError):
        fhs.fhs_create_problem(p, om, None, y, sig, vo, bo)
    om, y, sig, vo, bo = _args()
    y[0, 0] = np.nan
    with pytest.raises(fhs.FhsError):
        fhs.fhs_create_problem(p, om, None, y, sig, vo, bo)


def test_params_struct_layout(lib):
    # the ctypes mirror must have the C layout: defaults written by the library read back sanely
    p = fhs.default_params()
    assert p.kb_taps == 7 and p.wavelet_levels == 4 and p.n_wplanes == 64 and p.power_iters == 100
    assert abs(p.upsilon - 1e-3) < 1e-18 and abs(p.power_tol - 1e-7) < 1e-20
    assert p.gram_precision == fhs.GRAM_FP32 and p.data_reduction == 0
    # 7 int32 + pad, double, 2 int32, double, int32 + pad, 9 doubles, int32 + pad, double, 2 int32
    assert C.sizeof(fhs.fhs_params) == 160


def test_estimate_bytes_counts_g_factors(lib):
    """The footprint estimate is host-only; with the same visibility count,
    w-terms change it by exactly 8 bytes per extra stored G value (each row
    keeps its two 1-D factors of 7 + 2h taps)."""
    p = fhs.default_params(ny=64, nx=64, n_channels=2, n_subcubes=1, n_blocks=2, qy=2, qx=2, facet_overlap=0.1,
                           w_max=2000.0, pixel_size=1e-4)
    M = 5000
    w = np.linspace(0.0, 2000.0, M)
    r0, pk0 = fhs.fhs_estimate_bytes(p, np.zeros(M), M)
    r1, pk1 = fhs.fhs_estimate_bytes(p, w, M)
    P1 = p.n_wplanes - 1
    pa = np.minimum(np.floor(np.abs(w) / (2000.0 / P1) + 0.5).astype(np.int64), P1)
    T = 7 + 2 * ((8 * pa + P1) // (2 * P1))
    assert r1 - r0 == 8 * int(np.sum(2 * T - 14))
    assert pk0 > r0 and pk1 > r1
    r2, _ = fhs.fhs_estimate_bytes(p, np.zeros(2 * M), 2 * M)
    assert r2 > r0
    # data reduction keeps Lambda, y', the reduced dual and two work grids per channel
    p.data_reduction = 1
    r3, pk3 = fhs.fhs_estimate_bytes(p, np.zeros(M), M)
    K, L = 4 * 64 * 64, 2
    assert r3 - r0 == 36 * K * L + 20 * L and pk3 - pk0 == r3 - r0 + 8 * K * L


def test_dde_rejections_without_device(lib):
    """fhs_create_problem_dde refuses a NULL kernel array, and boxes that the 4
    DDE taps would widen past 16 (w-kernels of 4 extra taps per side at w_max),
    before touching the device."""
    p = fhs.default_params(ny=32, nx=32, n_channels=2, n_subcubes=1, n_blocks=2, w_max=2000.0, pixel_size=1e-4)
    om, y, sig, vo, bo = _args()
    h = C.c_void_p()
    st = lib.fhs_create_problem_dde(C.byref(p), om.ctypes.data_as(C.c_void_p), None, y.ctypes.data_as(C.c_void_p),
                                    sig.ctypes.data_as(C.c_void_p), vo.ctypes.data_as(C.c_void_p),
                                    bo.ctypes.data_as(C.c_void_p), None, None, None, C.byref(h))
    assert st == fhs.FHS_ERR_ARG and not h.value
    dde = np.zeros((len(om), 5, 5), dtype=np.complex128)
    dde[:, 2, 2] = 1.0
    w = np.full(len(om), 2000.0)
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_create_problem(p, om, w, y, sig, vo, bo, dde=dde)
    assert e.value.status == fhs.FHS_ERR_ARG
    assert "16 taps" in lib.fhs_last_error().decode()
    with pytest.raises(ValueError):
        fhs.fhs_create_problem(p, om, w, y, sig, vo, bo, dde=dde[:3])


def test_problem_methods_refuse_tensors_of_the_wrong_size():
    """The C entry points take bare pointers; the Problem methods check the
    caller's tensors against the problem's sizes first and raise
    FHS_ERR_ARG before any device work (here with CPU tensors and no
    problem handle: nothing reaches the library)."""
    torch = pytest.importorskip("torch")
    p = fhs.Problem.__new__(fhs.Problem)
    p.handle, p.L, p.ny, p.nx = None, 2, 16, 24
    p.params = fhs.fhs_params()
    p.info = fhs.fhs_info()
    p.info.n_vis, p.info.n_coef = 100, 1000
    short_img = torch.zeros(2 * 16 * 24 - 1)
    for call in (lambda: p.measure(short_img), lambda: p.residual(short_img), lambda: p.sara_analysis(short_img),
                 lambda: p.noise_from_model(short_img), lambda: p.adjoint(torch.zeros(101, dtype=torch.complex64)),
                 lambda: p.sara_synthesis(torch.zeros(2 * 1000 + 1))):
        with pytest.raises(fhs.FhsError) as e:
            call()
        assert e.value.status == fhs.FHS_ERR_ARG
