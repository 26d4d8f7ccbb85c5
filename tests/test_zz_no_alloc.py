"""fhs_sara_analysis_noalloc: the SARA analysis for callers that cannot
allocate device memory.

Some callers run with all of their device memory already handed to another
allocator (a framework's caching allocator or a fixed pool), or inside loops
where a cudaMalloc, and the device synchronisation it can bring, is not
acceptable.  For them the library offers one entry point whose scratch is a
static 16 MiB device array instead of memory it allocates.  This test calls
it through the C ABI twice in a row, on two different inputs, and checks each
result against the regular fhs_sara_analysis of a problem handle.  It lives
in its own file, collected last, and passes alone or after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_2209_07604_gb300 as fhs
from parity import rel
from paper_2209_07604_gb300 import synth

TOL_OP = 1e-5




@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07604_gb300 import build
    build.build()
    fhs.load_library()


def test_noalloc_analysis_matches_problem_analysis_twice():
    ny, nx, L, levels = 96, 160, 3, 4
    P = synth.make_problem("tiny", L=L)
    prob = fhs.Problem.from_synth(P, mu=0.0, mu_bar=0.0, sigma2=1.0, ny=ny, nx=nx, wavelet_levels=levels)
    n_coef = prob.info.n_coef
    from oracle import wavelets as owv
    S = owv.Sara(ny, nx, levels)
    assert fhs.sara_coefficient_count(ny, nx, levels) == n_coef == S.n_coef
    xs = [torch.tensor(synth.random_image((L, ny, nx), seed, nonneg=False), dtype=torch.float32, device="cuda")
          for seed in (21, 22)]
    for x in xs:                              # two calls in a row, different inputs
        ref = prob.sara_analysis(x).cpu().numpy()
        out = torch.full((L, n_coef), float("nan"), dtype=torch.float32, device="cuda")
        fhs.fhs_sara_analysis_noalloc(ny, nx, L, levels, x, out)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), "some coefficients were not written"
        assert rel(got, ref) < TOL_OP
        # and against the FP64 oracle's analysis of the same images
        assert rel(got, S.analysis(x.cpu().numpy().astype(np.float64))) < TOL_OP
    prob.close()


def test_noalloc_rejects_images_beyond_the_static_scratch():
    """The C entry point itself refuses sizes beyond its static scratch (called
    directly: the Python wrapper would refuse the small buffers first)."""
    import ctypes
    lib = fhs.load_library()
    x = torch.zeros((1, 16, 16), dtype=torch.float32, device="cuda")
    c = torch.zeros((1, 16), dtype=torch.float32, device="cuda")
    st = lib.fhs_sara_analysis_noalloc(2048, 2048, 1, 4, ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(c.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == fhs.FHS_ERR_ARG
    assert "static maximum" in lib.fhs_last_error().decode()


def test_noalloc_wrapper_checks_buffer_sizes():
    x = torch.zeros((1, 64, 64), dtype=torch.float32, device="cuda")
    c = torch.zeros((1, 100), dtype=torch.float32, device="cuda")
    with pytest.raises(fhs.FhsError) as e:
        fhs.fhs_sara_analysis_noalloc(64, 64, 1, 4, x, c)
    assert e.value.status == fhs.FHS_ERR_ARG
