"""Python binding of libfhs (Faceted HyperSARA PDFB on one GB300 GPU).

Argument marshalling only: every entry point forwards to the C ABI declared
in ``include/fhs.h`` (same names), passing raw pointers of numpy host arrays
or torch CUDA tensors and the current torch CUDA stream.  There is no CPU
path: if ``libfhs.so`` is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfhs.so")

FHS_OK, FHS_ERR_ARG, FHS_ERR_OOM, FHS_ERR_CUDA, FHS_ERR_TIMEOUT, FHS_ERR_STATE = range(6)
STATE_IMAGE, STATE_DUAL_DATA, STATE_DUAL_SARA, STATE_DUAL_NUCLEAR, STATE_WEIGHTS_SARA, STATE_WEIGHTS_NUC = range(6)

EXPORTED = [
    "fhs_default_params", "fhs_create_problem", "fhs_create_problem_dde", "fhs_noise_from_model", "fhs_destroy_problem", "fhs_get_info", "fhs_measure",
    "fhs_adjoint", "fhs_sara_analysis", "fhs_sara_synthesis", "fhs_pdfb_step", "fhs_reweight", "fhs_solve",
    "fhs_state_size", "fhs_get_state", "fhs_set_state", "fhs_operator_norms", "fhs_daubechies_filter",
    "fhs_last_error", "fhs_profile_enable", "fhs_profile_read", "fhs_kernel_launches",
    "fhs_sara_analysis_noalloc", "fhs_pdfb_step_batch", "fhs_use_graphs", "fhs_estimate_bytes",
    "fhs_server_create", "fhs_server_submit", "fhs_server_query", "fhs_server_wait", "fhs_server_stats",
    "fhs_server_destroy", "fhs_device_status", "fhs_autotune_bins", "fhs_residual", "fhs_adaptive_noise",
    "fhs_get_image", "fhs_workspace_bytes", "fhs_debug_unsatisfied_wait",
]
REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(4)
GRAM_FP32, GRAM_TF32, GRAM_BF16, GRAM_FP64 = range(4)
PHASES = ["primal", "fft_fwd", "degrid_grid", "l2ball", "fft_inv", "sara", "nuclear", "scatter"]


class FhsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libfhs status %d: %s" % (status, msg))
        self.status = status


class fhs_params(C.Structure):
    _fields_ = [
        ("ny", C.c_int32), ("nx", C.c_int32), ("n_channels", C.c_int32), ("n_subcubes", C.c_int32),
        ("n_blocks", C.c_int32), ("qy", C.c_int32), ("qx", C.c_int32), ("facet_overlap", C.c_double),
        ("kb_taps", C.c_int32), ("wavelet_levels", C.c_int32), ("w_max", C.c_double), ("n_wplanes", C.c_int32),
        ("pixel_size", C.c_double), ("mu", C.c_double), ("mu_bar", C.c_double), ("upsilon", C.c_double),
        ("upsilon_bar", C.c_double), ("tau", C.c_double), ("sigma0", C.c_double), ("sigma1", C.c_double),
        ("sigma2", C.c_double), ("power_iters", C.c_int32), ("power_tol", C.c_double),
        ("gram_precision", C.c_int32), ("data_reduction", C.c_int32),
    ]


class fhs_info(C.Structure):
    _fields_ = [
        ("n_vis", C.c_int64), ("nnz", C.c_int64), ("n_coef", C.c_int64), ("nuclear_size", C.c_int64),
        ("device_bytes", C.c_int64), ("n_facets", C.c_int32), ("iteration", C.c_int32), ("tau", C.c_double),
        ("sigma0", C.c_double), ("sigma1", C.c_double), ("sigma2", C.c_double), ("phi_norm2_max", C.c_double),
        ("n_gfac", C.c_int64), ("bin_dense_min", C.c_int32), ("bin_split", C.c_int32),
        ("mu", C.c_double), ("mu_bar", C.c_double), ("n_red", C.c_int64),
    ]


class fhs_adaptive_params(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("check_every", C.c_int32), ("settle_tol", C.c_double)]


class fhs_adaptive_result(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("n_checks", C.c_int32), ("n_updates", C.c_int32),
                ("satisfied", C.c_int32)]


class fhs_request(C.Structure):
    _fields_ = [
        ("params", fhs_params), ("omega", C.c_void_p), ("w", C.c_void_p), ("y", C.c_void_p),
        ("sigma", C.c_void_p), ("vis_offsets", C.c_void_p), ("block_offsets", C.c_void_p), ("eps", C.c_void_p),
        ("max_iter", C.c_int32), ("n_reweight", C.c_int32), ("rel_tol", C.c_double), ("check_every", C.c_int32),
    ]


class fhs_request_result(C.Structure):
    _fields_ = [
        ("state", C.c_int32), ("status", C.c_int32), ("iterations", C.c_int32), ("rel_change", C.c_double),
        ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double), ("device_bytes", C.c_int64),
    ]


_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libfhs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libfhs.so not found at %s: run __graft_entry__.build() (needs nvcc)" % path)
    lib = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "fhs_default_params": (None, [P(fhs_params)]),
        "fhs_create_problem": (C.c_int, [P(fhs_params), vp, vp, vp, vp, vp, vp, vp, vp, P(vp)]),
        "fhs_create_problem_dde": (C.c_int, [P(fhs_params), vp, vp, vp, vp, vp, vp, vp, vp, vp, P(vp)]),
        "fhs_noise_from_model": (C.c_int, [vp, vp, C.c_int32, vp, vp, vp]),
        "fhs_adaptive_noise": (C.c_int, [vp, P(fhs_adaptive_params), vp, vp, P(fhs_adaptive_result), vp]),
        "fhs_destroy_problem": (None, [vp]),
        "fhs_get_info": (C.c_int, [vp, P(fhs_info)]),
        "fhs_measure": (C.c_int, [vp, vp, vp, vp]),
        "fhs_adjoint": (C.c_int, [vp, vp, vp, vp]),
        "fhs_sara_analysis": (C.c_int, [vp, vp, vp, vp]),
        "fhs_sara_synthesis": (C.c_int, [vp, vp, vp, vp]),
        "fhs_pdfb_step": (C.c_int, [vp, i32, P(dbl), vp]),
        "fhs_reweight": (C.c_int, [vp, vp]),
        "fhs_solve": (C.c_int, [vp, i32, dbl, i32, i32, P(i32), vp]),
        "fhs_state_size": (C.c_int, [vp, i32, P(i64)]),
        "fhs_get_state": (C.c_int, [vp, i32, vp, vp]),
        "fhs_set_state": (C.c_int, [vp, i32, vp, vp]),
        "fhs_operator_norms": (C.c_int, [vp, i32, vp, vp]),
        "fhs_daubechies_filter": (C.c_int, [i32, vp]),
        "fhs_last_error": (C.c_char_p, []),
        "fhs_profile_enable": (C.c_int, [vp, i32]),
        "fhs_profile_read": (C.c_int, [vp, vp, P(i64)]),
        "fhs_kernel_launches": (C.c_int, [vp, P(i64)]),
        "fhs_sara_analysis_noalloc": (C.c_int, [i32, i32, i32, i32, vp, vp, vp]),
        "fhs_pdfb_step_batch": (C.c_int, [vp, i32, i32, vp, vp]),
        "fhs_use_graphs": (C.c_int, [vp, i32]),
        "fhs_estimate_bytes": (C.c_int, [P(fhs_params), vp, i64, P(i64), P(i64)]),
        "fhs_workspace_bytes": (C.c_int, [P(fhs_params), vp, i64, P(i64), P(i64)]),
        "fhs_get_image": (C.c_int, [vp, vp, vp]),
        "fhs_device_status": (C.c_int, [vp, vp]),
        "fhs_debug_unsatisfied_wait": (C.c_int, [vp, i32, vp]),
        "fhs_server_create": (C.c_int, [i64, i32, i32, P(vp)]),
        "fhs_server_submit": (C.c_int, [vp, P(fhs_request), P(i64)]),
        "fhs_server_query": (C.c_int, [vp, i64, P(fhs_request_result)]),
        "fhs_server_wait": (C.c_int, [vp, i64, dbl, vp, P(fhs_request_result)]),
        "fhs_server_stats": (C.c_int, [vp, P(i64), P(i64), P(i64)]),
        "fhs_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != FHS_OK:
        raise FhsError(status, load_library().fhs_last_error().decode())


def _stream(stream):
    """cudaStream_t handle: the given one (an integer handle or a torch stream),
    else torch's current stream (NULL, the legacy default stream, when torch
    sees no CUDA device)."""
    if stream is not None:
        return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    import torch
    if not torch.cuda.is_available():
        return C.c_void_p(0)
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _dev(t, dtype_name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch." + dtype_name):
        raise TypeError("expected a contiguous CUDA torch.%s tensor" % dtype_name)
    return C.c_void_p(t.data_ptr())


def default_params(**kw) -> fhs_params:
    p = fhs_params()
    load_library().fhs_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


# --- entry points (same names as the C ABI) ---------------------------------

def fhs_create_problem(params: fhs_params, omega, w, y, sigma, vis_offsets, block_offsets, eps=None, stream=None,
                       dde=None):
    """Without ``dde`` calls fhs_create_problem; with ``dde`` ([M_tot][5][5]
    complex, the DDE kernel of every visibility) fhs_create_problem_dde."""
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    yc = np.ascontiguousarray(y)
    if np.iscomplexobj(yc):
        yc = np.ascontiguousarray(np.stack([yc.real, yc.imag], axis=-1), dtype=np.float64)
    else:
        yc = np.ascontiguousarray(yc, dtype=np.float64)
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    vis_offsets = np.ascontiguousarray(vis_offsets, dtype=np.int64)
    block_offsets = np.ascontiguousarray(block_offsets, dtype=np.int64)
    eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    h = C.c_void_p()
    if dde is None:
        _check(load_library().fhs_create_problem(C.byref(params), _ptr(omega), _ptr(w), _ptr(yc), _ptr(sigma),
                                                 _ptr(vis_offsets), _ptr(block_offsets), _ptr(eps), _stream(stream),
                                                 C.byref(h)))
    else:
        d = np.asarray(dde, dtype=np.complex128).reshape(-1, 5, 5)
        if d.shape[0] != omega.shape[0]:
            raise ValueError(f"dde holds {d.shape[0]} kernels for {omega.shape[0]} visibilities")
        dd = np.ascontiguousarray(np.stack([d.real, d.imag], axis=-1), dtype=np.float64)
        _check(load_library().fhs_create_problem_dde(C.byref(params), _ptr(omega), _ptr(w), _ptr(yc), _ptr(sigma),
                                                     _ptr(vis_offsets), _ptr(block_offsets), _ptr(eps), _ptr(dd),
                                                     _stream(stream), C.byref(h)))
    return h


def fhs_destroy_problem(prob):
    load_library().fhs_destroy_problem(prob)


def fhs_get_info(prob) -> fhs_info:
    info = fhs_info()
    _check(load_library().fhs_get_info(prob, C.byref(info)))
    return info


def fhs_measure(prob, x, vis, stream=None):
    _check(load_library().fhs_measure(prob, _dev(x, "float32"), _dev(vis, "complex64"), _stream(stream)))


def fhs_adjoint(prob, vis, x, stream=None):
    _check(load_library().fhs_adjoint(prob, _dev(vis, "complex64"), _dev(x, "float32"), _stream(stream)))


def fhs_residual(prob, x, r, stream=None):
    """r = eta Re Phi^H (y - Phi x); x None gives the dirty image."""
    xp = C.c_void_p(None) if x is None else _dev(x, "float32")
    _check(load_library().fhs_residual(prob, xp, _dev(r, "float32"), _stream(stream)))


def fhs_noise_from_model(prob, x0, n_out, apply=False, stream=None):
    """(sigma, eps) float64 arrays of n_out values (blocks, or channels with data
    reduction) from the model cube x0; apply=True makes eps the l2 bounds."""
    sig = np.zeros(n_out)
    eps = np.zeros(n_out)
    _check(load_library().fhs_noise_from_model(prob, _dev(x0, "float32"), int(bool(apply)), _ptr(sig), _ptr(eps),
                                               _stream(stream)))
    return sig, eps


def fhs_adaptive_noise(prob, n_out, max_iter, check_every=10, settle_tol=1e-3, stream=None):
    """Adaptive noise estimation (Sec. 3.3 (ii)) on a problem that has not
    iterated: (sigma, eps, result) with n_out values each (blocks, or channels
    with data reduction) and result a dict of the counts."""
    ap = fhs_adaptive_params(int(max_iter), int(check_every), float(settle_tol))
    res = fhs_adaptive_result()
    sig = np.zeros(n_out)
    eps = np.zeros(n_out)
    _check(load_library().fhs_adaptive_noise(prob, C.byref(ap), _ptr(sig), _ptr(eps), C.byref(res),
                                             _stream(stream)))
    return sig, eps, {k: int(getattr(res, k)) for k, _ in fhs_adaptive_result._fields_}


def fhs_sara_analysis(prob, x, coef, stream=None):
    _check(load_library().fhs_sara_analysis(prob, _dev(x, "float32"), _dev(coef, "float32"), _stream(stream)))


def sara_coefficient_count(ny, nx, levels, n_db=8):
    """Coefficients per image of fhs_sara_analysis: the Dirac block plus, per
    basis db_p (filter length 2p), the three detail bands of every level and
    the last approximation, level sides n_{j+1} = floor((n_j + 2p - 1) / 2)."""
    n = int(ny) * int(nx)
    for p in range(1, n_db + 1):
        a, b = int(ny), int(nx)
        for _ in range(int(levels)):
            a, b = (a + 2 * p - 1) // 2, (b + 2 * p - 1) // 2
            n += 3 * a * b
        n += a * b
    return n


def fhs_sara_analysis_noalloc(ny, nx, n_images, levels, x, coef, stream=None):
    """SARA analysis for callers that cannot allocate device memory (static
    16 MiB scratch shared by all calls; overlapping calls race).  The tensors
    are checked against the sizes first: the C entry point cannot see how
    large the buffers behind its pointers are."""
    ny, nx, n_images, levels = int(ny), int(nx), int(n_images), int(levels)
    need_x = n_images * ny * nx
    need_c = n_images * sara_coefficient_count(ny, nx, levels) if ny > 0 and nx > 0 and levels > 0 else 0
    if x.numel() < need_x or coef.numel() < need_c:
        raise FhsError(FHS_ERR_ARG, "fhs_sara_analysis_noalloc: x holds %d of %d floats, coef %d of %d"
                       % (x.numel(), need_x, coef.numel(), need_c))
    _check(load_library().fhs_sara_analysis_noalloc(ny, nx, n_images, levels, _dev(x, "float32"),
                                                    _dev(coef, "float32"), _stream(stream)))


def fhs_sara_synthesis(prob, coef, x, stream=None):
    _check(load_library().fhs_sara_synthesis(prob, _dev(coef, "float32"), _dev(x, "float32"), _stream(stream)))


def fhs_pdfb_step(prob, n_iter=1, want_rel=False, stream=None):
    rel = C.c_double(0.0)
    _check(load_library().fhs_pdfb_step(prob, int(n_iter), C.byref(rel) if want_rel else None, _stream(stream)))
    return rel.value if want_rel else None


def fhs_reweight(prob, stream=None):
    _check(load_library().fhs_reweight(prob, _stream(stream)))


def fhs_solve(prob, max_iter, rel_tol, n_reweight=0, check_every=10, stream=None):
    it = C.c_int32(0)
    _check(load_library().fhs_solve(prob, int(max_iter), float(rel_tol), int(n_reweight), int(check_every),
                                    C.byref(it), _stream(stream)))
    return it.value


def fhs_state_size(prob, part) -> int:
    n = C.c_int64(0)
    _check(load_library().fhs_state_size(prob, int(part), C.byref(n)))
    return n.value


def fhs_get_state(prob, part, dst, stream=None):
    _check(load_library().fhs_get_state(prob, int(part), _dev(dst, "float32"), _stream(stream)))


def fhs_get_image(prob, x, stream=None):
    _check(load_library().fhs_get_image(prob, _dev(x, "float32"), _stream(stream)))


def fhs_set_state(prob, part, src, stream=None):
    _check(load_library().fhs_set_state(prob, int(part), _dev(src, "float32"), _stream(stream)))


def fhs_operator_norms(prob, n_iter, L, stream=None) -> np.ndarray:
    out = np.zeros(L, dtype=np.float64)
    _check(load_library().fhs_operator_norms(prob, int(n_iter), _ptr(out), _stream(stream)))
    return out


def fhs_daubechies_filter(p: int) -> np.ndarray:
    out = np.zeros(2 * p, dtype=np.float64)
    _check(load_library().fhs_daubechies_filter(int(p), _ptr(out)))
    return out


def fhs_pdfb_step_batch(probs, n_iter=1, streams=None, want_rel=False):
    """n_iter iterations of several problems, problem k on streams[k] (ints or torch streams)."""
    n = len(probs)
    arr = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in probs])
    sarr = None
    if streams is not None:
        sarr = (C.c_void_p * n)(*[int(getattr(st, "cuda_stream", st)) for st in streams])
    rel = np.zeros(n, dtype=np.float64)
    _check(load_library().fhs_pdfb_step_batch(arr, n, int(n_iter), sarr, _ptr(rel) if want_rel else None))
    return rel if want_rel else None


def fhs_use_graphs(prob, on: bool):
    _check(load_library().fhs_use_graphs(prob, 1 if on else 0))


def fhs_estimate_bytes(params: fhs_params, w, n_vis: int):
    """(resident, peak) device bytes of a problem before creating it."""
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    r, pk = C.c_int64(0), C.c_int64(0)
    _check(load_library().fhs_estimate_bytes(C.byref(params), _ptr(w), int(n_vis), C.byref(r), C.byref(pk)))
    return r.value, pk.value


def fhs_workspace_bytes(params: fhs_params, w, n_vis: int):
    """(resident, peak) device bytes; the same query as fhs_estimate_bytes."""
    w = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    r, pk = C.c_int64(0), C.c_int64(0)
    _check(load_library().fhs_workspace_bytes(C.byref(params), _ptr(w), int(n_vis), C.byref(r), C.byref(pk)))
    return r.value, pk.value


def fhs_profile_enable(prob, on: bool):
    _check(load_library().fhs_profile_enable(prob, 1 if on else 0))


def fhs_profile_read(prob):
    """(dict phase -> summed ms, timed iterations)."""
    ms = np.zeros(len(PHASES), dtype=np.float64)
    it = C.c_int64(0)
    _check(load_library().fhs_profile_read(prob, _ptr(ms), C.byref(it)))
    return dict(zip(PHASES, ms.tolist())), it.value


def fhs_device_status(prob, stream=None):
    """Raise FhsError(FHS_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(load_library().fhs_device_status(prob, _stream(stream)))


def fhs_debug_unsatisfied_wait(prob, max_polls, stream=None):
    """Test aid: a device wait that runs out and records a timeout in the problem's flag."""
    _check(load_library().fhs_debug_unsatisfied_wait(prob, int(max_polls), _stream(stream)))


def fhs_autotune_bins(prob, stream=None):
    """Time candidate tile binnings of the pass over G and keep the fastest;
    returns (dense_min, split) of the binning in use afterwards."""
    dm, sp = C.c_int32(0), C.c_int32(0)
    _check(load_library().fhs_autotune_bins(prob, _stream(stream), C.byref(dm), C.byref(sp)))
    return dm.value, sp.value


def fhs_kernel_launches(prob) -> int:
    n = C.c_int64(0)
    _check(load_library().fhs_kernel_launches(prob, C.byref(n)))
    return n.value


class Server:
    """Serving loop of libfhs (native threads): submit imaging requests, wait for images."""

    def __init__(self, hbm_budget_bytes: int, max_active: int = 8, check_every: int = 10):
        h = C.c_void_p()
        _check(load_library().fhs_server_create(int(hbm_budget_bytes), int(max_active), int(check_every),
                                                C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, params: fhs_params, omega, w, y, sigma, vis_offsets, block_offsets, max_iter, rel_tol,
               n_reweight=0, check_every=0, eps=None) -> int:
        arrs = dict(omega=np.ascontiguousarray(omega, dtype=np.float64),
                    w=None if w is None else np.ascontiguousarray(w, dtype=np.float64),
                    y=np.ascontiguousarray(np.stack([np.real(y), np.imag(y)], -1) if np.iscomplexobj(y) else y,
                                           dtype=np.float64),
                    sigma=np.ascontiguousarray(sigma, dtype=np.float64),
                    vis_offsets=np.ascontiguousarray(vis_offsets, dtype=np.int64),
                    block_offsets=np.ascontiguousarray(block_offsets, dtype=np.int64),
                    eps=None if eps is None else np.ascontiguousarray(eps, dtype=np.float64))
        req = fhs_request(params=params, max_iter=int(max_iter), n_reweight=int(n_reweight), rel_tol=float(rel_tol),
                          check_every=int(check_every))
        for k, a in arrs.items():
            setattr(req, k, None if a is None else a.ctypes.data)
        rid = C.c_int64(0)
        _check(load_library().fhs_server_submit(self.handle, C.byref(req), C.byref(rid)))   # copies the arrays
        return rid.value

    def submit_synth(self, prob, mu, mu_bar, max_iter, rel_tol, n_reweight=0, check_every=0, **kw) -> int:
        L, M = prob.omega.shape[:2]
        params = default_params(ny=prob.ny, nx=prob.nx, n_channels=L, n_subcubes=prob.C, n_blocks=prob.B,
                                qy=prob.qy, qx=prob.qx, facet_overlap=prob.overlap, w_max=prob.w_max,
                                pixel_size=prob.pixel_size, mu=mu, mu_bar=mu_bar)
        for k, v in kw.items():
            setattr(params, k, v)
        return self.submit(params, prob.omega.reshape(-1, 2), prob.w.reshape(-1), prob.y.reshape(-1), prob.sigma,
                           np.arange(L + 1, dtype=np.int64) * M, prob.block_offsets, max_iter, rel_tol, n_reweight,
                           check_every)

    def query(self, rid: int) -> fhs_request_result:
        r = fhs_request_result()
        _check(load_library().fhs_server_query(self.handle, int(rid), C.byref(r)))
        return r

    def wait(self, rid: int, shape=None, timeout: float = -1.0):
        r = fhs_request_result()
        img = None if shape is None else np.empty(shape, dtype=np.float32)
        _check(load_library().fhs_server_wait(self.handle, int(rid), float(timeout),
                                              None if img is None else img.ctypes.data, C.byref(r)))
        return img, r

    def stats(self):
        a, q, b = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        _check(load_library().fhs_server_stats(self.handle, C.byref(a), C.byref(q), C.byref(b)))
        return a.value, q.value, b.value

    def close(self):
        if self.handle:
            load_library().fhs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- convenience wrapper ----------------------------------------------------

class Problem:
    """Owns one libfhs problem built from host arrays; device tensors via torch."""

    def __init__(self, params: fhs_params, omega, w, y, sigma, vis_offsets, block_offsets, eps=None, stream=None,
                 dde=None):
        self.params = params
        self.L = int(params.n_channels)
        self.ny, self.nx = int(params.ny), int(params.nx)
        self.handle = fhs_create_problem(params, omega, w, y, sigma, vis_offsets, block_offsets, eps, stream, dde)
        self.info = fhs_get_info(self.handle)

    @classmethod
    def from_synth(cls, prob, mu, mu_bar, stream=None, dde=None, **kw):
        """Build from a ``synth.Problem`` (all channels share one visibility count);
        ``dde`` (L, M, 5, 5) complex folds DDE kernels into G."""
        L, M = prob.omega.shape[:2]
        params = default_params(ny=prob.ny, nx=prob.nx, n_channels=L, n_subcubes=prob.C, n_blocks=prob.B,
                                qy=prob.qy, qx=prob.qx, facet_overlap=prob.overlap, w_max=prob.w_max,
                                pixel_size=prob.pixel_size, mu=mu, mu_bar=mu_bar)
        for k, v in kw.items():
            setattr(params, k, v)
        vis_off = np.arange(L + 1, dtype=np.int64) * M
        return cls(params, prob.omega.reshape(-1, 2), prob.w.reshape(-1), prob.y.reshape(-1), prob.sigma,
                   vis_off, prob.block_offsets, None, stream, dde)

    def close(self):
        if self.handle:
            fhs_destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _img(self):
        import torch
        return torch.empty((self.L, self.ny, self.nx), dtype=torch.float32, device="cuda")

    @staticmethod
    def _need(t, n, what):
        """The C entry points take bare device pointers and cannot see how
        large the buffers behind them are: a caller's tensor of the wrong size
        is refused here, before any device work."""
        if t.numel() != n:
            raise FhsError(FHS_ERR_ARG, "%s holds %d elements, the problem needs %d" % (what, t.numel(), n))

    def measure(self, x):
        import torch
        self._need(x, self.L * self.ny * self.nx, "image cube x")
        vis = torch.empty(self.info.n_vis, dtype=torch.complex64, device="cuda")
        fhs_measure(self.handle, x, vis)
        return vis

    def adjoint(self, vis):
        self._need(vis, self.info.n_vis, "visibilities vis")
        x = self._img()
        fhs_adjoint(self.handle, vis, x)
        return x

    def residual(self, x=None):
        """eta_l Re Phi_l^H (y_l - Phi_l x_l); the dirty image when x is None."""
        if x is not None:
            self._need(x, self.L * self.ny * self.nx, "image cube x")
        r = self._img()
        fhs_residual(self.handle, x, r)
        return r

    def noise_from_model(self, x0, apply=False):
        """Noise levels and l2 bounds from a model cube (per block; per channel with
        data reduction)."""
        self._need(x0, self.L * self.ny * self.nx, "model cube x0")
        n = self.L if int(self.params.data_reduction) else self.L * int(self.params.n_blocks)
        return fhs_noise_from_model(self.handle, x0, n, apply)

    def adaptive_noise(self, max_iter, check_every=10, settle_tol=1e-3):
        """Adaptive noise estimation (Sec. 3.3 (ii)) before the run: (sigma, eps, counts)."""
        n = self.L if int(self.params.data_reduction) else self.L * int(self.params.n_blocks)
        out = fhs_adaptive_noise(self.handle, n, max_iter, check_every, settle_tol)
        self.info = fhs_get_info(self.handle)
        return out

    def sara_analysis(self, x):
        import torch
        self._need(x, self.L * self.ny * self.nx, "image cube x")
        c = torch.empty((self.L, self.info.n_coef), dtype=torch.float32, device="cuda")
        fhs_sara_analysis(self.handle, x, c)
        return c

    def sara_synthesis(self, c):
        self._need(c, self.L * self.info.n_coef, "coefficients c")
        x = self._img()
        fhs_sara_synthesis(self.handle, c, x)
        return x

    def step(self, n_iter=1, want_rel=False):
        return fhs_pdfb_step(self.handle, n_iter, want_rel)

    def reweight(self):
        fhs_reweight(self.handle)

    def solve(self, max_iter, rel_tol, n_reweight=0, check_every=10):
        return fhs_solve(self.handle, max_iter, rel_tol, n_reweight, check_every)

    def get_state(self, part):
        import torch
        t = torch.empty(fhs_state_size(self.handle, part), dtype=torch.float32, device="cuda")
        fhs_get_state(self.handle, part, t)
        return t

    def set_state(self, part, t):
        self._need(t, fhs_state_size(self.handle, part), "state part %d" % int(part))
        fhs_set_state(self.handle, part, t)

    def image(self):
        x = self._img()
        fhs_get_image(self.handle, x)
        return x

    def operator_norms(self, n_iter=100):
        return fhs_operator_norms(self.handle, n_iter, self.L)

    def autotune_bins(self, stream=None):
        """Measure candidate binnings of the pass over G; keep the fastest."""
        out = fhs_autotune_bins(self.handle, stream)
        self.info = fhs_get_info(self.handle)
        return out
