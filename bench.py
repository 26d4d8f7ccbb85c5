"""Benchmark: Faceted HyperSARA PDFB iterations/s on one GB300 (libfhs).

One step = one PDFB iteration of the whole hot path (primal step, F, the dual
pass over G with the data-dual update, the l2-ball factors, the scatter pass
over G, F^H, SARA analysis + weighted l21 dual + synthesis, per-facet Gram +
FP64 eig + SVT dual) over the workload, by default the 2048 x 2048,
32-channel, 1.28e8-visibility imaging configuration (4 spectral sub-cubes,
8 x 8 facets, 8 blocks).  Prints one JSON line.  ``--impl reference`` times
the FP64 CPU oracle on a bounded sample of the same workload instead, on all
host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "vla_2048"


def _metric(workload: str) -> str:
    from paper_2209_07604_gb300 import synth
    sp = synth.WORKLOADS[workload]
    w = ", w-projection" if sp["w_max"] > 0 else ""
    return ("PDFB iter/s (%d^2 x %d ch, %.3g vis%s); Phi/Phi^H vis/s alongside"
            % (sp["ny"], sp["L"], sp["L"] * sp["M"], w))

MU, MU_BAR = 1e-2, 1e-1            # regularisation used for timing (cost does not depend on it)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi SM clock / throttle sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.rows.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 3 + i and r[3 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(value: float) -> float:
    """Largest value over the ranks of the default process group (the job's
    time is its slowest rank's); identity when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _profile_traffic(workload: str, kernel_file: str):
    """DRAM bytes per full launch of the dual and the scatter pass over G at
    the workload, and the limiter line, from the committed ncu summary
    profiles/data_term_passes_<workload>.md; valid only while the kernel
    source is unchanged (its sha256 is recorded there).  None otherwise."""
    path = os.path.join(ROOT, "profiles", "data_term_passes_%s.md" % workload)
    src = os.path.join(ROOT, "paper_2209_07604_gb300", "csrc", kernel_file)
    try:
        txt = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    m_sha = re.search(r"kernel source sha256:\s*([0-9a-f]{64})", txt)
    if not m_sha or m_sha.group(1) != sha:
        return None
    out = {}
    for key in ("dual", "scatter"):
        m = re.search(r"^%s pass dram bytes per full launch:\s*([0-9.eE+]+)" % key, txt, re.M)
        out[key] = float(m.group(1)) if m else None
    for key in ("dual", "scatter"):
        m = re.search(r"^%s pass limiter:\s*(.+)$" % key, txt, re.M)
        out[key + "_limiter"] = m.group(1).strip() if m else None
    return out


def data_term_bytes(info, L, KH, M):
    """Algorithmic HBM bytes of the data term's two passes over G, (dual,
    scatter).  Dual pass: G factors 8 B per stored value (2T per row), per row
    meta 8 B + factor offset 8 B, per visibility y 8 B and the dual d read
    8 B + written 8 B, the forward spectrum read once (its stored half: KH
    complex cells per channel).  Scatter pass: the factors, meta and offsets
    again, d read 8 B, the folded adjoint written once (KH cells)."""
    dual = info.n_gfac * 8 + M * (8 + 8 + 8 + 8 + 8) + L * KH * 8
    scatter = info.n_gfac * 8 + M * (8 + 8 + 8) + L * KH * 8
    return dual, scatter


def phase_bytes(info, P, L, K, M):
    """Algorithmic HBM bytes per iteration of every phase of the PDFB
    iteration (the least traffic each phase's result needs):
    primal      29 B per pixel-channel: x, the SARA adjoint, the nuclear dual
                over the facet cover (1.2 on average) and the data adjoint
                (the real C2R output) read, x, xbar and the real zero-padded
                grid written;
    fft_fwd/inv R2C / C2R: the real grid (4 B per cell) and the half
                spectrum (8 B per stored cell) read or written once;
    dual        G factors, row data, y, d read and written, forward grid;
    scatter     G factors, row data, d read, channel grids written;
    sara        the dual W read and written, the weights read (one per
                coefficient row), xbar read and the adjoint term written;
    nuclear     the facet duals P read and written, xbar over the facets read."""
    N = P.ny * P.nx
    KH = 2 * P.ny * (P.nx + 1)                 # half-spectrum cells per channel: K1 x (K2/2 + 1)
    dual, scatter = data_term_bytes(info, L, KH, M)
    fft = L * (4 * K + 8 * KH)
    return {"primal": 29 * N * L, "fft_fwd": fft, "fft_inv": fft, "degrid_grid": dual,
            "scatter": scatter, "sara": (2 * L + P.C) * info.n_coef * 4 + 2 * N * L * 4,
            "nuclear": 3 * info.nuclear_size * 4}


def run_gpu(args):
    import torch
    import paper_2209_07604_gb300 as fhs
    from paper_2209_07604_gb300 import synth

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    # a stream of its own: the legacy default stream cannot be captured, so the iteration would
    # run launch by launch instead of as the replayed CUDA graph of the production path
    torch.cuda.set_stream(torch.cuda.Stream())
    fhs.load_library()
    t0 = time.time()
    P = synth.make_problem(args.workload)
    L, M = P.omega.shape[:2]
    dde = None
    if args.dde:
        # 5x5 DDE kernels per visibility (Sec. 3.1); w halved so that the w-kernels add at most
        # 2 taps per side and every box stays within 16 taps
        P.w *= 0.5
        dde = synth.random_dde(L, M, 7604 + 100 * synth.WORKLOADS[args.workload]["config_id"] + 99)
    gen_s = time.time() - t0
    Mtot = L * M
    stream = torch.cuda.current_stream()

    # ---- end-to-end: host buffers -> problem (H2D inside) -> solve -> image D2H
    torch.cuda.synchronize()
    omega = np.ascontiguousarray(P.omega.reshape(-1, 2))
    wv = np.ascontiguousarray(P.w.reshape(-1))
    yv = np.ascontiguousarray(np.stack([P.y.real, P.y.imag], -1).reshape(-1, 2))
    vis_off = np.arange(L + 1, dtype=np.int64) * M
    gram = {"fp32": fhs.GRAM_FP32, "tf32": fhs.GRAM_TF32, "bf16": fhs.GRAM_BF16, "fp64": fhs.GRAM_FP64}[args.gram]
    params = fhs.default_params(ny=P.ny, nx=P.nx, n_channels=L, n_subcubes=P.C, n_blocks=P.B, qy=P.qy, qx=P.qx,
                                facet_overlap=P.overlap, w_max=P.w_max, pixel_size=P.pixel_size, mu=MU,
                                mu_bar=MU_BAR, gram_precision=gram, data_reduction=int(args.reduction))
    spec = synth.WORKLOADS[args.workload]
    e2e_iters = args.e2e_iters if args.e2e_iters > 0 else max(int(spec["n_iter"]), 2)
    e2e_rw = int(spec["n_reweight"]) if args.e2e_iters <= 0 else (1 if e2e_iters >= 2 else 0)
    img_host = torch.empty((L, P.ny, P.nx), dtype=torch.float32, pin_memory=True)
    t_e2e = time.perf_counter()
    prob = fhs.Problem(params, omega, wv, yv, P.sigma, vis_off, P.block_offsets, dde=dde)
    setup_s = time.perf_counter() - t_e2e
    prob.solve(e2e_iters, 0.0, n_reweight=e2e_rw, check_every=max(1, e2e_iters))
    img_host.copy_(prob.image(), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t_e2e
    if ws > 1:
        e2e_s = max_over_ranks(e2e_s)          # the job ends with its slowest rank
    h2d = omega.nbytes + wv.nbytes + yv.nbytes + P.sigma.nbytes + vis_off.nbytes + P.block_offsets.nbytes
    if dde is not None:
        h2d += dde.nbytes
        del dde
    d2h = img_host.numel() * 4
    info = prob.info

    # ---- device-resident timing of K iterations (problem already on the GPU)
    if args.autotune:
        prob.autotune_bins()
    info = prob.info
    for _ in range(args.warmup):
        prob.step(1)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    launches0 = fhs.fhs_kernel_launches(prob.handle)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        prob.step(args.steps)            # production path: one CUDA graph per iteration
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = fhs.fhs_kernel_launches(prob.handle) - launches0
    # per-phase device time: the same number of iterations right after, with
    # event pairs recorded on this stream around every phase (launched kernel
    # by kernel, since tracing and graph replay exclude each other)
    fhs.fhs_profile_enable(prob.handle, True)
    prob.step(args.steps)
    torch.cuda.synchronize()
    fhs.fhs_profile_enable(prob.handle, False)
    phases, n_prof = fhs.fhs_profile_read(prob.handle)
    if ws > 1:
        ms = max_over_ranks(ms)
        torch.distributed.barrier()
    ms_step = ms / args.steps

    # Phi and Phi^H alone through the C ABI (fhs_measure / fhs_adjoint), device buffers
    xs = torch.rand((L, P.ny, P.nx), device="cuda", dtype=torch.float32)
    vis = torch.empty(Mtot, dtype=torch.complex64, device="cuda")
    img = torch.empty((L, P.ny, P.nx), dtype=torch.float32, device="cuda")
    for _ in range(3):
        fhs.fhs_measure(prob.handle, xs, vis)
        fhs.fhs_adjoint(prob.handle, vis, img)
    n_op = 10
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(n_op):
        fhs.fhs_measure(prob.handle, xs, vis)
    e[1].record(stream)
    for _ in range(n_op):
        fhs.fhs_adjoint(prob.handle, vis, img)
    e[2].record(stream)
    torch.cuda.synchronize()
    phi_ms = e[0].elapsed_time(e[1]) / n_op
    phit_ms = e[1].elapsed_time(e[2]) / n_op
    del xs, vis, img

    # rooflines: every phase of the iteration against its algorithmic bytes; the dominant
    # kernel is the longer of the two passes over G
    K = 4 * P.ny * P.nx
    peak, peak_kind = _peaks()
    pbytes = phase_bytes(info, P, L, K, Mtot)
    if args.reduction:
        # two normal-mode passes per iteration (H Xhat, then H Lambda v): factors, row meta and
        # offsets, the input grid read and the output grid written once each per pass
        pbytes["degrid_grid"] = pbytes["scatter"] = info.n_gfac * 8 + Mtot * 16 + 2 * L * K * 8
    pms = {k: v / max(n_prof, 1) for k, v in phases.items()}
    rl_phases = {}
    for k, b in pbytes.items():
        if pms.get(k, 0.0) > 0:
            a = b / (pms[k] * 1e-3) / 1e9
            rl_phases[k] = {"ms": pms[k], "algorithmic_bytes": int(b), "achieved": a, "frac": a / peak}
    dom = "degrid_grid" if pms["degrid_grid"] >= pms["scatter"] else "scatter"
    prof = _profile_traffic(args.workload, "k_binned.cu")
    if prof is None or args.dde or args.reduction:
        prof = {}
    pkey = "dual" if dom == "degrid_grid" else "scatter"
    achieved = rl_phases[dom]["achieved"]
    # visibilities through Phi and Phi^H per second inside the PDFB iteration
    vis_s = Mtot / (ms_step * 1e-3)
    out = {
        "metric": _metric(args.workload),
        "value": ws * 1e3 / ms_step,
        "unit": "iter/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 (FP64 reductions, eig, weights; facet Gram %s)" % args.gram,
        "data": "synthetic (seeded VLA-like uv/w, Gaussian-blob sky, 40 dB)",
        "config": {"workload": args.workload, "image": "%dx%d" % (P.ny, P.nx), "channels": L,
                   "subcubes": P.C, "vis_per_channel": M, "blocks": P.B, "facets": "%dx%d" % (P.qy, P.qx),
                   "facet_overlap": P.overlap, "w_max": P.w_max, "nnz_G": info.nnz,
                   "l2": "inputs larger than L2 (G factors alone %.1f GB per iteration)" % (info.n_gfac * 8 / 1e9),
                   "mu": MU, "mu_bar": MU_BAR, "gram": args.gram,
                   "bins": {"dense_min": info.bin_dense_min, "split": info.bin_split,
                            "autotuned": bool(args.autotune)},
                   "dde": "5x5 kernel per visibility, w halved" if args.dde else None,
                   "data_reduction": ({"gridded_points": int(info.n_red), "visibilities": int(Mtot)}
                                      if args.reduction else None)},
        "vis_per_s": ws * vis_s,
        "phi_vis_per_s": ws * Mtot / (phi_ms * 1e-3),
        "phi_adjoint_vis_per_s": ws * Mtot / (phit_ms * 1e-3),
        "e2e": {"value": ws * e2e_iters / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": h2d / e2e_iters,
                "d2h_bytes_per_step": d2h / e2e_iters,
                "what": "create from host arrays (sort, G build, Lanczos norm estimate) + %d iterations with %d "
                        "reweighting(s) + image to pinned host" % (e2e_iters, e2e_rw),
                "seconds": e2e_s, "setup_seconds": setup_s},
        "gpu_launches": int(launches),
        "phases_ms_per_step": {k: v / max(n_prof, 1) for k, v in phases.items()},
        "roofline": {"kernel": ("degrid_grid_binned_kernel<kDual>: dual pass over G" if dom == "degrid_grid"
                                else "degrid_grid_binned_kernel<kScatter>: scatter pass over G"),
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": prof.get(pkey), "algorithmic_bytes": int(pbytes[dom]), "peak_source": peak_kind,
                     "limiter": prof.get(pkey + "_limiter")},
        "roofline_phases": rl_phases,
        "clocks": clk.summary(),
        "device_bytes": info.device_bytes,
        "generate_seconds": gen_s,
    }
    if rank == 0 and not args.no_cpu_baseline and ws == 1 and not args.dde and not args.reduction:
        out["cpu_baseline"] = cpu_baseline(args.workload)
    prob.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (cpu_baseline of the GPU arm, and the
# reference arm): a bounded sample of the workload, timed in one process per
# core at the same time, scaled per unit of work to one full iteration.
# ---------------------------------------------------------------------------
ORACLE_SAMPLE = dict(n_vis=20_000, sara_side=384)     # per worker; the same in both arms


def _host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_WORKER_CACHE = {}


def _oracle_worker(args):
    """One worker's share of the sample (a spawned process with one thread):
    the oracle's own operations of one PDFB iteration on a piece of the
    workload, each timed.  Returns per-unit seconds.  The sample's inputs (a
    problem of n_vis visibilities per channel with the workload's geometry and
    its G rows for one channel) are built on a worker's first round only."""
    workload, wid, n_vis, side = args
    from paper_2209_07604_gb300 import synth
    from oracle import nufft as onf, prox as oprox, wavelets as owv
    key = (workload, n_vis)
    if key not in _WORKER_CACHE:
        _WORKER_CACHE.clear()
        # same geometry and distributions as the workload, n_vis visibilities per channel
        _WORKER_CACHE[key] = {"P": synth.make_problem(workload, M=n_vis)}
    cache = _WORKER_CACHE[key]
    P = cache["P"]
    l = wid % P.L
    if l not in cache:
        geom = onf.Geometry(P.ny, P.nx, w_max=P.w_max, n_wplanes=64, pixel_size=P.pixel_size)
        cache[l] = onf.Operator(P.omega[l:l + 1], P.w[l:l + 1], P.sigma[l:l + 1], geom)
    op = cache[l]
    L, Lc = P.L, P.L // P.C
    nnz = op.G[0].nnz
    rng = np.random.default_rng(wid)
    x = rng.uniform(0, 1, (P.ny, P.nx))
    out = {}
    # per channel: Z, F, F^H, Z^H (zero-pad + scaling, two FFTs on the K grid)
    t0 = time.perf_counter()
    g = op.fzx(x)
    op.zf_adj(g)
    out["fft_channel"] = time.perf_counter() - t0
    # per entry of G: Phi's G, the block l2-ball dual steps, G^H
    yw = P.y[l] / P.sigma[l]
    bo = P.block_offsets[l]
    eps = oprox.eps_blocks(n_vis, np.diff(bo))
    t0 = time.perf_counter()
    phix = op.G[0] @ g.ravel()
    v = np.zeros(n_vis, complex)
    for b in range(len(bo) - 1):
        v[bo[b]:bo[b + 1]] = oprox.l2ball_dual(v[bo[b]:bo[b + 1]], phix[bo[b]:bo[b + 1]], yw[bo[b]:bo[b + 1]],
                                               eps[b], 1e-6)
    (op.G[0].conj().T @ v)
    out["g_entry"] = (time.perf_counter() - t0) / nnz
    out["row_nnz"] = nnz / n_vis
    # per pixel-channel: SARA analysis, weighted l21 dual, synthesis (one channel, a side^2 crop)
    sd = min(side, P.ny, P.nx)
    S = owv.Sara(sd, sd)
    xs = x[None, :sd, :sd]
    t0 = time.perf_counter()
    A = S.analysis(xs)
    W = oprox.l21_dual(np.zeros_like(A), A, 1.0, MU, np.ones(A.shape[1]))
    S.synthesis(W)
    out["sara_px"] = (time.perf_counter() - t0) / (sd * sd)
    # per facet-pixel-channel: the nuclear dual step of one facet of a sub-cube
    facets = oprox.nuclear_facets(P.ny, P.nx, P.qy, P.qx, P.overlap)
    y0, y1, x0, x1 = facets[wid % len(facets)]
    Xq = rng.uniform(0, 1, (Lc, y1 - y0, x1 - x0))
    t0 = time.perf_counter()
    oprox.nuclear_dual(np.zeros_like(Xq), Xq, 0.25, MU_BAR, np.ones(Lc))
    out["nuc_px"] = (time.perf_counter() - t0) / Xq.size
    # per pixel-channel: the primal step (projection, extrapolation, relative change)
    Xa, Aa = rng.uniform(0, 1, (3, P.ny, P.nx)), rng.uniform(-1, 1, (3, P.ny, P.nx))
    t0 = time.perf_counter()
    Xp = np.maximum(0.0, Xa - 0.33 * (Aa + Aa + Aa))
    Xb = 2.0 * Xp - Xa
    np.linalg.norm(Xp - Xa), np.linalg.norm(Xp), Xb.sum()
    out["primal_px"] = (time.perf_counter() - t0) / Xa.size
    return out


class OracleTimer:
    """A pool of spawned single-thread processes, one per host core, that
    time the oracle's sample together (rounds of ORACLE_SAMPLE)."""

    def __init__(self, workload: str):
        import multiprocessing as mp
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.workload = workload
        self.n = _host_cores()
        self.pool = mp.get_context("spawn").Pool(self.n)

    def round(self):
        """One round: every worker times its share; returns (per-unit medians, wall seconds)."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, [(self.workload, w, ORACLE_SAMPLE["n_vis"], ORACLE_SAMPLE["sara_side"])
                                             for w in range(self.n)])
        wall = time.perf_counter() - t0
        return {k: float(np.median([r[k] for r in res])) for k in res[0]}, wall

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_seconds_per_iter(workload: str, u: dict, cores: int) -> float:
    """One PDFB iteration of the full workload on `cores` cores from per-unit
    costs measured with every core busy: channels x (zero-pad, FFT, FFT^H,
    crop) + G entries x (G, l2 ball, G^H) + pixel-channels x (SARA + primal) +
    facet-pixel-channels x nuclear dual, divided by the cores (the sub-cubes,
    channels and facets of an iteration are independent pieces of work)."""
    from paper_2209_07604_gb300 import synth
    from oracle import prox as oprox
    spec = synth.WORKLOADS[workload]
    L, M, ny, nx = spec["L"], spec["M"], spec["ny"], spec["nx"]
    fac = oprox.nuclear_facets(ny, nx, spec["qy"], spec["qx"], spec["overlap"])
    nuc_units = sum((y1 - y0) * (x1 - x0) for (y0, y1, x0, x1) in fac) * L
    serial = (L * u["fft_channel"] + u["row_nnz"] * L * M * u["g_entry"]
              + ny * nx * L * (u["sara_px"] + u["primal_px"]) + nuc_units * u["nuc_px"])
    return serial / cores


def oracle_config1_run():
    """The oracle as it stands, one core, on the whole 128^2 x 4-channel
    problem of 2e4 visibilities per channel: 50 PDFB iterations (no
    extrapolation); returns the per-iteration times."""
    from paper_2209_07604_gb300 import synth
    from oracle import pdfb
    P = synth.make_problem("small_128")
    steps = pdfb.Steps(tau=0.99 / 3.0, sigma0=0.25, sigma1=1.0, sigma2=1e-6)
    o = pdfb.FHS(P.omega, P.w, P.y, P.sigma, P.block_offsets, P.ny, P.nx, P.C, P.qy, P.qx, P.overlap,
                 mu=MU, mu_bar=MU_BAR, steps=steps)
    ts = []
    for _ in range(P.n_iter):
        t0 = time.perf_counter()
        o.step()
        ts.append(time.perf_counter() - t0)
    return ts


def _config1_summary(ts):
    return {"workload": "small_128 (128^2, 4 channels, 2e4 visibilities per channel, 2x2 facets)",
            "iterations": len(ts), "wall_s": float(np.sum(ts)),
            "s_per_iter_median3": float(np.median(ts[1:4])), "cores": 1,
            "what": "the whole problem, no extrapolation; median of iterations 2-4 after one warm-up"}


def _sample_text(n):
    return ("per core (%d single-thread processes at once): one channel's zero-pad + FFT + FFT^H + crop on the "
            "full oversampled grid, G, l2-ball duals and G^H of %d visibilities, SARA analysis + l21 dual + "
            "synthesis on a %d^2 crop of one channel, the nuclear dual of one facet of a sub-cube, the primal "
            "step on 3 channels; per-unit costs (channel, G entry, pixel-channel, facet-pixel-channel) scaled to "
            "one full iteration and divided by the cores" % (n, ORACLE_SAMPLE["n_vis"], ORACLE_SAMPLE["sara_side"]))


def cpu_baseline(workload):
    """Oracle iterations/s on the host cores for the workload: one warm-up
    round and one timed round of the sample, plus the real 50-iteration run of
    the 128^2 configuration on one core."""
    tm = OracleTimer(workload)
    try:
        tm.round()
        u, wall = tm.round()
    finally:
        tm.close()
    spi = oracle_seconds_per_iter(workload, u, tm.n)
    c1 = _config1_summary(oracle_config1_run())
    return {"value": 1.0 / spi, "unit": "iter/s", "cores": tm.n, "kind": "oracle", "extrapolated": True,
            "sample": _sample_text(tm.n), "seconds_per_iter": spi, "sample_wall_s": wall, "per_unit_s": u,
            "config1": c1}


def run_reference(args):
    """The oracle as the reference arm (rank 0 only; other ranks exit): each
    step is one round of the same sample as the GPU arm's cpu_baseline."""
    ws, rank, local = _dist()
    if rank != 0:
        return
    tm = OracleTimer(args.workload)
    per, walls, units = [], [], []
    try:
        for i in range(args.warmup + args.steps):
            u, wall = tm.round()
            if i >= args.warmup:
                per.append(oracle_seconds_per_iter(args.workload, u, tm.n))
                walls.append(wall)
                units.append(u)
    finally:
        tm.close()
    s_step = float(np.median(per))
    val = 1.0 / s_step
    c1 = _config1_summary(oracle_config1_run())
    print(json.dumps({
        "impl": "reference", "metric": _metric(args.workload), "value": val, "unit": "iter/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(walls)) * 1e3,
        "seconds_per_iter_estimate": s_step,
        "note": "value = one full iteration of the workload estimated from each step's bounded sample (all host "
                "cores); ms_per_step = the wall time of one sample round, what each step actually ran",
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded VLA-like uv/w, Gaussian-blob sky, 40 dB)",
        "config": {"workload": args.workload},
        "cpu_baseline": {"value": val, "unit": "iter/s", "cores": tm.n, "kind": "oracle", "extrapolated": True,
                         "sample": "each step: " + _sample_text(tm.n), "sample_wall_s_median": float(np.median(walls)),
                         "config1": c1},
        "e2e": {"value": val, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


SERVE_MIXES = {  # (ny, nx, L, C, M per channel, B, facets, w_max)
    # the serving configuration: images 256^2 to 4096^2, 4 to 64 channels (at most 32 per
    # sub-cube), 1e5 to 2e7 visibilities per channel; the largest request holds about 40 GB
    "config5": [
        (256, 256, 4, 1, 100_000, 2, 2, 2000.0),
        (512, 512, 16, 2, 500_000, 4, 2, 2000.0),
        (1024, 1024, 64, 2, 100_000, 4, 4, 2000.0),
        (1024, 1024, 8, 2, 2_000_000, 4, 4, 2000.0),
        (2048, 2048, 16, 2, 2_000_000, 8, 8, 0.0),
        (4096, 4096, 6, 1, 20_000_000, 8, 8, 0.0),
    ],
    # a small mix (images up to 1536 x 1024, up to 8 channels, up to 1e6 visibilities per channel)
    "small": [
        (256, 256, 4, 1, 100_000, 2, 2, 2000.0),
        (512, 512, 8, 2, 200_000, 2, 2, 2000.0),
        (256, 256, 8, 1, 400_000, 4, 2, 0.0),
        (1024, 1024, 4, 1, 300_000, 4, 4, 2000.0),
        (512, 512, 4, 2, 1_000_000, 4, 2, 2000.0),
        (1536, 1024, 4, 1, 200_000, 2, 4, 0.0),
    ],
}


def _serve_pass(reqs, arrivals, max_active, budget, check_every):
    import paper_2209_07604_gb300 as fhs
    sv = fhs.Server(hbm_budget_bytes=budget, max_active=max_active, check_every=check_every)
    t0 = time.perf_counter()
    ids = []
    for (P, kw), ta in zip(reqs, arrivals):
        dt = ta - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(sv.submit_synth(P, **kw))
    res = [sv.wait(i)[1] for i in ids]
    makespan = time.perf_counter() - t0
    sv.close()
    lat = np.array([r.t_done - r.t_submit for r in res])
    vis_iter = sum(P.omega.shape[0] * P.omega.shape[1] * r.iterations for (P, _), r in zip(reqs, res))
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "makespan_s": makespan,
            "images_per_hour": len(res) * 3600.0 / makespan, "vis_per_s": vis_iter / makespan,
            "iterations": [int(r.iterations) for r in res],
            "failed": int(sum(r.state != fhs.REQ_DONE for r in res))}


def run_serve(args):
    """Continuous batching vs one request at a time, same Poisson arrivals."""
    import torch
    import paper_2209_07604_gb300 as fhs
    from paper_2209_07604_gb300 import synth
    torch.cuda.set_device(0)
    fhs.load_library()
    mix = SERVE_MIXES[args.serve_mix]
    pool, sizes = [], []
    for k, (ny, nx, L, C, M, B, Q, wmax) in enumerate(mix):
        P = synth.make_problem("vla_1024", trial=k, ny=ny, nx=nx, L=L, C=C, M=M, B=B, qy=Q, qx=Q, w_max=wmax)
        params = fhs.default_params(ny=ny, nx=nx, n_channels=L, n_subcubes=C, n_blocks=B, qy=Q, qx=Q,
                                    facet_overlap=P.overlap, w_max=P.w_max, pixel_size=P.pixel_size, mu=MU,
                                    mu_bar=MU_BAR)
        sizes.append(fhs.fhs_estimate_bytes(params, P.w.reshape(-1), L * M))
        pool.append(P)
    rng = np.random.default_rng(7604)
    n = args.serve_requests
    reqs = [(pool[rng.integers(len(pool))], dict(mu=MU, mu_bar=MU_BAR, max_iter=args.serve_iters,
                                                   rel_tol=1e-5, n_reweight=1, check_every=10))
            for _ in range(n)]
    arrivals = np.cumsum(rng.exponential(1.0 / args.serve_rate, size=n))
    budget = int(args.serve_budget_gb * (1 << 30))
    batched = _serve_pass(reqs, arrivals, args.serve_active, budget, 10)
    serial = _serve_pass(reqs, arrivals, 1, budget, 10)
    print(json.dumps({
        "mode": "serve", "metric": "imaging requests: p50/p99 time to image, images/hour, visibilities/s",
        "unit": "s", "requests": n, "arrival_rate_per_s": args.serve_rate,
        "mix": [dict(zip(["ny", "nx", "L", "C", "M_per_channel", "B", "facets", "w_max"], m),
                     resident_gb=sz[0] / 1e9, peak_gb=sz[1] / 1e9) for m, sz in zip(mix, sizes)],
        "mix_name": args.serve_mix,
        "iterations_per_request": args.serve_iters, "hbm_budget_gb": args.serve_budget_gb,
        "continuous_batching": batched, "one_at_a_time": serial,
        "speedup_p99": serial["p99_s"] / batched["p99_s"], "speedup_throughput": batched["images_per_hour"] /
        serial["images_per_hour"], "data": "synthetic"}))


def run_batch(args):
    """Batched uneven problems: N seeded problems with image sizes from {256^2, 512^2,
    1024^2, 1536x1024}, L in {4, 8, 16}, M per channel log-uniform on [1e5, 2e6],
    w-terms up to 2000 wavelengths (7-15 taps), facet grids 2x2 to 6x6 with 10-20 %
    overlap.  All problems step together (one stream each, iterations submitted
    round-robin, each a replayed CUDA graph) against the same problems stepped one
    after another; the metric is problem-iterations and visibilities per second."""
    import torch
    import paper_2209_07604_gb300 as fhs
    from paper_2209_07604_gb300 import synth
    torch.cuda.set_device(0)
    fhs.load_library()
    rng = np.random.Generator(np.random.Philox(7604 + 100 * 4))
    sizes = [(256, 256), (512, 512), (1024, 1024), (1536, 1024)]
    specs = []
    for k in range(args.batch_problems):
        ny, nx = sizes[rng.integers(len(sizes))]
        L = int(rng.choice([4, 8, 16]))
        M = int(np.exp(rng.uniform(np.log(1e5), np.log(2e6))))
        q = int(rng.integers(2, 7))
        specs.append(dict(ny=ny, nx=nx, L=L, C=max(1, L // 8), M=M, B=2, qy=q, qx=q,
                          overlap=float(rng.uniform(0.1, 0.2)), w_max=2000.0))
    t0 = time.time()
    probs, streams = [], []
    n_vis = 0
    for k, sp in enumerate(specs):
        P = synth.make_problem("vla_1024", trial=100 + k, **sp)
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            probs.append(fhs.Problem.from_synth(P, mu=MU, mu_bar=MU_BAR, stream=st))
        streams.append(st)
        n_vis += P.L * P.M
        del P
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    handles = [p.handle for p in probs]
    fhs.fhs_pdfb_step_batch(handles, args.warmup, streams)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(0) as clk:
        ev[0].record()
        for st in streams:                      # start after everything queued so far
            torch.cuda.current_stream().wait_stream(st)
        fhs.fhs_pdfb_step_batch(handles, args.steps, streams)
        for st in streams:
            torch.cuda.current_stream().wait_stream(st)
        ev[1].record()
        torch.cuda.synchronize()
    batched_s = ev[0].elapsed_time(ev[1]) * 1e-3
    serial_s = 0.0
    for p, st in zip(probs, streams):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            p.step(args.steps)
            e1.record(st)
        st.synchronize()
        serial_s += e0.elapsed_time(e1) * 1e-3
    dev_bytes = sum(p.info.device_bytes for p in probs)
    for p in probs:
        p.close()
    it = args.batch_problems * args.steps
    print(json.dumps({
        "mode": "batch", "metric": "batched uneven problems: problem-iterations/s and visibilities/s",
        "unit": "problem-iter/s", "problems": args.batch_problems, "steps": args.steps, "warmup": args.warmup,
        "value": it / batched_s, "vis_per_s": n_vis * args.steps / batched_s,
        "one_at_a_time": {"value": it / serial_s, "vis_per_s": n_vis * args.steps / serial_s},
        "speedup": serial_s / batched_s, "visibilities": n_vis, "device_bytes": dev_bytes,
        "setup_seconds": setup_s, "clocks": clk.summary(),
        "config": {"specs": specs}, "data": "synthetic"}))


def run_adaptive(args):
    """Adaptive noise estimation (Sec. 3.3 (ii)) at the workload: the data get extra noise so
    that their effective whitened noise level is 2.5 times the nominal one the bounds assume;
    the phase runs at most args.steps iterations with a check every 10 once the relative change
    is below --adaptive-settle, on a fresh problem (a first problem takes the warm-up phase).  The metric is PDFB iterations/s
    through the phase, checks and their host round trips included; the plain iteration with the
    priors active is timed after it on the same problem."""
    import torch
    import paper_2209_07604_gb300 as fhs
    from paper_2209_07604_gb300 import synth
    torch.cuda.set_device(0)
    torch.cuda.set_stream(torch.cuda.Stream())
    fhs.load_library()
    P = synth.make_problem(args.workload)
    L, M = P.omega.shape[:2]
    s_eff = 2.5
    rng = np.random.Generator(np.random.Philox(7604 + 100 * synth.WORKLOADS[args.workload]["config_id"] + 98))
    n = (rng.standard_normal((L, M)) + 1j * rng.standard_normal((L, M))) * np.sqrt((s_eff ** 2 - 1.0) / 2.0)
    y = P.y + P.sigma[:, None] * n
    del n
    omega = np.ascontiguousarray(P.omega.reshape(-1, 2))
    wv = np.ascontiguousarray(P.w.reshape(-1))
    yv = np.ascontiguousarray(np.stack([y.real, y.imag], -1).reshape(-1, 2))
    del y
    vis_off = np.arange(L + 1, dtype=np.int64) * M
    params = fhs.default_params(ny=P.ny, nx=P.nx, n_channels=L, n_subcubes=P.C, n_blocks=P.B, qy=P.qy, qx=P.qx,
                                facet_overlap=P.overlap, w_max=P.w_max, pixel_size=P.pixel_size, mu=MU,
                                mu_bar=MU_BAR, data_reduction=int(args.reduction))
    check_every = 10
    warm = fhs.Problem(params, omega, wv, yv, P.sigma, vis_off, P.block_offsets)
    warm.adaptive_noise(args.warmup, check_every, args.adaptive_settle)
    warm.close()
    prob = fhs.Problem(params, omega, wv, yv, P.sigma, vis_off, P.block_offsets)
    # the nominal bounds (unit whitened noise, Eq. 2) the phase starts from
    mb = np.diff(P.block_offsets, axis=1).astype(np.float64).ravel()
    eps0 = np.sqrt((M + 2.0 * np.sqrt(M)) * mb / M)
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        ev[0].record(stream)
        sig, eps, res = prob.adaptive_noise(args.steps, check_every, args.adaptive_settle)
        ev[1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ev[2].record(stream)
        prob.step(args.steps)
        ev[3].record(stream)
        torch.cuda.synchronize()
    ms_phase = ev[0].elapsed_time(ev[1])
    ms_plain = ev[2].elapsed_time(ev[3])
    prob.close()
    print(json.dumps({
        "mode": "adaptive", "metric": "PDFB iter/s through the adaptive noise phase (Sec. 3.3 (ii))",
        "unit": "iter/s", "value": res["iterations"] / (ms_phase * 1e-3), "wall_iter_per_s": res["iterations"] / wall,
        "phase": res, "check_every": check_every, "settle_tol": args.adaptive_settle,
        "plain_iteration": {"value": args.steps / (ms_plain * 1e-3), "unit": "iter/s", "priors": "active"},
        "eps_over_nominal_median": None if args.reduction else float(np.median(eps / eps0)),
        "effective_noise_over_nominal": s_eff, "clocks": clk.summary(),
        "config": {"workload": args.workload, "data_reduction": bool(args.reduction)},
        "data": "synthetic (the workload's data plus extra noise to 2.5x the nominal level)"}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="fhs", choices=["fhs", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--e2e-iters", type=int, default=0,
                    help="iterations of the end-to-end run (0: the workload's own, with its reweightings)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="measure candidate tile binnings of the pass over G before timing")
    ap.add_argument("--gram", default="fp32", choices=["fp32", "tf32", "bf16", "fp64"],
                    help="arithmetic of the nuclear facet Gram (tf32/bf16: tensor cores)")
    ap.add_argument("--dde", action="store_true",
                    help="fold seeded 5x5 DDE kernels into G (w halved to keep boxes within 16 taps)")
    ap.add_argument("--reduction", action="store_true",
                    help="visibility-gridding data reduction: Phi' = Lambda H F Z, one l2 ball per channel")
    ap.add_argument("--mode", default="pdfb", choices=["pdfb", "serve", "batch", "adaptive"])
    ap.add_argument("--adaptive-settle", type=float, default=3e-3,
                    help="--mode adaptive: relative change below which a check acts")
    ap.add_argument("--batch-problems", type=int, default=24)
    ap.add_argument("--serve-mix", default="config5", choices=sorted(SERVE_MIXES))
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=4.0)
    ap.add_argument("--serve-iters", type=int, default=200)
    ap.add_argument("--serve-active", type=int, default=8)
    ap.add_argument("--serve-budget-gb", type=float, default=200.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.mode == "serve":
        run_serve(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "adaptive":
        run_adaptive(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
