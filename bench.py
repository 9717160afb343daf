"""Benchmark: ramp-preconditioned PD-TV iterations/sec on the low-dose
workload at scale (512 x 512 image of 20 random ellipses, 720 parallel views
over 180 degrees, 736 bins, transmission Poisson I0 = 5e3 with statistical
weights, beta = 0.005, 30 iterations of Algorithm 1 per solve).

One step = one ct_pdtv_solve call: setup (kappa, tau, taps, Lanczos step
sizes) and 30 iterations, all on the GPU; repeated calls replay the
library's CUDA graph of the solve (--eager: CTPD_SOLVE_GRAPHS=0, every call
launches its kernels).  value = iterations/sec over all ranks (each rank
solves its own slice: independent replicas, weak scaling, no collective on
the data path).  e2e: the same calls with the inputs copied from pinned
host memory and x copied back, every step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--eager]

--impl reference times the FP64 CPU oracle (the reference implementation
of this project) on the same workload and metric, one PD iteration per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORK = dict(name="lowdose_512x512_v720_b736", n=512, views=720, bins=736, ellipses=20,
            i0=5e3, beta=0.005, iters=30, tv_iters=10, norm_iters=12)
METRIC = "PD-TV iterations/sec (512^2, 720 views, 736 bins, low-dose Alg. 1)"
UNIT = "iterations/s"
L2_FLUSH_BYTES = 512 << 20      # > 129 MB L2
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max clock (context)
SMEM_PEAK_TBPS = 152 * 128 * 2.070e9 / 1e12         # SMs x 128 shared-memory bytes per clock x max clock
# DRAM bytes (read + write) per launch of each operator's main kernel at this
# workload, from one ncu capture of the kernel (dram__bytes_read.sum +
# dram__bytes_write.sum); update together with the kernels, None when no
# capture of the current kernel exists.  A: k_project_qbal<4> (the
# work-balanced projector, 12 items' threads per block, 4 steps per pass);
# AT: k_backproject_orbit_cl<true> (mu_bar and x read once).
TRAFFIC_BYTES = {"A": 1.14304e6, "AT": 3.080704e6}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t_ms, device="cpu"):
    """The slowest rank's time (replicas: no collective on the data path,
    one all-reduce of this scalar after the timed region)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_ms)
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(units_per_rank, world, t_ms):
    """Whole-job throughput: units all ranks processed / slowest rank's time."""
    return units_per_rank * world / (t_ms / 1e3)


def phantom(seed):
    return synth.ellipse_phantom(WORK["n"], WORK["ellipses"], seed) * (2.0 / WORK["n"])


# ----------------------------------------------------------------------
# clocks sampled while the timed region runs
# ----------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._th = None

    def _run(self):
        cmd = ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
               "--format=csv,noheader,nounits"]
        while not self._stop.is_set():
            try:
                out = subprocess.run(cmd, capture_output=True, text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._th = threading.Thread(target=self._run, daemon=True)
        self._th.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._th.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 3 + i and s[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ----------------------------------------------------------------------
# algorithmic work of the dominant kernel (backprojection A^T)
# ----------------------------------------------------------------------
def joseph_nnz(n, v_count, b_count):
    """Non-zeros of the Joseph system matrix (count of (ray, pixel) weights
    that are non-zero), from the geometry definition in include/ctpd.h."""
    h, hb = 0.5 * (n - 1), 0.5 * (b_count - 1)
    steps = np.arange(n) - h
    d = np.arange(b_count) - hb
    nnz = 0
    for v in range(v_count):
        t = v * math.pi / v_count
        c, s = math.cos(t), math.sin(t)
        rows = (4 * v <= v_count) or (4 * v >= 3 * v_count)
        a, m = (1 / c, -s / c) if rows else (1 / s, -c / s)
        u = h + d[:, None] * a + steps[None, :] * m
        i0 = np.floor(u)
        f = u - i0
        nnz += int((((i0 >= 0) & (i0 < n)) & (f < 1)).sum() + (((i0 + 1 >= 0) & (i0 + 1 < n)) & (f > 0)).sum())
    return nnz


# ----------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on the host cores
# ----------------------------------------------------------------------
def oracle_inputs(seed=0):
    import oracle as O
    x = phantom(seed)
    b, w = synth.poisson_data(O.project(x, WORK["views"], WORK["bins"]), WORK["i0"], seed + 100)
    kappa = float(np.mean(1.0 / w))
    tau = O.default_tau(0, WORK["views"], kappa)
    taps = O.ramp_taps(0, WORK["views"], WORK["bins"], tau, kappa)
    return b, w, tau, taps


def oracle_iterations(b, w, tau, taps, k, state=None):
    # the oracle as it stands: OpenMP over every core
    import oracle as O
    return O.pdtv(b, w, taps, 0, WORK["beta"], tau, 0.5, WORK["tv_iters"], k, WORK["n"], state=state)[0]


def _oracle_rate(name, iters, threads):
    """iterations/s of the oracle's Algorithm 1 / 2 on a workload of
    synth.CONFIGS (oracle-projected data, sigma 0.5 / 0.9: timing only)."""
    import oracle as O
    cfg = synth.CONFIGS[name]
    N, V, B = cfg["n"], cfg["views"], cfg["bins"]
    x = synth.ellipse_phantom(N, cfg["ellipses"], 0) * cfg["scale"]
    if cfg["mode"] == "lowdose":
        b, w = synth.poisson_data(O.project(x, V, B), cfg["i0"], 100)
        kappa = float(np.mean(1.0 / w))
        mode, sigma = 0, 0.5
    else:
        b, w, kappa, mode, sigma = O.project(x, V, B), None, 0.0, 1, 0.9
    tau = O.default_tau(mode, V, kappa)
    taps = O.ramp_taps(mode, V, B, tau, kappa)
    O.set_threads(threads)
    t0 = time.perf_counter()
    O.pdtv(b, w, taps, mode, cfg["beta"], tau, sigma, 10, iters, N)
    dt = time.perf_counter() - t0
    O.set_threads(0)
    return iters / dt, dt


def cpu_baseline():
    """The FP64 oracle as it stands on this host's cores: the three
    single-slice workloads, a bounded number of iterations each, on one
    thread and on every core (OpenMP over views / image rows; the results
    do not depend on the thread count).  value: the bench workload on every
    core."""
    nproc = os.cpu_count() or 1
    runs = {}
    for name, iters in (("lowdose_64", 20), ("fewview_512", 5), ("lowdose_512", 2)):
        for threads in (1, nproc):
            rate, dt = _oracle_rate(name, iters, threads)
            runs[f"{name}_threads{threads}"] = {"iterations_per_s": rate, "iterations": iters, "seconds": dt}
    value = runs[f"lowdose_512_threads{nproc}"]["iterations_per_s"]
    return {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle",
            "sample": f"2 iterations of Algorithm 1 at 512^2/720 views/736 bins on {nproc} threads "
                      f"(FP64 C oracle, setup excluded); runs: 20 iterations at 64^2/90/95, 5 of the "
                      f"100 at 512^2/32/736, 2 of the 30 at 512^2/720/736, each on 1 and {nproc} threads",
            "runs": runs}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    b, w, tau, taps = oracle_inputs()
    st = None
    for _ in range(args.warmup):
        st = oracle_iterations(b, w, tau, taps, 1, st)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        st = oracle_iterations(b, w, tau, taps, 1, st)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORK["name"], "n": WORK["n"], "views": WORK["views"],
                       "bins": WORK["bins"], "beta": WORK["beta"], "i0": WORK["i0"],
                       "iters_per_step": 1, "l2": "cpu"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                             "sample": "one Algorithm-1 iteration per step, FP64 C oracle, "
                                       "OpenMP over every core, setup excluded"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------
# batched form: 64 slices of mixed size, view count and mode
# ----------------------------------------------------------------------
def _time_graph(P, bs, steps):
    """ms per replay of one CUDA graph of bs.run() (after one eager call)."""
    import torch
    stream = torch.cuda.current_stream()
    bs.run()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        bs.run()
    graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_batched(P, steps=3, count=64, seed=0):
    """slices/s of one ct_pdtv_solve_batched call (captured in a CUDA graph):
    the persistent form (setups on the stream pool, every iteration of every
    slice in one persistent launch) and the stream-pool form, against the
    same slices solved one after another with ct_pdtv_solve."""
    import torch
    shapes = synth.mixed_slices(count, seed)
    slices, geoms = [], {}
    for n, v, nb, mode, sd in shapes:
        g = geoms.setdefault((n, v, nb), P.Geometry(n, v, nb))
        x = synth.ellipse_phantom(n, 10, sd) * ((2.0 / n) if mode == 0 else 1.0)
        p = P.ct_project(g, torch.from_numpy(x.astype(np.float32)).cuda())
        if mode == 0:
            bb, ww = synth.poisson_data(p.cpu().numpy(), 1e4, sd)
            b = torch.from_numpy(bb.astype(np.float32)).cuda()
            w = torch.from_numpy(ww.astype(np.float32)).cuda()
        else:
            b, w = p, None
        slices.append((g, b, w, P.PDTVParams(mode=mode, iters=30, beta=0.005)))
    stream = torch.cuda.current_stream()
    # launch shapes per distinct geometry and the faster form, both tuned before capture
    bs = P.BatchedSolve(slices, autotune=True)
    chosen = bs.form
    t_form = {}
    for form in (P.CT_BATCH_AUTO, P.CT_BATCH_POOL):
        bs.form = form
        t_form[form] = _time_graph(P, bs, steps)
    bs.form = chosen
    t_batched = t_form[chosen]
    t_persistent, t_pool = t_form[P.CT_BATCH_AUTO], t_form[P.CT_BATCH_POOL]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the same slices one after another through the single-slice solve
    ws = bs.ws
    for i, (g, b, w, prm) in enumerate(slices):
        P.ct_pdtv_solve(g, b, w, prm, x_out=bs.x[i], workspace=ws[i], report=False)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for i, (g, b, w, prm) in enumerate(slices):
            P.ct_pdtv_solve(g, b, w, prm, x_out=bs.x[i], workspace=ws[i], report=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / steps
    return {"workload": f"{count} slices, N in (256,384,512), views in (32,90,360,720), "
                        f"bins = ceil(1.44 N), low-dose if V*B > N^2 else few-view, 30 iterations",
            "form": "persistent" if chosen == P.CT_BATCH_AUTO else "stream pool",
            "form_choice": "the faster of the two forms in one untimed trial each (BatchedSolve autotune)",
            "batched_slices_per_s": count / (t_batched / 1e3), "batched_ms": t_batched,
            "persistent_slices_per_s": count / (t_persistent / 1e3), "persistent_ms": t_persistent,
            "pool_slices_per_s": count / (t_pool / 1e3), "pool_ms": t_pool,
            "single_slices_per_s": count / (t_single / 1e3), "single_ms": t_single,
            "speedup": t_single / t_batched}


def measure_unrolled(P, steps=3):
    """Differentiable form: forward + backward of 10 unrolled iterations for a
    batch of 16 slices (256^2, 180 views, 368 bins, I0 = 1e4) with learnable
    log beta and 128 one-sided taps, MSE loss; against the plain solve of one
    such slice (10 iterations, setup included)."""
    import torch
    N, V, B, S = 256, 180, 368, 16
    g = P.Geometry(N, V, B)
    g.autotune(batch=S)   # launch shapes for the batch of the unrolled form (untimed)
    g1 = P.Geometry(N, V, B)
    g1.autotune()         # and for the single-slice solve it is compared with
    xt = torch.from_numpy(np.stack([synth.ellipse_phantom(N, 10, s) * (2.0 / N) for s in range(S)])
                          .astype(np.float32)).cuda()
    p = P.ct_project(g, xt).cpu().numpy()
    bb, ww = synth.poisson_data(p, 1e4, 1)
    b = torch.from_numpy(bb.astype(np.float32)).cuda()
    w = torch.from_numpy(ww.astype(np.float32)).cuda()
    _, rep = P.ct_pdtv_solve(g, b[0], w[0], P.PDTVParams(mode=0, iters=0, beta=0.01))
    taps0 = P.ct_ramp_taps(g, 0, rep["tau"], rep["kappa"])
    m = P.UnrolledReconstructor(g, taps0, 0.01, rep["tau"], 0.9 * rep["sigma"], iters=10, tv_iters=10, half=128)
    stream = torch.cuda.current_stream()

    def step():
        m.zero_grad(set_to_none=True)
        loss = ((m(b, w) - xt) ** 2).mean()
        loss.backward()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_fb = e0.elapsed_time(e1) / steps
    prm = P.PDTVParams(mode=0, iters=10, beta=0.01)
    wsp = P.workspace_for(g1, prm)
    x1 = torch.empty(N, N, device="cuda")
    for _ in range(2):
        P.ct_pdtv_solve(g1, b[0], w[0], prm, x_out=x1, workspace=wsp, report=False)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps * 4):
        P.ct_pdtv_solve(g1, b[0], w[0], prm, x_out=x1, workspace=wsp, report=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_one = e0.elapsed_time(e1) / (steps * 4)
    return {"workload": "16 slices of 256^2, 180 views, 368 bins, I0 1e4, 10 unrolled iterations, "
                        "learnable log beta + 128 taps, MSE loss, forward + backward",
            "fwd_bwd_slices_per_s": S / (t_fb / 1e3), "fwd_bwd_ms": t_fb,
            "plain_solve_slices_per_s": 1.0 / (t_one / 1e3), "plain_solve_ms": t_one,
            "tuning": g.tuning, "plain_solve_tuning": g1.tuning}


CHECKPOINTS = (1, 3, 10, 30, 100, 300, 1000)


def _trajectory(P, g, b, w, mode, precond, beta, v_true, scale, tv_accel=0, eps=0.0, checkpoints=CHECKPOINTS):
    """Iterates of one solve at CHECKPOINTS (resumed solves continue the
    same iteration exactly): RMSE of x / scale against the phantom v_true
    and the relative data residual |A x - b| / |b|."""
    import torch
    prm = P.PDTVParams(mode=mode, iters=checkpoints[0], tv_iters=10, precond=precond, beta=beta,
                       norm_iters=WORK["norm_iters"], tv_accel=tv_accel, eps=eps)
    ws = P.workspace_for(g, prm)
    x = torch.empty(g.n, g.n, device="cuda")
    xs, rmse, resid = {}, {}, {}
    done = 0
    bn = float(torch.linalg.norm(b))
    for k in checkpoints:
        q = P.PDTVParams(**{**prm.__dict__, "iters": k - done, "resume": 1 if done else 0})
        P.ct_pdtv_solve(g, b, w, q, x_out=x, workspace=ws, report=False)
        done = k
        xs[k] = x.clone()
        rmse[k] = float(torch.sqrt(torch.mean((x.double() / scale - v_true) ** 2)))
        resid[k] = float(torch.linalg.norm(P.ct_project(g, x) - b)) / bn
    return xs, rmse, resid


def _solve_rate(P, g, b, w, mode, precond, beta, iters, steps=3, tv_accel=0, eps=0.0):
    """iterations/s of a whole solve (setup included), CUDA events."""
    import torch
    prm = P.PDTVParams(mode=mode, iters=iters, tv_iters=10, precond=precond, beta=beta, norm_iters=WORK["norm_iters"],
                       tv_accel=tv_accel, eps=eps)
    ws = P.workspace_for(g, prm)
    x = torch.empty(g.n, g.n, device="cuda")
    for _ in range(2):
        P.ct_pdtv_solve(g, b, w, prm, x_out=x, workspace=ws, report=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        P.ct_pdtv_solve(g, b, w, prm, x_out=x, workspace=ws, report=False)
    e1.record()
    torch.cuda.synchronize()
    return iters * steps / (e0.elapsed_time(e1) / 1e3)


def measure_fewview_vs_cp(P):
    """The few-view workload (512^2, 32 views, 736 bins, noiseless b = A v,
    100 iterations of Algorithm 2): the ramp preconditioner of Eq. 32 and the
    few-view smoothed ramp against plain Chambolle-Pock (D = I) on the same
    GPU kernels: whole-solve iterations/s and, after 3 / 10 / 30 / 100
    iterations, the RMSE to the phantom and |A x - b| / |b|."""
    import torch
    N, V, B = WORK["n"], 32, WORK["bins"]
    g = P.Geometry(N, V, B)
    g.autotune()
    v_true = synth.ellipse_phantom(N, WORK["ellipses"], 0)
    b = P.ct_project(g, torch.from_numpy(v_true.astype(np.float32)).cuda())
    vt = torch.from_numpy(v_true).cuda()
    cps = (3, 10, 30, 100)
    out = {"workload": f"{N}^2, {V} views, {B} bins, noiseless b = A v, Alg. 2, 100 iterations per solve",
           "checkpoints": list(cps), "tuning": g.tuning}
    for label, pc in (("preconditioned_eq32", 1), ("smoothed_ramp", 3), ("plain_cp", 0)):
        _, rmse, resid = _trajectory(P, g, b, None, 1, pc, 0.0, vt, 1.0, checkpoints=cps)
        out[label] = {"rmse": [rmse[k] for k in cps], "rel_residual": [resid[k] for k in cps],
                      "iterations_per_s": _solve_rate(P, g, b, None, 1, pc, 0.0, 100)}
    return out


def measure_convergence(P):
    """Preconditioners and prox forms on the same GPU kernels: the ramp D of
    Eq. 24 / Eq. 32 with the projected-gradient prox, the same with the FGP
    prox (tv_accel 1), plain Chambolle-Pock (D = I) and, for low-dose, the
    shift-variant split D (precond 2), for few-view the smoothed ramp with
    kappa = tau l (precond 3).  RMSE to the phantom, data residual
    and distance to the 1000-iteration iterate x* of the Eq. 24 run after
    1 .. 1000 iterations, for six workloads: low-dose at the bench size
    (512^2, 720 views, I0 5e3, beta 0.005), the same with the phantom's
    attenuation times 5 (a dense object: counts spread over two decades),
    the same slice with beta 500 (a TV weight that shapes the image),
    few-view (512^2, 32 views, 736 bins, noiseless b = A v, Alg. 2), and the
    paper's shapes (256^2 with 1200 views low-dose at beta 500, and with 32
    views few-view; 369 bins), and the error-tolerant few-view form (Sec. 5)
    on the 512^2 / 32-view slice with Gaussian noise of 1 % of the mean line
    integral and eps = |noise| (x*: the smoothed ramp's 1000-iteration
    iterate); plus whole-solve rates (iterations/s, setup included, 30
    iterations low-dose, 100 few-view)."""
    import torch
    out = {}
    # (name, N, views, bins, mode, beta, attenuation factor); the last two are
    # the paper's own shapes (Sec. 4: 256^2, 1200 views low-dose; 32 views few-view)
    cases = [("lowdose", WORK["n"], WORK["views"], WORK["bins"], 0, WORK["beta"], 1.0),
             ("lowdose_dense", WORK["n"], WORK["views"], WORK["bins"], 0, WORK["beta"], 5.0),
             ("lowdose_tv", WORK["n"], WORK["views"], WORK["bins"], 0, 500.0, 1.0),
             ("fewview", WORK["n"], 32, WORK["bins"], 1, 0.0, 1.0),
             ("paper_lowdose_256_v1200", 256, 1200, 369, 0, 500.0, 1.0),
             ("paper_fewview_256_v32", 256, 32, 369, 1, 0.0, 1.0),
             ("fewview_eps", WORK["n"], 32, WORK["bins"], 1, 0.0, 1.0)]
    for name, N, V, B, mode, beta, dense in cases:
        epsf = name == "fewview_eps"
        g = P.Geometry(N, V, B)
        g.autotune()
        v_true = synth.ellipse_phantom(N, WORK["ellipses"], 0)
        scale = (2.0 / N) * dense if mode == 0 else 1.0
        p = P.ct_project(g, torch.from_numpy((v_true * scale).astype(np.float32)).cuda())
        if mode == 0:
            bb, ww = synth.poisson_data(p.cpu().numpy(), WORK["i0"], 100)
            b = torch.from_numpy(bb.astype(np.float32)).cuda()
            w = torch.from_numpy(ww.astype(np.float32)).cuda()
        else:
            b, w = p, None
        eps = 0.0
        if epsf:
            gen = torch.Generator(device="cpu").manual_seed(7)
            noise = (0.01 * float(p.abs().mean()) * torch.randn(p.shape, generator=gen)).cuda()
            b = p + noise
            eps = float(torch.linalg.norm(noise))
        vt = torch.from_numpy(v_true).cuda()
        if epsf:
            arms = [("preconditioned", 1, 0), ("smoothed_ramp", 3, 0), ("plain_cp", 0, 0)]
        else:
            arms = [("preconditioned", 1, 0), ("preconditioned_fgp", 1, 1), ("plain_cp", 0, 0)]
            arms.insert(2, ("shift_variant", 2, 0) if mode == 0 else ("smoothed_ramp", 3, 0))
        runs = {label: _trajectory(P, g, b, w, mode, pc, beta, vt, scale, acc, eps) for label, pc, acc in arms}
        xstar = runs["smoothed_ramp" if epsf else "preconditioned"][0][CHECKPOINTS[-1]]
        xn = float(torch.linalg.norm(xstar))
        entry = {"workload": f"{N}^2, {V} views, {B} bins, " +
                             (f"Poisson I0 5e3, attenuation x{dense}, beta {beta}, Alg. 1" if mode == 0
                              else "b = A v + Gaussian noise (1 % of the mean line integral), "
                                   "min TV s.t. |Ax - b| <= eps = |noise| (Sec. 5)" if epsf
                              else "noiseless b = A v, Alg. 2"),
                 "checkpoints": list(CHECKPOINTS)}
        if epsf:
            entry["eps_over_norm_b"] = eps / float(torch.linalg.norm(b))
        if mode == 0:
            entry["weight_range"] = [float(w.min()), float(w.max())]
        for label, (xs, rmse, resid) in runs.items():
            entry[label] = {"rmse": [rmse[k] for k in CHECKPOINTS],
                            "rel_residual": [resid[k] for k in CHECKPOINTS],
                            "rel_dist_to_xstar": [float(torch.linalg.norm(xs[k] - xstar)) / xn
                                                  for k in CHECKPOINTS]}
        iters = 100 if mode == 1 else WORK["iters"]
        entry[f"iterations_per_s_{iters}"] = {label: _solve_rate(P, g, b, w, mode, pc, beta, iters, tv_accel=acc,
                                                                 eps=eps)
                                              for label, pc, acc in arms}
        out[name] = entry
    return out


# ----------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------
def run_ours(args):
    import torch
    import __graft_entry__ as entry
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        entry.build()
    if world > 1:
        dist.barrier()
    entry.build()
    import paper_1609_06041_gb300 as P

    N, V, B = WORK["n"], WORK["views"], WORK["bins"]
    g = P.Geometry(N, V, B)
    if args.tuning:
        # fixed launch shapes (for profiler runs, whose timing would mislead the tuner)
        ip, pr, osl, tvr, *pf = (int(t) for t in args.tuning.split(","))
        g.set_tuning(items_per_block=ip, proj_rows=pr, orbit_slices=osl, tv_rows=tvr, proj_form=pf[0] if pf else 0)
        tuning = {**g.tuning, "source": "fixed"}
    else:
        tuning = {**g.autotune(), "source": "autotune"}   # by measurement, once per geometry, untimed
    # synthetic slice for this rank: phantom -> A (on the GPU) -> Poisson data
    xt = torch.from_numpy(phantom(rank).astype(np.float32)).cuda()
    p = P.ct_project(g, xt).cpu().numpy()
    b_np, w_np = synth.poisson_data(p, WORK["i0"], rank + 100)
    b = torch.from_numpy(b_np.astype(np.float32)).cuda()
    w = torch.from_numpy(w_np.astype(np.float32)).cuda()
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=WORK["iters"], tv_iters=WORK["tv_iters"],
                       precond=1, norm_iters=WORK["norm_iters"], beta=WORK["beta"])
    ws = P.workspace_for(g, prm)
    x = torch.empty(N, N, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, device="cuda")
    stream = torch.cuda.current_stream()

    def solve():
        P.ct_pdtv_solve(g, b, w, prm, x_out=x, workspace=ws, report=False)

    for _ in range(max(args.warmup, 3)):
        solve()
    torch.cuda.synchronize()
    # repeated calls replay the library's CUDA graph of this solve (captured
    # by the first call after the warm-up ones above); its kernels count as
    # launched on every replay
    step = solve

    def timed_steps(fn, k):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        torch.cuda.synchronize()
        for i in range(k):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            fn()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(c) for a, c in ev)

    # ---- timed region: K solves, L2 flushed between them (untimed) ----
    launches0 = P.ct_kernel_launches()
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        t_local = timed_steps(step, args.steps)
    launches = P.ct_kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    t_ms = max_over_ranks(t_local, device="cuda")
    value = job_value(WORK["iters"] * args.steps, world, t_ms)

    # ---- breakdown: setup vs iterations (resume runs iterations only) ----
    _, rep = P.ct_pdtv_solve(g, b, w, prm, x_out=x, workspace=ws, report=True)
    prm_r = P.PDTVParams(**{**prm.__dict__, "resume": 1})
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    flush.fill_(1.0)
    e0.record(stream)
    for _ in range(reps):
        P.ct_pdtv_solve(g, b, w, prm_r, x_out=x, workspace=ws, report=False)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / reps
    step_ms = t_ms / args.steps

    # ---- dominant kernel: A^T on this workload, CUDA events, same stream ----
    mub = torch.randn(V, B, device="cuda")
    img = torch.empty(N, N, device="cuda")
    for _ in range(3):
        P.ct_backproject(g, mub, img)
    nrep = 50
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(nrep):
        P.ct_backproject(g, mub, img)
    k1.record(stream)
    torch.cuda.synchronize()
    at_ms = k0.elapsed_time(k1) / nrep
    # A: the projector kernel alone (its band partial sums, the form the
    # solve's Step 3 takes), and ct_project with the reduction for context
    parts = torch.empty(P.ct_project_bands_count(g), V, B, device="cuda")
    for _ in range(3):
        P.ct_project_bands(g, img, parts)
    fw0, fw1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fw0.record(stream)
    for _ in range(nrep):
        P.ct_project_bands(g, img, parts)
    fw1.record(stream)
    torch.cuda.synchronize()
    a_ms = fw0.elapsed_time(fw1) / nrep
    fw0.record(stream)
    for _ in range(nrep):
        P.ct_project(g, img, mub)
    fw1.record(stream)
    torch.cuda.synchronize()
    a_red_ms = fw0.elapsed_time(fw1) / nrep
    nnz = joseph_nnz(N, V, B)
    flops = 2.0 * nnz
    # measured FP32 FMA peak (scalar and packed f32x2 FMA chains), clocks sampled
    with ClockSampler(local) as peak_clock:
        fma_scalar = P.ct_probe_fp32_fma(False)
        fma_packed = P.ct_probe_fp32_fma(True)
    fp32_peak = max(fma_scalar, fma_packed)
    # dominant operator: the slower of A (ct_project_bands: the projector
    # kernel) and A^T (ct_backproject: the orbit kernel, its slices added in
    # a thread-block cluster); both carry 2 nnz(A) algorithmic flops
    a_kernel = "k_project_qbal" if g.tuning.get("proj_form") == 2 else "k_project_quad"
    at_kernel = "k_backproject_orbit_cl" if g.tuning.get("orbit_slices", 0) != 1 else "k_backproject_orbit"
    dom_name, dom_ms, dom_key = (f"ct_backproject (A^T, {at_kernel})", at_ms, "AT") \
        if at_ms >= a_ms else (f"ct_project_bands (A, {a_kernel})", a_ms, "A")
    achieved = flops / (dom_ms / 1e3) / 1e12

    # ---- end to end through the public API with host buffers ----
    b_h = torch.from_numpy(b_np.astype(np.float32)).pin_memory()
    w_h = torch.from_numpy(w_np.astype(np.float32)).pin_memory()
    x_h = torch.empty(N, N).pin_memory()

    def e2e_step():
        # host buffers straight into the C-ABI call: the library copies b and
        # w in and x out through its workspace, inside its solve graph
        P.ct_pdtv_solve(g, b_h, w_h, prm, x_out=x_h, workspace=ws, report=False)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ee[i][0].record(stream)
        e2e_step()
        ee[i][1].record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(c) for a, c in ee), device="cuda")
    e2e_value = job_value(WORK["iters"] * args.steps, world, e2e_ms)

    forms = None
    if not args.no_forms and world == 1:
        forms = {"batched": measure_batched(P), "differentiable": measure_unrolled(P),
                 "fewview_vs_plain_cp": measure_fewview_vs_cp(P)}

    clocks = sampler.summary()
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": step_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORK["name"], "n": N, "views": V, "bins": B,
                       "beta": WORK["beta"], "i0": WORK["i0"], "iters_per_step": WORK["iters"],
                       "tv_iters": WORK["tv_iters"], "norm_iters": WORK["norm_iters"],
                       "l2": "flushed between steps (512 MB write, untimed)",
                       "launch": ("ct_pdtv_solve calls, each replaying the library's CUDA graph of the solve"
                                  if not args.eager else "ct_pdtv_solve calls launching their kernels (no graph)"),
                       "parallelism": f"replicas x{world}", "tuning": tuning},
            # iterations_only_eager: resumed solves, which read their iteration
            # count back to the host and so launch their kernels one by one
            "breakdown_ms": {"solve": step_ms, "iterations_only_eager": loop_ms,
                             "per_iteration_eager": loop_ms / WORK["iters"],
                             "A_launch": a_ms, "A_with_reduction": a_red_ms, "AT_launch": at_ms},
            "loop_iterations_per_s": WORK["iters"] / (loop_ms / 1e3) * world,
            # effective operator bandwidth: (4 N^2 + 4 V B) bytes per pass
            "operator_GBps": {"A": (4.0 * N * N + 4.0 * V * B) / (a_ms / 1e3) / 1e9,
                              "AT": (4.0 * N * N + 4.0 * V * B) / (at_ms / 1e3) / 1e9},
            "report": {k: rep[k] for k in ("tau", "sigma", "kappa", "norm_ADA", "norm_WDW")},
            "roofline": {"kernel": dom_name, "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s", "frac": achieved / fp32_peak,
                         "traffic": TRAFFIC_BYTES.get(dom_key), "traffic_unit": "bytes/launch",
                         "algorithmic_flops": flops, "nnz": nnz, "launch_ms": dom_ms,
                         "peak_source": "measured: ct_probe_fp32_fma, the faster of scalar and packed "
                                        "(f32x2) FMA chains, CUDA events, same process",
                         "peak_probe": {"scalar_tflops": fma_scalar, "packed_f32x2_tflops": fma_packed,
                                        "clocks": peak_clock.summary(),
                                        "nominal_tflops": FP32_NOMINAL_TFLOPS}},
            # the projector's binding resource: every Joseph sample reads one
            # interpolation pair (8 bytes) from shared memory; samples = nnz / 2
            "roofline_shared_memory": {"kernel": f"ct_project_bands (A, {a_kernel})", "achieved": 8.0 * (nnz / 2) / (a_ms / 1e3) / 1e12,
                                       "peak": SMEM_PEAK_TBPS, "unit": "TB/s",
                                       "frac": 8.0 * (nnz / 2) / (a_ms / 1e3) / 1e12 / SMEM_PEAK_TBPS,
                                       "peak_source": "152 SMs x 128 B/clock x 2070 MHz"},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": 2 * V * B * 4, "d2h_bytes_per_step": N * N * 4},
            "gpu_launches": launches,
            "clocks": clocks,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_ncu_case(args):
    """A short, fixed launch sequence for ncu captures: build the workload's
    data, then one solve with 2 power iterations and 3 iterations."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    import paper_1609_06041_gb300 as P
    N, V, B = WORK["n"], WORK["views"], WORK["bins"]
    g = P.Geometry(N, V, B)
    if args.tuning:
        # fixed launch shapes (items_per_block, proj_rows, orbit_slices, tv_rows),
        # so the captured launches are not the tuner's trial launches
        ip, pr, osl, tvr, *pf = (int(t) for t in args.tuning.split(","))
        g.set_tuning(items_per_block=ip, proj_rows=pr, orbit_slices=osl, tv_rows=tvr, proj_form=pf[0] if pf else 0)
    else:
        g.autotune()
    xt = torch.from_numpy(phantom(0).astype(np.float32)).cuda()
    p = P.ct_project(g, xt).cpu().numpy()
    b_np, w_np = synth.poisson_data(p, WORK["i0"], 100)
    b = torch.from_numpy(b_np.astype(np.float32)).cuda()
    w = torch.from_numpy(w_np.astype(np.float32)).cuda()
    prm = P.PDTVParams(mode=P.CT_LOWDOSE, iters=3, tv_iters=WORK["tv_iters"], precond=1,
                       norm_iters=2, beta=WORK["beta"])
    torch.cuda.synchronize()
    # the solve alone between profiler start and stop, so that a capture with
    # --profile-from-start off sees none of the tuner's trial launches
    torch.cuda.profiler.start()
    x, rep = P.ct_pdtv_solve(g, b, w, prm)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"ncu_case": "solve", "report": rep}))
    return 0


def run_ncu_batched(args):
    """A short fixed sequence for ncu captures of the persistent batched
    launch: 8 slices (256^2 and 384^2, 32 and 90 views, both modes), 5
    iterations each, one ct_pdtv_solve_batched call in the persistent form."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    import paper_1609_06041_gb300 as P
    slices = []
    for i, (n, v) in enumerate([(256, 32), (256, 90), (384, 32), (384, 90)] * 2):
        g = P.Geometry(n, v, synth.bins_for(n))
        x = synth.ellipse_phantom(n, 10, i)
        mode = i % 2
        p = P.ct_project(g, torch.from_numpy((x * ((2.0 / n) if mode == 0 else 1.0)).astype(np.float32)).cuda())
        if mode == 0:
            bb, ww = synth.poisson_data(p.cpu().numpy(), 1e4, i)
            b = torch.from_numpy(bb.astype(np.float32)).cuda()
            w = torch.from_numpy(ww.astype(np.float32)).cuda()
        else:
            b, w = p, None
        slices.append((g, b, w, P.PDTVParams(mode=mode, iters=5, beta=0.005)))
    P.ct_batched_options(P.CT_BATCH_AUTO)
    xs, reps = P.ct_pdtv_solve_batched(slices)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": "batched", "slices": len(slices), "k": [r["k"] for r in reps]}))
    return 0


def measure_eps(P, steps=5):
    """The error-tolerant few-view form (Sec. 5) against the equality form on
    the few-view slice (512^2, 32 views, 736 bins, the few-view smoothed
    ramp, 100 iterations per solve): Gaussian noise of 1 % of the mean line
    integral, eps = |noise|; whole-solve iterations/s (setup included) and
    the final relative residual over eps."""
    import torch
    N, V, B = WORK["n"], 32, WORK["bins"]
    g = P.Geometry(N, V, B)
    g.autotune()   # launch shapes for this geometry (untimed)
    p = P.ct_project(g, torch.from_numpy(synth.ellipse_phantom(N, WORK["ellipses"], 0).astype(np.float32)).cuda())
    gen = torch.Generator(device="cpu").manual_seed(7)
    noise = (0.01 * float(p.abs().mean()) * torch.randn(p.shape, generator=gen)).cuda()
    b = p + noise
    eps = float(torch.linalg.norm(noise))
    out = {"workload": f"{N}^2, {V} views, {B} bins, b = A v + 1 % Gaussian noise, eps = |noise|, "
                       "few-view smoothed ramp, 100 iterations", "tuning": g.tuning}
    for name, e in (("equality", 0.0), ("eps", eps)):
        prm = P.PDTVParams(mode=P.CT_FEWVIEW, iters=100, precond=3, eps=e)
        ws = P.workspace_for(g, prm)
        x = torch.empty(N, N, device="cuda")
        for _ in range(2):
            P.ct_pdtv_solve(g, b, None, prm, x_out=x, workspace=ws, report=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            P.ct_pdtv_solve(g, b, None, prm, x_out=x, workspace=ws, report=False)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"iterations_per_s": 100 * steps / (e0.elapsed_time(e1) / 1e3),
                     "residual_over_eps": float(torch.linalg.norm(P.ct_project(g, x) - b)) / eps}
    return out


def run_form(args):
    """One of the forms' measurements alone, as one JSON line."""
    import __graft_entry__ as entry
    entry.build()
    import paper_1609_06041_gb300 as P
    fn = {"batched": measure_batched, "differentiable": measure_unrolled, "fewview_cp": measure_fewview_vs_cp,
          "convergence": measure_convergence, "eps": measure_eps}[args.form]
    print(json.dumps({"form": args.form, **fn(P)}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched, differentiable and convergence measurements")
    ap.add_argument("--ncu-case", nargs="?", const="solve", default="", choices=["solve", "batched"],
                    help="run a short fixed launch sequence for ncu captures: one solve of the bench workload "
                         "(solve) or one persistent batched call of 8 small slices (batched)")
    ap.add_argument("--eager", action="store_true",
                    help="time eager ct_pdtv_solve calls instead of replaying one captured CUDA graph of the solve")
    ap.add_argument("--tuning", default="",
                    help="fixed launch shapes 'items,rows,orbit_slices,tv_rows[,proj_form]' instead of the autotuner")
    ap.add_argument("--form", default="", choices=["", "batched", "differentiable", "fewview_cp", "convergence", "eps"],
                    help="run only this form's measurement")
    args = ap.parse_args()
    if args.eager:
        os.environ["CTPD_SOLVE_GRAPHS"] = "0"   # read when the library first solves
    if args.form:
        return run_form(args)
    if args.ncu_case == "batched":
        return run_ncu_batched(args)
    if args.ncu_case:
        return run_ncu_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
