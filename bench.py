#!/usr/bin/env python3
"""Benchmark of the Duplex-GS hot path on GB300.

Workload: the multi-scale scene (100,000 cells x 10 Gaussians = 1M, SH
degree 3, cell axes log-uniform [0.001, 1] in [-10,10]^3, seed 0) rendered
from 8 seeded cameras on a sphere of radius 15 at 1920x1080.  One step = the
whole hot path over that batch: binning (cull, depth sort over cells, scan,
emit, tile sort, ranges), Gaussian projection, hybrid blend, L1 loss to
seeded target images, blend adjoint and projection adjoint.
Metric: Mpix/s fwd+bwd = views * W * H / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-serve]

Under torchrun (N > 1) every rank renders its own 8 views (independent
units, no collective on the data path): weak scaling, max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_IMG, H_IMG, N_VIEWS = 1920, 1080, 8
METRIC = "Mpix/s fwd+bwd at 1M Gaussians 1080p"
UNIT = "Mpix/s"
WORKLOAD = "multiscale-1M-gaussians (100k cells x 10, SH3) 8 views 1920x1080 fwd+bwd L1"
# FP32 operations of one (pixel, Gaussian) pair that passes the AABB test,
# counted from the kernels: forward 23 (offset 2, quadratic form 8, exp2 1,
# opacity and clamp 2, colour 6, alpha sum 1, transmittance 3); backward
# adds 37 (alpha adjoint 8, colour 7, v_n 3, opacity 2, quadratic 3,
# mean 8, conic 6) to the 23 of the replay.
FLOP_FWD = 23
FLOP_BWD = 60


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def measured_traffic(kernel, views):
    """DRAM bytes per launch from the committed ncu record, if the kernel
    source is unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_blend_bwd.json")
    if kernel != "blend_bwd" or not os.path.exists(path):
        return None
    rec = json.load(open(path))
    src = os.path.join(ROOT, rec["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != rec["sha256"]:
        return None
    return rec["bytes_per_launch"] * views / rec["views_in_capture"]


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x clock
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [r[0] for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def dist_setup(args, backend=None):
    """One process per GPU under torchrun (RANK / LOCAL_RANK / WORLD_SIZE /
    MASTER_* from the environment): NCCL on GPUs, gloo otherwise."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def flat_grads(G, C, device):
    """The explicit Gaussians' gradients (mean, log-scale, quaternion, logit,
    SH: 59 floats per Gaussian at SH degree 3) as views of one flat buffer,
    so a data-parallel step sums them across ranks with one all-reduce."""
    import torch
    shapes = dict(g_mean=(G, 3), g_log_scale=(G, 3), g_quat=(G, 4), g_logit=(G,), g_sh=(G, C, 3))
    flat = torch.empty(sum(int(np.prod(v)) for v in shapes.values()), dtype=torch.float32, device=device)
    out, o = {}, 0
    for k, shp in shapes.items():
        n = int(np.prod(shp))
        out[k] = flat[o:o + n].view(shp)
        o += n
    return flat, out


def reduce_grads(flat, world):
    """Data-parallel fwd+bwd over views: every rank renders its own views of
    the same scene, so the per-Gaussian gradients are summed across ranks
    (the step's one exchange).  Nothing to do on one rank."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)


def weak_value(ms_total, world, px_per_rank_step, steps):
    """Whole-job Mpix/s: every rank renders its own views (weak scaling), so
    the job processed world x px x steps pixels in the slowest rank's time."""
    return world * px_per_rank_step * steps / (ms_total / 1e3) / 1e6


def cameras_for(rank, n_views=N_VIEWS):
    from paper_2508_03180_gb300 import synth
    return synth.sphere_cameras(n_views, 15.0, W_IMG, H_IMG, seed0=N_VIEWS * rank)


def cpu_sample(scene, cam, rows, threads_note=True):
    """Oracle fwd+bwd on tile rows [0, rows) of one view; returns (pixels, seconds)."""
    import oracle
    H, W = int(cam[1]), int(cam[0])
    rng = np.random.default_rng(7)
    dl = rng.standard_normal((3, H, W)) / (3 * H * W)
    t0 = time.perf_counter()
    oracle.render_and_grad(scene, cam, dl, tile_rows=(0, rows))
    dt = time.perf_counter() - t0
    return rows * 16 * W, dt


def run_reference(args):
    """The oracle (CPU, FP64) on the machine's host cores, same metric."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2508_03180_gb300 import synth
    oracle.build()
    scene = synth.scene_multiscale()
    cams = [c.as_array() for c in cameras_for(0)]
    budget_s = 150.0 / max(1, args.steps + args.warmup)
    # calibrate the band height on one tile row
    _, t1 = cpu_sample(scene, cams[0], 1)
    rows = int(max(1, min(68, budget_s / max(t1, 1e-3))))
    px_tot, t_tot = 0, 0.0
    for i in range(args.warmup + args.steps):
        px, dt = cpu_sample(scene, cams[i % N_VIEWS], rows)
        if i >= args.warmup:
            px_tot += px
            t_tot += dt
    v = px_tot / t_tot / 1e6
    sample = f"oracle fwd+bwd (FP64) on tile rows 0..{rows - 1} ({rows * 16} px rows) of one 1920x1080 view per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVE_RATES = (200.0, 500.0, 1000.0, 1500.0, 2000.0, 2250.0, 2500.0, 2750.0, 3000.0, 3500.0, 4000.0, 4500.0,
               5000.0, 6000.0)
SERVE_SLO_MS = (2.0, 3.0, 5.0, 20.0)


def at_p99(rows, slos=SERVE_SLO_MS):
    """For each p99 target: the highest offered rate whose p99 latency stays
    within it, with the frames/s and p99 measured there (None if no rate
    does)."""
    out = {}
    for slo in slos:
        ok = [r for r in rows if r["p99_ms"] <= slo]
        best = max(ok, key=lambda r: r["offered_rps"]) if ok else None
        out[f"{slo:g}ms"] = None if best is None else {"offered_rps": best["offered_rps"], "fps": best["fps"],
                                                       "p99_ms": best["p99_ms"]}
    return out


def serving_bench(rctx, rates=SERVE_RATES, n_req=400, seed=0):
    """Open-loop Poisson arrivals over 3 resident scenes (100k, 500k, 2M
    Gaussians), resolutions uniform over {640x480, 1280x720, 1920x1080,
    3840x2160}.  The same request trace is served by continuous batching
    (up to 8 views per launch chain, 2 chains in flight) and one request at a
    time, at each offered rate; 200 req/s is the configured load, the higher
    rates locate each system's saturation.  `at_p99` compares the modes at
    equal p99 latency: per p99 target, the highest rate each sustains within
    it and the frames/s there."""
    import torch

    from paper_2508_03180_gb300 import synth
    scenes = [synth.scene_small(seed=s, n_cells=n) for s, n in ((1, 12_500), (2, 62_500), (3, 250_000))]
    sids = [rctx.upload_scene(s) for s in scenes]
    res_opts = [(640, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_req):
        s = int(rng.integers(0, 3))
        W, H = res_opts[int(rng.integers(0, 4))]
        cam = synth.sphere_cameras(1, 3.0, W, H, seed0=10_000 + i)[0]
        reqs.append((sids[s], cam, W, H))
    gaps = rng.exponential(1.0, n_req)
    outs = [torch.empty(3 * H * W, device="cuda") for (_, _, W, H) in reqs]

    def run(max_batch, rate, graphs=True):
        arrivals = np.cumsum(gaps / rate)
        rctx.serve_start(max_batch=max_batch, queue_cap=8192, graphs=graphs)
        # warm-up: the whole trace as one burst, so buffers reach their
        # capacities and the graphs of the scene sets exist before timing
        for t in [rctx.submit(sid, cam, outs[i]) for i, (sid, cam, W, H) in enumerate(reqs)]:
            rctx.poll(t, -1)
        st0 = rctx.serve_stats()
        t0 = time.perf_counter()
        tickets = []
        for i, (sid, cam, W, H) in enumerate(reqs):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(rctx.submit(sid, cam, outs[i]))
        lat, bs = [], []
        for t in tickets:
            r = rctx.poll(t, -1)
            lat.append(r.t_done_ms - r.t_submit_ms)
            bs.append(r.batch_size)
        t_end = time.perf_counter()
        st1 = rctx.serve_stats()
        rctx.serve_stop()
        return {"offered_rps": rate, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "fps": n_req / (t_end - t0),
                "mean_batch": float(np.mean(bs)), "batches": st1["batches"] - st0["batches"],
                "graph_captures": st1["graphs_captured"] - st0["graphs_captured"],
                "overflow_reruns": st1["overflow_retries"] - st0["overflow_retries"]}

    out = {"workload": "3 resident scenes (100k, 500k, 2M Gaussians), Poisson arrivals, 640x480..3840x2160",
           "requests_per_rate": n_req,
           "modes": {"batched": "up to 8 views per chain, each batch one CUDA-graph replay",
                     "batched_no_graph": "up to 8 views per chain, plain launches, sort length read back midway",
                     "one_at_a_time": "one view per chain, CUDA-graph replay"},
           "batched": [], "batched_no_graph": [], "one_at_a_time": []}
    for rate in rates:
        out["batched"].append(run(8, rate))
        out["batched_no_graph"].append(run(8, rate, graphs=False))
        out["one_at_a_time"].append(run(1, rate))
    out["at_p99"] = {m: at_p99(out[m]) for m in ("batched", "batched_no_graph", "one_at_a_time")}
    for s in sids:
        rctx.release_scene(s)
    return out


def _timed(fn, reps=3):
    """Median device time (ms) of fn() -> dgs_stats with timing, after one warm-up."""
    fn()
    return float(np.median([fn().ms_total for _ in range(reps)]))


def comparators_bench(rctx, n_views=8):
    """The large-scale workload (1M cells x 10 Gaussians on a ground plane,
    SH 3) from 8 street-level cameras, forward only, rendered three ways in
    the same library: Duplex-GS (cells sorted), per-Gaussian global-sort
    alpha-blending, and sort-free weighted sums (plain WSR, tau = inf).  The
    analogue of the paper's sort-length table: entries sorted by depth and
    (tile, primitive) pairs sorted by tile, with device times."""
    from paper_2508_03180_gb300 import _lib as L
    from paper_2508_03180_gb300 import synth
    scene = synth.scene_large()
    sid = rctx.upload_scene(scene)
    out = {"workload": "large-scale 1M cells x 10 Gaussians (10M), SH3, 8 street-level cameras, forward",
           "resolutions": {}}
    try:
        for (W, H) in ((1920, 1080), (3840, 2160)):
            cams = synth.street_cameras(n_views, W, H, seed0=0)
            slots = rctx.set_cameras(cams)
            img = torch_empty(n_views * 3 * W * H)
            px = n_views * W * H

            def duplex():
                st = L.dgs_stats()
                st.timing = 1
                L.dgs_render(rctx.ctx, sid, slots, img.data_ptr(), L.DGS_DEVICE, False, 0, st)
                return st

            def comp(mode):
                def f():
                    cfg = L.dgs_compare_config()
                    cfg.mode = mode
                    st = L.dgs_stats()
                    st.timing = 1
                    L.dgs_render_compare(rctx.ctx, sid, slots, cfg, img.data_ptr(), 0, 0, st)
                    return st
                return f

            res = {}
            for name, fn, depth_entries in (("duplex", duplex, n_views * scene.N),
                                            ("alpha_blend", comp(L.DGS_COMPARE_ALPHA), n_views * scene.G),
                                            ("wsr", comp(L.DGS_COMPARE_WSR), 0)):
                ms = _timed(fn)
                st = fn()
                res[name] = {"ms": ms, "mpix_s": px / (ms / 1e3) / 1e6, "depth_sort_entries": depth_entries,
                             "tile_sort_pairs": int(st.sort_length), "kept_entries": int(st.visible_cells)}
            for name in ("alpha_blend", "wsr"):
                res[name]["time_vs_duplex"] = res[name]["ms"] / res["duplex"]["ms"]
                res[name]["pairs_vs_duplex"] = res[name]["tile_sort_pairs"] / max(1, res["duplex"]["tile_sort_pairs"])
            out["resolutions"][f"{W}x{H}"] = res
    finally:
        rctx.release_scene(sid)
    return out


def small_fwdbwd_bench(rctx, steps=10):
    """The small scene (2,048 cells x 8 Gaussians, SH 3 from the RGB draws)
    at 1920x1080, a batch of 4 views, L1 loss, forward + backward."""
    import torch

    from paper_2508_03180_gb300 import synth
    scene = synth.scene_small(seed=0, sh_degree=3)
    sid = rctx.upload_scene(scene)
    try:
        cams = synth.sphere_cameras(4, 3.0, 1920, 1080, seed0=0)
        slots = rctx.set_cameras(cams)
        n = 4 * 3 * 1080 * 1920
        img, dl = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        loss = torch.empty(1, device="cuda")
        target = torch.from_numpy(synth.target_image(4, 1080, 1920, seed=7)).cuda().reshape(-1)
        G = scene.G
        grads = dict(g_mean=torch.empty(G, 3, device="cuda"), g_log_scale=torch.empty(G, 3, device="cuda"),
                     g_quat=torch.empty(G, 4, device="cuda"), g_logit=torch.empty(G, device="cuda"),
                     g_sh=torch.empty(G, 16, 3, device="cuda"))

        def step():
            _, state, _ = rctx.render(sid, cams, want_state=True, out=img, slots=slots)
            rctx.loss_l1(img, target, dl, loss)
            rctx.backward(state, dl, grads)
            rctx.release_state(state)

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        return {"workload": "small 2,048 cells x 8 Gaussians (16k), SH3, 4 views 1920x1080 fwd+bwd L1",
                "ms_per_step": ms, "mpix_s": 4 * 1920 * 1080 / (ms / 1e3) / 1e6}
    finally:
        rctx.release_scene(sid)


def neural_fwdbwd_bench(rctx, fp32_tflops, steps=5, F=32, H=32, K=10):
    """Neural cells (Sec. III-IV: four one-hidden-layer decoders per cell,
    random weights) on the multi-scale layout (100,000 cells x 10 Gaussians
    in [-10,10]^3, semi-axes over [0.001, 1]), the headline's 8 views at
    1920x1080, L1 loss, forward + backward to the weights, features and
    offsets.  The decode's products run on the tensor cores at these widths
    and its adjoint's on the CUDA cores; both are reported against the
    measured FP32 FMA rate for comparison, their FLOPs per decoded (view,
    cell) counted from the kernels' loops.  Timed steps render without stats
    (asynchronously); one untimed render reads the counts."""
    import torch

    from paper_2508_03180_gb300 import _lib as L
    from paper_2508_03180_gb300 import synth
    scene = synth.neural_scene(n_cells=100_000, K=K, F=F, H=H, seed=0, box=10.0, axes_lo=0.001, axes_hi=1.0)
    sid = rctx.upload_scene(scene)
    try:
        cams = cameras_for(0)
        slots = rctx.set_cameras(cams)
        n = len(cams) * 3 * H_IMG * W_IMG
        img, dl = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        loss = torch.empty(1, device="cuda")
        target = torch.from_numpy(synth.target_image(len(cams), H_IMG, W_IMG, seed=7)).cuda().reshape(-1)
        P = sum(H * (F + 4) + H + o * H + o for o in (K, 3 * K, 3 * K, 4 * K))  # packed decoder weights
        grads = dict(g_mlp=torch.empty(P, device="cuda"), g_feat=torch.empty(scene.N, F, device="cuda"),
                     g_offset=torch.empty(scene.G, 3, device="cuda"))

        def step():  # asynchronous: the decode's sample count stays on the device
            _, state, _ = rctx.render(sid, cams, want_state=True, out=img, slots=slots)
            rctx.loss_l1(img, target, dl, loss)
            rctx.backward(state, dl, grads)
            rctx.release_state(state)

        for _ in range(3):
            step()
        _, st0, st = rctx.render(sid, cams, want_state=True, out=img, slots=slots, stats=True)  # the counts, untimed
        rctx.release_state(st0)
        torch.cuda.synchronize()
        rctx.profile_enable(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
        e1.record()
        torch.cuda.synchronize()
        prof = rctx.profile_read()
        rctx.profile_enable(False)
        ms = e0.elapsed_time(e1) / steps
        vis = int(st.visible_cells)
        fma_fwd = 4 * H * (F + 4) + 11 * K * H
        fma_bwd = 4 * H * (F + 4) + 2 * 11 * K * H + 4 * H * F + 4 * H * (F + 5) + 11 * K * (H + 1)
        out = {"workload": f"neural 100,000 cells x {K} Gaussians, F={F}, H={H}, multi-scale layout, "
                           f"{len(cams)} views {W_IMG}x{H_IMG} fwd+bwd L1",
               "ms_per_step": ms, "mpix_s": len(cams) * W_IMG * H_IMG / (ms / 1e3) / 1e6,
               "decoded_view_cells_per_step": vis,
               "stage_ms_per_step": {k: v[0] / steps for k, v in prof.items() if v[1] > 0}}
        for name, fma in (("decode", fma_fwd), ("decode_bwd", fma_bwd)):
            t = prof[name][0] / steps
            if vis and t > 0:
                tf = 2.0 * fma * vis / (t / 1e3) / 1e12
                out[name] = {"ms": t, "flop_per_view_cell": 2 * fma, "tflops": tf,
                             "frac": tf / fp32_tflops if fp32_tflops else None,
                             "peak": "FP32 FMA rate of measured (dgs_probe_alu)"}
        return out
    finally:
        rctx.release_scene(sid)


def torch_empty(n):
    import torch
    return torch.empty(n, device="cuda")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--views", type=int, default=N_VIEWS, help="views per step (profiling of smaller cases)")
    ap.add_argument("--leg", default="all", choices=["all", "neural"],
                    help="neural: only the neural-cell fwd+bwd leg (its JSON object), for profiling the decode")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch

    from paper_2508_03180_gb300 import synth
    from paper_2508_03180_gb300.renderer import Context
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    rctx = Context(device=local)
    if args.leg == "neural":
        if rank == 0:
            alu = rctx.probe_alu()
            print(json.dumps(neural_fwdbwd_bench(rctx, alu["fp32_tflops"], steps=args.steps)), flush=True)
        rctx.close()
        return
    scene = synth.scene_multiscale()
    sid = rctx.upload_scene(scene)
    nv = args.views
    cams = cameras_for(rank, nv)
    slots = rctx.set_cameras(cams)
    G, N, C = scene.G, scene.N, 16
    target = torch.from_numpy(synth.target_image(nv, H_IMG, W_IMG, seed=100 + rank)).cuda().reshape(-1)
    img = torch.empty(nv * 3 * H_IMG * W_IMG, device="cuda")
    dl = torch.empty_like(img)
    loss = torch.empty(1, device="cuda")
    gflat, grads = flat_grads(G, C, "cuda")

    def step():
        _, state, _ = rctx.render(sid, cams, want_state=True, out=img, slots=slots)
        rctx.loss_l1(img, target, dl, loss)
        rctx.backward(state, dl, grads)
        rctx.release_state(state)
        reduce_grads(gflat, world)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # work counters of one step (outside the timed region)
    _, st0, stats = rctx.render(sid, cams, want_state=True, out=img, slots=slots, stats=True)
    cnt = rctx.counts(st0)
    rctx.release_state(st0)
    torch.cuda.synchronize()

    alu = rctx.probe_alu()  # measured FP32 and exp2 issue rates (outside the timed region)
    stream = torch.cuda.current_stream()
    clocks = Clocks(local)
    barrier(world)
    torch.cuda.synchronize()
    rctx.profile_enable(True)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    prof = rctx.profile_read()
    rctx.profile_enable(False)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world)
    px_step = nv * W_IMG * H_IMG
    value = weak_value(ms, world, px_step, args.steps)

    # dominant kernel and its roofline
    stage_ms = {k: v[0] / max(1, v[1]) for k, v in prof.items() if v[1] > 0}
    total_stage = sum(v[0] for v in prof.values())
    dom = max(prof, key=lambda k: prof[k][0])
    peaks, src = load_peaks()
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if dom in ("blend_fwd", "blend_bwd"):
        flop = cnt["inbox_rendered"] * (FLOP_FWD if dom == "blend_fwd" else FLOP_BWD)
        ach = flop / (stage_ms[dom] / 1e3) / 1e12
        derived = fp32_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        peak = alu["fp32_tflops"]
        # SFU work: one exp2 per in-AABB pair (forward); exp2 and a reciprocal (adjoint)
        sfu = cnt["inbox_rendered"] * (1 if dom == "blend_fwd" else 2)
        traffic = measured_traffic(dom, nv)
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic,
                "peak_source": "measured: FP32 FMA rate of dgs_probe_alu on this GPU (of measured); derived "
                               f"152 SM x 128 lanes x 2 x 2070 MHz = {derived:.1f}",
                "flop_per_launch": flop, "flop_per_unit": FLOP_FWD if dom == "blend_fwd" else FLOP_BWD,
                "units_per_launch": cnt["inbox_rendered"], "unit_def": "(pixel, Gaussian) pairs inside the AABB of "
                                                                        "blended cells",
                "sfu": {"ops_per_launch": sfu, "achieved_per_s": sfu / (stage_ms[dom] / 1e3),
                        "peak_per_s": alu["ex2_per_s"], "frac": sfu / (stage_ms[dom] / 1e3) / alu["ex2_per_s"]},
                "hbm": None if traffic is None else
                {"bytes_per_launch": traffic, "achieved_gbs": traffic / (stage_ms[dom] / 1e3) / 1e9,
                 "peak_gbs": peaks["hbm_gbs"], "frac": traffic / (stage_ms[dom] / 1e3) / 1e9 / peaks["hbm_gbs"]}}
    else:
        nbytes = {"project_fwd": G * (59 * 4) + nv * G * 48, "project_bwd": G * (59 * 4) * 2 + nv * G * 96}
        b = nbytes.get(dom, 0)
        ach = b / (stage_ms[dom] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "peak_source": src}

    # end to end through the C ABI with host buffers: parameters arrive from
    # pinned host memory (scene update), gradients and loss return to it
    import ctypes

    from paper_2508_03180_gb300 import _lib as L
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).pin_memory()
            for k in ("g_mean", "g_scale", "g_quat", "g_logit", "g_sh")}
    hflat = torch.empty(gflat.numel(), dtype=torch.float32).pin_memory()
    hgr, o = {}, 0
    for k, v in grads.items():  # views of the pinned flat buffer, in the device buffer's order
        hgr[k] = hflat[o:o + v.numel()].view(v.shape)
        o += v.numel()
    hloss = torch.empty(1).pin_memory()
    desc = L.dgs_scene_desc()
    desc.num_cells, desc.K, desc.sh_degree, desc.location = N, scene.K, scene.sh_degree, L.DGS_HOST
    for k, v in host.items():
        setattr(desc, k, v.data_ptr())
    gstruct = L.dgs_grads()
    gstruct.location = L.DGS_HOST
    for k, v in hgr.items():
        setattr(gstruct, k, v.data_ptr())
    h2d = sum(v.numel() * 4 for v in host.values())
    d2h = sum(v.numel() * 4 for v in hgr.values()) + 4

    def e2e_step():
        L.dgs_scene_update(rctx.ctx, sid, desc, stream.cuda_stream)
        _, state, _ = rctx.render(sid, cams, want_state=True, out=img, slots=slots)
        rctx.loss_l1(img, target, dl, loss)
        if world == 1:  # the adjoint writes the gradients straight into the pinned host arrays
            L.dgs_render_backward(rctx.ctx, state, dl.data_ptr(), L.DGS_DEVICE, gstruct, stream.cuda_stream)
        else:  # data parallel: summed across ranks on the device, then one download
            rctx.backward(state, dl, grads)
            reduce_grads(gflat, world)
            hflat.copy_(gflat, non_blocking=True)
        hloss.copy_(loss, non_blocking=True)
        rctx.release_state(state)

    e2e_value = None
    if not args.no_e2e:
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        e2 = args.steps
        for _ in range(e2):
            e2e_step()
        torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        e2e_value = world * px_step * e2 / t_e2e / 1e6

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if nv == N_VIEWS else WORKLOAD.replace("8 views", f"{nv} views"),
                       "views_per_step": nv, "resolution": [W_IMG, H_IMG],
                       "gaussians": G, "cells": N, "l2": "inputs larger than L2 (236 MB parameters, 384 MB records)",
                       "sort_length_per_step": int(stats.sort_length), "visible_cells_per_step": int(stats.visible_cells),
                       "termination_ratio": 1.0 - cnt["inbox_rendered"] / max(1, cnt["inbox_all"]),
                       "counts_per_step": cnt},
            "fwd_mpix_s": None,
            "stage_ms_per_step": {k: prof[k][0] / args.steps for k in prof},
            "stage_share": {k: prof[k][0] / total_stage for k in prof if total_stage > 0},
            "roofline": roof, "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": None}
    fwd_ms = sum(prof[k][0] for k in ("cell_project", "depth_sort", "count_scan", "emit", "tile_sort",
                                       "tile_ranges", "project_fwd", "blend_fwd")) / args.steps
    line["fwd_mpix_s"] = px_step / (fwd_ms / 1e3) / 1e6 if fwd_ms > 0 else None
    line["fps"] = {"fwd_bwd": world * nv * args.steps / (ms / 1e3), "fwd": nv / (fwd_ms / 1e3) if fwd_ms > 0 else None}
    line["alu_probe"] = alu
    line["streaming"] = streaming_stages(prof, args.steps, nv, scene, stats, peaks)
    line["forward_chain"] = forward_chain(line["streaming"], prof, args.steps, px_step, stats, scene, cnt, peaks,
                                          alu["fp32_tflops"] if alu else None)
    # kernel launches per step: binning 11 + sort passes + projection + blend + backward 2 + loss 2
    line["gpu_launches"] = int(args.steps * launches_per_step(stats))

    if rank == 0 and not args.no_compare:
        try:
            line["comparators"] = comparators_bench(rctx)
            line["small_fwd_bwd"] = small_fwdbwd_bench(rctx)
            line["neural_fwd_bwd"] = neural_fwdbwd_bench(rctx, alu.get("fp32_tflops") if alu else None)
        except Exception as e:  # reported beside the headline, never instead of it
            line["comparators"] = {"error": str(e)}
    if rank == 0 and not args.no_serve:
        try:
            line["serving"] = serving_bench(rctx)
        except Exception as e:  # serving is reported beside the headline, never instead of it
            line["serving"] = {"error": str(e)}
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        c0 = cams[0].as_array()
        _, t1 = cpu_sample(scene, c0, 1)
        rows = int(max(1, min(68, 15.0 / max(t1, 1e-3))))
        px, dt = cpu_sample(scene, c0, rows)
        line["cpu_baseline"] = {"value": px / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": f"oracle fwd+bwd (FP64) on tile rows 0..{rows - 1} of view 0 "
                                          f"({rows * 16 * W_IMG} px)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    rctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def streaming_stages(prof, steps, nv, scene, stats, peaks):
    """Algorithmic HBM bytes of the memory-bound stages of one step and their
    fraction of the measured copy bandwidth (CUDA-event stage times)."""
    E = nv * scene.N                          # (view, cell) entries
    L = int(stats.sort_length)                # (tile, cell) pairs
    T = int(stats.num_tiles)
    vis_rec = int(stats.visible_cells) * scene.K  # records of Gaussians of visible cells
    G, P = scene.G, 59 * 4                    # parameter bytes per Gaussian
    tile_passes = max(1, math.ceil(max(1, math.ceil(math.log2(max(2, T)))) / 8))
    algo = {
        "cell_project": E * (44 + 24),                     # cell parameters read, key/val/rect/depth/count written
        "depth_sort": E * (4 + 4 * 16),                    # histogram read + 4 passes of 8 B read + 8 B written
        "count_scan": E * 28,                              # gather and two-pass scan
        "emit": L * 8 + E * 12,                            # pairs written, entry offsets/rects read
        "tile_sort": L * (4 + tile_passes * 16),
        "tile_ranges": L * 4 + T * 8,
        "project_fwd": G * P + vis_rec * 48,               # parameters once per batch, one record per view
        "project_bwd": 2 * G * P + vis_rec * 48,           # parameters read, gradients written, records' grads read
    }
    out = {}
    for k, b in algo.items():
        if k not in prof or prof[k][1] == 0:
            continue
        ms = prof[k][0] / steps
        gbs = b / (ms / 1e3) / 1e9
        out[k] = {"bytes": int(b), "ms": ms, "gbs": gbs, "frac": gbs / peaks["hbm_gbs"]}
    tb = sum(v["bytes"] for v in out.values())
    tm = sum(v["ms"] for v in out.values())
    out["all"] = {"bytes": int(tb), "ms": tm, "gbs": tb / (tm / 1e3) / 1e9, "frac": tb / (tm / 1e3) / 1e9 / peaks["hbm_gbs"]}
    return out


def forward_chain(streaming, prof, steps, px, stats, scene, cnt, peaks, fp32_tflops):
    """The forward chain (binning, projection, blend) against the HBM roofline:
    its algorithmic bytes (the streaming stages' bytes, plus the blend's
    record read, image and per-pixel state writes) over its device time, and
    the fraction it could reach at best with the blend at the measured FP32
    rate (its counted FLOPs) and every streaming stage at the copy bandwidth:
    the blend's arithmetic, not memory, bounds the chain."""
    fwd = ("cell_project", "depth_sort", "count_scan", "emit", "tile_sort", "tile_ranges", "project_fwd")
    stream_bytes = sum(streaming[k]["bytes"] for k in fwd if k in streaming)
    blend_bytes = int(stats.visible_cells) * scene.K * 48 + px * (12 + 8)
    total = stream_bytes + blend_bytes
    t = sum(prof[k][0] for k in fwd + ("blend_fwd",)) / steps / 1e3
    hbm = peaks["hbm_gbs"] * 1e9
    out = {"bytes": int(total), "ms": t * 1e3, "gbs": total / t / 1e9, "frac": total / t / hbm,
           "blend_ms": prof["blend_fwd"][0] / steps}
    if fp32_tflops:
        t_blend = cnt["inbox_rendered"] * FLOP_FWD / (fp32_tflops * 1e12)
        t_min = t_blend + stream_bytes / hbm + blend_bytes / hbm
        out["frac_ceiling_at_alu_bound"] = total / t_min / hbm
        out["blend_ms_at_fp32_peak"] = t_blend * 1e3
    return out


def launches_per_step(stats, device_sized=True):
    # kernels of one fwd+bwd step: cell projection 1; depth sort 2 + 4 passes; gather 1; scan 3;
    # emit 1; tile sort 2 + ceil(bits/8) passes; ranges 1; projection 1; blend 1; loss 2;
    # blend adjoint 1; projection adjoint 2 (geometry, then colour); a render without stats keeps
    # the pair count on the device: + the pair-count clamp 1 and the tile sort's copy-back 1
    # (which decides on the device whether the result needs it)
    tiles = int(stats.num_tiles)
    bits = max(1, math.ceil(math.log2(max(2, tiles))))
    return (1 + (2 + 4) + 1 + 3 + 1 + (2 + math.ceil(bits / 8)) + 1 + 1 + 1 + 2 + 1 + 2
            + (2 if device_sized else 0))


if __name__ == "__main__":
    main()
