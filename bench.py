"""Throughput of the differentiable light-stage render (forward + loss + gradient).

One step = one pass of the whole hot path over one synthetic face:
geometry (morphable model, pose, normals, BVH refits, silhouettes), the
Monte-Carlo render, the Eq. 1 loss, and the gradient (interior term,
primary-visibility edges, shadow-boundary edges, normal/geometry adjoints).
Metric: forward+backward samples per second at 256x256, 16 spp, 20 lights
(35,709-vertex face, 14 lights on), in Msamples/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank renders its own face (replicas, weak
scaling): the path has no exchange step.  `--impl reference` times the CPU
oracle on the host cores on a bounded pixel sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Msamples/s at 256² 20 lights"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
# Scenes of the full-face configuration (theta seeds 1..8) timed after the
# headline run, and the timed steps of each
N_SCENES = 8
SCENE_STEPS = 10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-pixels", type=int, default=768, help="cpu_baseline leg: oracle pixels (all spp)")
    ap.add_argument("--ref-pixels", type=int, default=128, help="reference arm: oracle pixels per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--api", default="step", choices=["step", "calls"],
                    help="step: fr_step (fused render, loss and interior adjoint); calls: fr_render, fr_loss and "
                         "fr_render_backward")
    ap.add_argument("--profile-steps", type=int, default=0, help="only run this many steps, no extras (ncu)")
    ap.add_argument("--profile-res", type=int, default=0, help="with --profile-steps: image side (small ncu case)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self.rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self.rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate(t_step_ms: float, samples_per_rank: int, world: int, device=None):
    """Whole-job throughput of replicas: the slowest rank's step time (max over
    ranks) and the samples of all ranks.  Returns (t_step_ms, Msamples/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([t_step_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step_ms = float(t.item())
    return t_step_ms, world * samples_per_rank / (t_step_ms * 1e-3) / 1e6


def workload():
    from paper_1910_05200_gb300 import synthetic as S
    scene, theta, c = S.make_workload("full", seed=1)
    return scene, theta, c


def workload_config(c, scene):
    return {"workload": f"full face {scene.V:,} verts / {scene.F:,} tris, {c['W']}x{c['H']}, {c['spp']} spp, "
                        f"20 lights ({c['n_on']} on), fwd+loss+bwd",
            "W": c["W"], "H": c["H"], "spp": c["spp"], "lights": 20, "lights_on": c["n_on"],
            "vertices": scene.V, "triangles": scene.F, "l2": "flushed between timed steps (512 MB write)"}


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and the cpu_baseline leg)

def oracle_step_time(scene, theta, c, n_pix, seed):
    """Oracle forward + backward on n_pix pixels (all spp) of the full workload."""
    from oracle import Oracle, default_config
    from paper_1910_05200_gb300 import synthetic as S
    o = Oracle()
    W, H, spp = c["W"], c["H"], c["spp"]
    cfg = default_config(W=W, H=H, spp=spp, seed=seed)
    pix = S.random_pixels(W, H, n_pix, seed=seed)
    dI = np.zeros((H * W, 3))
    dI[pix] = np.random.default_rng(seed).normal(size=(len(pix), 3))
    t0 = time.perf_counter()
    o.render(cfg, scene, theta, pixels=pix)
    o.render_backward(cfg, scene, theta, dI.reshape(H, W, 3))
    dt = time.perf_counter() - t0
    return dt, len(pix) * spp


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    scene, theta, c = workload()
    cores = os.cpu_count() or 1
    for i in range(args.warmup):
        oracle_step_time(scene, theta, c, max(2, args.ref_pixels // 4), seed=100 + i)
    times, samples = [], 0
    for i in range(args.steps):
        dt, n = oracle_step_time(scene, theta, c, args.ref_pixels, seed=i)
        times.append(dt)
        samples += n
    total = sum(times)
    value = samples / total / 1e6
    sample_desc = (f"{args.ref_pixels} random pixels of {c['W']}x{c['H']} x {c['spp']} spp per step, fwd+bwd "
                   f"(adjoint on those pixels); samples/s extrapolated to the full frame")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(c, scene),
            "cpu_baseline": {"value": value, "unit": "Msamples/s", "cores": cores, "kind": "oracle",
                             "sample": sample_desc, "extrapolated": True},
            "e2e": {"value": value, "unit": "Msamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm

def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1910_05200_gb300 import synthetic as S
    from paper_1910_05200_gb300 import facert

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    scene, theta, c = workload()
    W, H, spp = c["W"], c["H"], c["spp"]
    if args.profile_steps and args.profile_res:
        W = H = args.profile_res
    r = facert.Renderer(scene, device=local)
    stream = torch.cuda.current_stream(dev)
    th = torch.tensor(theta, device=dev)
    # target: a render of perturbed parameters (another face under the same lights)
    th_t = th.clone()
    th_t[:250] += 0.3 * torch.randn(250, device=dev, generator=torch.Generator(dev).manual_seed(rank))
    target = r.render(th_t, W, H, 256 if args.profile_steps == 0 else spp, seed=999)
    image = torch.empty(H, W, 3, device=dev)
    d_image = torch.empty_like(image)
    grad = torch.empty(r.P, device=dev, dtype=torch.float64)
    loss = None
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    seed0 = 1000 * rank

    def run_step(th_, tgt_, seed):
        """One step through the public API: image, loss (returned) and gradient."""
        if args.api == "step":
            return r.step(th_, tgt_, W, H, spp, seed=seed, image=image, d_image=d_image, grad=grad)[1]
        r.render(th_, W, H, spp, seed=seed, out=image)
        ls = r.loss(th_, image, tgt_, d_image=d_image)
        r.backward(th_, d_image, W, H, spp, seed=seed, grad=grad)
        return ls

    def step(i):
        nonlocal loss
        loss = run_step(th, target, seed0 + i)

    if args.profile_steps:
        for i in range(args.profile_steps):
            step(i)
        torch.cuda.synchronize()
        r.sync()
        return

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    r.sync()

    # --- device-timed steps (inputs resident in HBM) -------------------------
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []   # per-step phase times from the library's own events (same stream)
    r.set_timing(True)
    launches0 = r.launches()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        loss = run_step(th, target, seed0 + args.warmup + i)
        ev[i][1].record(stream)
        phases.append(r.timings())        # synchronises between steps (outside the step's events)
    torch.cuda.synchronize()
    launches = r.launches() - launches0
    r.set_timing(False)
    if world > 1:
        dist.barrier()
    clocks.stop()
    r.sync()
    ms = [a.elapsed_time(b) for a, b in ev]
    ph_mean = {k: float(np.mean([p[k] for p in phases])) for k in phases[0]}
    if args.api == "step":      # fr_step's fused kernel is timed as the forward phase
        ph_mean["forward_loss_interior_fused"] = ph_mean.pop("forward")
        ph_mean.pop("interior")
    samples = W * H * spp
    t_step, value = aggregate(float(np.mean(ms)), samples, world, dev)

    # --- end to end through the public API, host buffers ---------------------
    th_h = torch.tensor(theta).pin_memory()
    tgt_h = target.cpu().pin_memory()
    grad_h = torch.empty(r.P, dtype=torch.float64).pin_memory()
    loss_h = torch.empty(1, dtype=torch.float64).pin_memory()
    th_d = torch.empty_like(th)
    tgt_d = torch.empty_like(target)
    e2e_ev = []
    for i in range(max(3, args.steps // 2)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        th_d.copy_(th_h, non_blocking=True)
        tgt_d.copy_(tgt_h, non_blocking=True)
        ls = run_step(th_d, tgt_d, 7 + i)
        grad_h.copy_(grad, non_blocking=True)
        loss_h.copy_(ls, non_blocking=True)
        b.record(stream)
        e2e_ev.append((a, b))
    torch.cuda.synchronize()
    t_e2e = float(np.mean([a.elapsed_time(b) for a, b in e2e_ev]))
    h2d = th_h.numel() * 4 + tgt_h.numel() * 4
    d2h = grad_h.numel() * 8 + 8

    # --- the other scenes of the full-face configuration: theta seeds 1..8 ----
    # (seed 1 is the headline above); same mesh and context, each with its own
    # target, warm-up and timed steps, L2 flushed between steps
    scene_ms = []
    for sd in range(1, N_SCENES + 1):
        th_s = torch.tensor(S.make_workload("full", seed=sd)[1], device=dev)
        th_st = th_s.clone()
        th_st[:250] += 0.3 * torch.randn(250, device=dev, generator=torch.Generator(dev).manual_seed(sd))
        tgt_s = r.render(th_st, W, H, 256, seed=999)
        for i in range(args.warmup):
            run_step(th_s, tgt_s, 5000 + i)
        evs = []
        for i in range(SCENE_STEPS):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run_step(th_s, tgt_s, 6000 + i)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        scene_ms.append(float(np.mean([a.elapsed_time(b) for a, b in evs])))
    r.sync()
    scenes = {"theta_seeds": list(range(1, N_SCENES + 1)), "steps_each": SCENE_STEPS, "ms_per_step": scene_ms,
              "median_value": float(samples / (np.median(scene_ms) * 1e-3) / 1e6), "unit": "Msamples/s"}

    # --- roofline: the dominant kernel and the whole step -------------------
    # counters of one step through the benchmarked call (reset by the call)
    r.set_counters(True)
    run_step(th, target, seed0 + args.warmup)
    cnt = [int(x) for x in r.counters()]
    r.set_counters(False)
    from paper_1910_05200_gb300 import roofline as RF
    peaks = facert.probe_peaks(local)            # measured FMA and L2 roofs, SM count
    clk = clocks.summary()
    peak = peaks["fp32_tflops"]
    flops_sedge = float(RF.sedge_search_flops(cnt))
    t_sedge = ph_mean["shadow_edge_search"] * 1e-3
    achieved = flops_sedge / t_sedge / 1e12
    flops_step = float(RF.step_flops(cnt, samples, c["n_on"]))
    step_achieved = flops_step / (t_step * 1e-3) / 1e12
    l2_bytes = RF.SEDGE_L2_BYTES
    roof = {"bound": "alu", "kernel": "k_bwd_sedge (shadow-edge search and pick)", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": RF.SEDGE_TRAFFIC_BYTES,
            "peak_note": "measured: FP32 FMA probe (fr_probe_peaks) on this GPU, best of 5 runs",
            "peak_nominal": RF.fp32_peak_tflops(clk.get("sm_mhz") or 2070.0, peaks["sm_count"]),
            "sm_count": peaks["sm_count"],
            "l2_peak_gbs": peaks["l2_read_gbs"],
            "l2_bytes": l2_bytes,
            "l2_frac": (l2_bytes / t_sedge / 1e9 / peaks["l2_read_gbs"]) if l2_bytes else None,
            "flops_per_launch": flops_sedge, "ms_per_launch": ph_mean["shadow_edge_search"],
            "contributions": {"kernel": "k_bwd_sedge_add", "ms_per_launch": ph_mean["shadow_edge_contributions"],
                              "flops_per_launch": float(RF.sedge_add_flops(cnt))},
            "counts_sedge": dict(zip(("ray_nodes", "tri_tests", "edge_nodes_per_warp", "edge_tests", "clip_tests",
                                      "edges_classified_per_warp"), cnt[RF.K_SEDGE:RF.K_SEDGE + 6])),
            "step": {"flops_per_step": flops_step, "ms_per_step": t_step, "achieved": step_achieved,
                     "frac": step_achieved / peak, "unit": "TFLOP/s"}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Msamples/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(c, scene),
                "api": "fr_step" if args.api == "step" else "fr_render + fr_loss + fr_render_backward",
                "ms_phases": ph_mean,
                "e2e": {"value": world * samples / (t_e2e * 1e-3) / 1e6, "unit": "Msamples/s",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": t_e2e},
                "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "scenes": scenes,
                "loss": float(loss.item())}
        if not args.no_cpu_baseline and world == 1:
            dt, n = oracle_step_time(scene, theta, c, args.cpu_pixels, seed=3)
            line["cpu_baseline"] = {"value": n / dt / 1e6, "unit": "Msamples/s", "cores": os.cpu_count(),
                                    "kind": "oracle", "extrapolated": True,
                                    "sample": f"{args.cpu_pixels} random pixels of {W}x{H} x {c['spp']} spp, "
                                              f"fwd+bwd with the adjoint on those pixels, {dt:.1f} s; samples/s "
                                              f"extrapolated to the full frame"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
