#!/usr/bin/env python
"""Throughput of one rendered frame of a posed performer (rays/s).

Workload: 512x512 image, 128 samples per ray, occupancy bitfield 128^3
(~15-18 % of cells set), hash grid of 16 levels x 2 features with 2^19 f16
entries (N 16..2048), canonical MLP 32-64-64-64-4, residual MLP with 6 PE
bands, 64^3 x 25 float32 weight volume, early ray termination at T < 1e-4.
One step = a fresh pose (forward kinematics + posed occupancy bitfield) and
the whole render (ray march with compaction, the fused per-sample field,
compositing), through the C ABI.  Synthetic, seeded inputs shaped like the
paper's workloads (one ~1.7 m performer in a 2 m box, 128 samples per ray).

With torchrun (N > 1) every rank renders its own frames (independent
replicas, no collective: weak scaling).  --impl reference times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/sec (512x512 frame render, 128 samples/ray, occupancy + ERT)"
# The paper's own speed figures (one RTX 3080 Ti, ZJU-MoCap; Table 1, Table 2, Sec. 5): context
# only, on other hardware and other data, never a ratio target.
PAPER_CONTEXT = {
    "hardware": "RTX 3080 Ti (Ampere), tiny-cuda-nn fp16 MLPs",
    "inference": "1.209 frames/s at 1024x1024 (at most ~1.27 M rays/s), +213 % over HumanNeRF",
    "training": "3.92 h for 150K iterations of 2400 rays (~94 ms per iteration), -44.5 % against HumanNeRF",
}
UNIT = "rays/s"
L2_FLUSH_BYTES = 512 << 20          # larger than the 129 MB L2


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--mlp", default="bf16", choices=["f32", "bf16", "f16", "fp8"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--mma", choices=["pipeline", "tcgen05", "sync", "sync2"], default="pipeline",
                   help="bf16/f16 MLP path: the warp-specialised tcgen05 pipeline (default), tcgen05 with one "
                        "group per tile, or warp-level mma.sync over one or two m-tiles")
    p.add_argument("--cpu-pixels", type=int, default=24576)
    p.add_argument("--train-steps", type=int, default=5)
    p.add_argument("--train-only", action="store_true", help="time only the training step")
    p.add_argument("--train-rays", type=int, default=1 << 18, help="rays per training batch")
    p.add_argument("--train-full", action="store_true",
                   help="with --train-only: train the pose refiner and CNN_skel as well (patch batches)")
    p.add_argument("--train-layout", choices=["uniform", "patch"], default="uniform",
                   help="uniform random pixels, or 6 patches of 20x20 per image with MSE weight 0.2")
    p.add_argument("--serve-seconds", type=float, default=30.0, help="length of the serving run (0 = skip)")
    p.add_argument("--serve-only", action="store_true", help="run only the serving scenario")
    p.add_argument("--serve-slots", type=int, default=2, help="concurrent requests on the device (server slots)")
    p.add_argument("--no-sweep", dest="sweep", action="store_false", help="skip the precision sweep")
    p.add_argument("--sweep-only", action="store_true", help="run only the precision sweep")
    return p.parse_args()


def dist_setup(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling (200 ms) of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def workload():
    from paper_2306_16541_gb300 import synth
    cfg = synth.config_frame512()
    rng = np.random.default_rng(4321)
    poses = [synth.random_pose(rng) for _ in range(8)]
    return cfg, poses


def cpu_baseline(cfg, poses, n_pixels, seed=0):
    """The FP64 oracle, as it stands, on n_pixels random pixels of the same frame."""
    import torch
    from oracle import field as OF
    from oracle import render as OR
    cam = cfg["camera"]
    rng = np.random.default_rng(seed)
    px = rng.integers(0, cam.width, n_pixels)
    py = rng.integers(0, cam.height, n_pixels)
    P = OF.Params(cfg["subject"])
    t0 = time.perf_counter()
    OR.render_pixels(cfg["subject"], P, poses[0], cam, px, py, True)
    dt = time.perf_counter() - t0
    # the same oracle on one core, on a smaller sample of the same pixels
    threads = torch.get_num_threads()
    n1 = max(256, n_pixels // 16)
    torch.set_num_threads(1)
    try:
        t1 = time.perf_counter()
        OR.render_pixels(cfg["subject"], P, poses[0], cam, px[:n1], py[:n1], True)
        dt1 = time.perf_counter() - t1
    finally:
        torch.set_num_threads(threads)
    return dict(value=n_pixels / dt, unit=UNIT, cores=threads, kind="oracle",
                sample=f"{n_pixels} random pixels of one 512x512 frame (128 samples each, occupancy; "
                       f"FP64 torch CPU, no early termination), {dt:.1f} s",
                one_core={"value": n1 / dt1, "unit": UNIT, "cores": 1,
                          "sample": f"the first {n1} of those pixels, {dt1:.1f} s"},
                host=_host_cpu())


def _host_cpu() -> str:
    """The host's CPU model and logical core count (from /proc/cpuinfo or lscpu)."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return f"{model or 'unknown CPU'}, {os.cpu_count()} logical cores"


def train_bench(nr, device, steps, warmup=2, n=1 << 18, layout="uniform", full=False):
    """Training-step time on the training workload: 16 frames of 512x512 with seeded
    poses, targets rendered from a seeded ground-truth field of the tiny workload's
    shape, 2^18 random pixel rays x 128 stratified samples, forward + backward +
    Adam (lr 1e-2, beta (0.9, 0.99)).  CUDA events on the training stream.
    layout "patch" draws the rays as 6 patches of 20x20 pixels per image (110 images,
    264,000 rays) and weights the MSE by 0.2 (Sec. 5.2).  full: the whole motion model of
    Sec. 4 is trained as well -- the pose refiner MLP_theta (4 x 256) and the weight volume
    generated by CNN_skel (channels 1024-512-256-128-64, prior = the initial volume)."""
    import torch
    from paper_2306_16541_gb300 import synth
    gt = synth.subject(700, hash_scale=0.5, res_last_std=0.02)
    gt["mlp_layers"][-1][1][3] = 3.0
    gt["mlp_params"] = synth.pack_layers(gt["mlp_layers"])
    trainee = synth.subject(700)
    frames = synth.training_frames(701, 16, res=512)
    G = nr.Subject(gt, device=device)
    targets = []
    for i, cam in enumerate(frames["cameras"]):
        G.set_pose(frames["axis_angle"][i], frames["root_t"][i])
        targets.append(G.render(cam, nr.make_opts("f32"))[..., :3].clone())
    G.close()
    targets = torch.stack(targets)
    Sub = nr.Subject(trainee, device=device)
    Sub.set_frames(frames["axis_angle"], frames["root_t"], frames["cameras"])
    if full:
        Sub.set_pose_refiner(synth.refiner_layers(703))
        Sub.set_weight_cnn(synth.cnn_layers(704), synth.cnn_latent(705),
                           np.log(np.asarray(trainee["wvol"], np.float64) + 1e-6).astype(np.float32))
    gen = torch.Generator(device="cuda").manual_seed(702)
    batches = []
    weight = 0.0
    if layout == "patch":
        weight = nr.PAPER_MSE_WEIGHT
        n_img = (n + 2399) // 2400
        n = n_img * 2400
    for k in range(steps + warmup):
        if layout == "patch":
            pb = synth.patch_batch(710 + k, 16, n_img)
            f, px, py = (torch.from_numpy(pb[c].astype(np.int32)).cuda() for c in ("frame", "px", "py"))
        else:
            f = torch.randint(0, 16, (n,), device="cuda", generator=gen, dtype=torch.int32)
            px = torch.randint(0, 512, (n,), device="cuda", generator=gen, dtype=torch.int32)
            py = torch.randint(0, 512, (n,), device="cuda", generator=gen, dtype=torch.int32)
        batches.append((f, px, py, targets[f.long(), py.long(), px.long()].contiguous()))
    losses = []
    for k in range(warmup):
        losses.append(Sub.train_step(*batches[k], 128, 5000 + k, lr=1e-2, lr_scale=nr.PAPER_LR_SCALE,
                                     loss_weight=weight))
    torch.cuda.synchronize()
    ms = []
    for k in range(warmup, warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        losses.append(Sub.train_step(*batches[k], 128, 5000 + k, lr=1e-2, lr_scale=nr.PAPER_LR_SCALE,
                                     loss_weight=weight))
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    Sub.close()
    shape = "6 patches of 20x20 per image, MSE weight 0.2" if layout == "patch" else "uniform pixels"
    extra = ", pose refiner 4x256 + CNN_skel 1024-512-256-128-64" if full else ""
    return {"workload": f"16 frames 512x512, {n} rays ({shape}) x 128 samples, fp32 forward+backward+Adam{extra}",
            "lr": "1e-2 (hash, canonical MLP), 1e-3 (weight volume, residual MLP)",
            "ms": statistics.mean(ms), "ms_min": min(ms), "ms_steps": [round(v, 2) for v in ms],
            "steps": steps, "warmup": warmup,
            "rays_per_s": n / (statistics.mean(ms) / 1000.0),
            "samples_per_s": n * 128 / (statistics.mean(ms) / 1000.0),
            "loss_first": losses[0], "loss_last": losses[-1]}


def occupancy_bench(nr, device, mlp, steps=5):
    """Density-grid occupancy (Sec. 2.3 for subjects without ellipsoids) on the frame workload's
    field with a body-shaped density: the canonical refresh (sigma at 128^3 cell centres,
    threshold 1e-3, dilation 1), the posing through the warp (128^3 cells), and a 512x512x128
    frame rendered with the grid, against the same frame without skipping."""
    import torch
    from paper_2306_16541_gb300 import synth
    cfg = synth.config_frame512()
    subj = synth.shaped_density(cfg["subject"])
    S = nr.Subject(subj, device=device)
    cam = nr.make_camera(cfg["camera"])
    out = torch.empty(cam.height, cam.width, 4, device="cuda")
    rng = np.random.default_rng(3300)
    poses = [synth.random_pose(rng) for _ in range(steps + 1)]

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    S.set_pose(*poses[0])
    S.refresh_occupancy(1e-3, 1)
    S.occupancy()
    refresh = [timed(lambda: S.refresh_occupancy(1e-3, 1)) for _ in range(steps)]
    pose_ms, frame_grid, frame_full, live_grid, live_full = [], [], [], [], []
    opts_g = nr.make_opts(mlp, "f16", True, 1e-4, profile=True)
    opts_n = nr.make_opts(mlp, "f16", False, 1e-4, profile=True)
    for p in poses[1:]:
        S.set_pose(*p)
        pose_ms.append(timed(lambda: S.occupancy()))          # posing + a 256 KiB readback
        frame_grid.append(timed(lambda: S.render(cam, opts_g, out)))
        live_grid.append(S.stage_times()["live_samples"])
        frame_full.append(timed(lambda: S.render(cam, opts_n, out)))
        live_full.append(S.stage_times()["live_samples"])
    S.close()
    n_rays = cam.width * cam.height
    return {"workload": "frame 512x512x128 field with body-shaped density, canonical and posed grids 128^3",
            "refresh_ms": statistics.mean(refresh), "pose_ms": statistics.mean(pose_ms),
            "frame_ms_grid": statistics.mean(frame_grid), "frame_ms_no_skip": statistics.mean(frame_full),
            "rays_per_s_grid": n_rays / (statistics.mean(frame_grid) / 1000.0),
            "live_samples_grid": statistics.mean(live_grid), "live_samples_no_skip": statistics.mean(live_full)}


def serve_bench(nr, device, mlp, rate=240.0, duration=3.0, n_subjects=8, max_slots=16, policy=None, baseline=True):
    """Multi-user serving: n_subjects frame-workload subjects resident on the device, Poisson
    arrivals at `rate` req/s for `duration` s, each request a random subject, a camera on the
    2.5 m sphere, a fresh pose (<= 30 deg per bone) and 256^2 / 512^2 / 1024^2 with probabilities
    0.3 / 0.5 / 0.2, 128 samples, occupancy, ERT.  Latency = submit to completion.  The same
    requests are then rendered one at a time through nr_set_pose + nr_render (a plain queue)."""
    import torch
    from paper_2306_16541_gb300 import synth
    subs = [nr.Subject(synth.config_frame512(seed=3000 + i)["subject"], device=device) for i in range(n_subjects)]
    reqs = synth.request_stream(3100, n_subjects, rate, duration)
    opts = nr.make_opts(mlp, "f16", True, 1e-4)
    sizes = [q["camera"].width * q["camera"].height for q in reqs]
    arena = torch.empty(sum(sizes) * 4, device="cuda")
    outs, off = [], 0
    for n in sizes:
        outs.append(arena[off:off + 4 * n])
        off += 4 * n
    srv = nr.Server(max_bytes=max_slots * (1200 << 20), max_slots=max_slots, device=device)   # 2^20-ray chunks
    if policy:
        srv.set_policy(**policy)
    for S in subs:
        srv.add_subject(S)
    # warm-up: one request per resolution
    warm = [srv.submit(srv.request(0, q["camera"], q["axis_angle"], q["root_t"], opts, outs[i]))
            for i, q in enumerate(reqs[:6])]
    for w in warm:
        srv.wait(w, 120000)
    torch.cuda.synchronize()
    # the request records are built before the clock starts; each is submitted at its arrival
    # time (a sleep to within 1 ms of it, then a spin: a plain sleep wakes late and bunches arrivals)
    built = [srv.request(q["subject"], q["camera"], q["axis_angle"], q["root_t"], opts, outs[i])
             for i, q in enumerate(reqs)]
    t0 = time.perf_counter()
    ids = []
    for q, rq in zip(reqs, built):
        due = t0 + q["t_arrive"]
        dt = due - time.perf_counter()
        if dt > 1e-3:
            time.sleep(dt - 1e-3)
        while time.perf_counter() < due:
            pass
        ids.append(srv.submit(rq))
    lat = [srv.wait(i, 600000) for i in ids]
    t_end = time.perf_counter()
    st = srv.stats()
    srv.close()
    by_res = {}
    for q, l in zip(reqs, lat):
        by_res.setdefault(q["camera"].width, []).append(l)
    # one at a time through the plain path (service times), then a FIFO queue over the same arrivals
    service = []
    for i, q in enumerate(reqs if baseline else []):
        S = subs[q["subject"]]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        S.set_pose(q["axis_angle"], q["root_t"])
        nr.nr_render(S.h, nr.make_camera(q["camera"]), opts, outs[i])
        e1.record()
        torch.cuda.synchronize()
        service.append(e0.elapsed_time(e1))
    for S in subs:
        S.close()
    fifo, t_free = [], 0.0
    for q, sv in zip(reqs, service):
        start = max(q["t_arrive"] * 1000.0, t_free)
        t_free = start + sv
        fifo.append(t_free - q["t_arrive"] * 1000.0)
    pct = lambda v, p: float(np.percentile(np.asarray(v), p))
    return {"workload": f"{n_subjects} subjects (512^2-workload fields, bf16 MLP), Poisson {rate:g} req/s for "
                        f"{duration:g} s, 256/512/1024 px at 0.3/0.5/0.2, 128 samples, occupancy + ERT",
            "requests": len(reqs), "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": max(lat),
            "p50_ms_by_res": {str(k): pct(v, 50) for k, v in sorted(by_res.items())},
            "p99_ms_by_res": {str(k): pct(v, 99) for k, v in sorted(by_res.items())},
            "rays_per_s": sum(sizes) / (t_end - t0), "peak_active": st["peak_active"], "slots": st["slots"],
            "one_at_a_time": ({"rays_per_s": sum(sizes) / (sum(service) / 1000.0),
                               "p50_ms": pct(fifo, 50), "p99_ms": pct(fifo, 99),
                               "mean_service_ms": float(np.mean(service))} if baseline else None)}


SWEEP_REFERENCE = os.path.join(ROOT, "tests", "golden", "sweep_oracle_pixels.txt")


def sweep_reference() -> dict:
    """The FP64 oracle's RGBA at the sweep's pixels, stored by tests/golden/make_sweep_reference.py:
    {variant: (px, py, rgba [n][4])}."""
    rows = {}
    with open(SWEEP_REFERENCE) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows.setdefault(t[0], []).append([float(v) for v in t[1:]])
    out = {}
    for name, r in rows.items():
        a = np.array(r, np.float64)
        out[name] = (a[:, 0].astype(np.int64), a[:, 1].astype(np.int64), a[:, 2:6])
    return out


def sweep_bench(nr, device):
    """Precision sweep: 1920x1080, 192 samples per ray, the tiny workload's field with 2^20
    entries per level (and a textured variant), no occupancy.  Every MLP tier (f32 on CUDA
    cores, f32_tc = float32 accuracy on the tensor cores, bf16, f16, fp8 on the default tcgen05
    pipeline, fp8_sync = fp8 on warp-level mma.sync) x hash-feature tier
    (f32, f16): rays/s (CUDA events), PSNR, max-abs and per-pixel error percentiles against the
    FP64 oracle's values at seeded pixels (stored by tests/golden/make_sweep_reference.py), and
    PSNR against the f32 GPU image."""
    import torch
    from paper_2306_16541_gb300 import synth
    cfg, variants = synth.sweep_variants()
    cam = cfg["camera"]
    stored = sweep_reference()
    px, py = synth.sweep_pixels(cam.width, cam.height)
    out = {}
    for variant, subj in variants:
        spx, spy, ref = stored[variant]
        if not (np.array_equal(spx, px) and np.array_equal(spy, py)):
            raise RuntimeError(f"{SWEEP_REFERENCE} holds other pixels than the sweep's; regenerate it")
        S = nr.Subject(subj, device=device)
        S.set_pose(*cfg["pose"])
        img = torch.empty(cam.height, cam.width, 4, device="cuda")
        base = None
        rows = []
        for mlp in ("f32", "f32_tc", "bf16", "f16", "fp8", "fp8_sync"):
            for feat in ("f32", "f16"):
                dtype = {"f32_tc": "f32", "fp8_sync": "fp8"}.get(mlp, mlp)
                opts = nr.make_opts(dtype, feat, False, 0.0, f32_tc=mlp == "f32_tc", mma_sync=mlp == "fp8_sync")
                S.render(cam, opts, img)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                S.render(cam, opts, img)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                got = img.cpu().numpy()
                if base is None:
                    base = got.copy()
                d = got[py, px] - ref
                mse = float((d ** 2).mean())
                mse_gpu = float(((got - base) ** 2).mean())
                rows.append({"mlp": mlp, "feat": feat, "ms": ms, "rays_per_s": cam.width * cam.height / (ms / 1e3),
                             "psnr_vs_oracle_db": (10 * np.log10(1.0 / mse)) if mse > 0 else float("inf"),
                             "max_abs_vs_oracle": float(np.abs(d).max()),
                             "abs_err_p50_p99_vs_oracle": [float(np.percentile(np.abs(d), 50)),
                                                           float(np.percentile(np.abs(d), 99))],
                             "psnr_vs_f32_gpu_db": (10 * np.log10(1.0 / mse_gpu)) if mse_gpu > 0 else float("inf")})
        S.close()
        out[variant] = rows
    return {"workload": "1920x1080, 192 samples, 8x2 levels of 2^20 entries, MLP 32-64-64-4, no occupancy",
            "oracle_pixels": int(len(px)), "oracle_values": "tests/golden/sweep_oracle_pixels.txt", "tiers": out}


def oracle_pixels_time(cfg, poses, n_pixels, seed):
    """Seconds the FP64 oracle, as it stands, takes for n_pixels random pixels of the frame."""
    from oracle import field as OF
    from oracle import render as OR
    cam = cfg["camera"]
    rng = np.random.default_rng(seed)
    px = rng.integers(0, cam.width, n_pixels)
    py = rng.integers(0, cam.height, n_pixels)
    P = OF.Params(cfg["subject"])
    t0 = time.perf_counter()
    OR.render_pixels(cfg["subject"], P, poses[0], cam, px, py, True)
    return time.perf_counter() - t0


def run_reference(a):
    """The reference arm: the FP64 oracle on the host cores; a step is 256 random pixels of the
    512 x 512 x 128 frame (the whole frame would take minutes), timed as it runs."""
    import torch
    rank, world, local = dist_setup(a.gpus)
    if rank != 0:
        return
    cfg, poses = workload()
    n_px = 256
    times = []
    for i in range(a.warmup + a.steps):
        dt = oracle_pixels_time(cfg, poses, n_px, seed=i)
        if i >= a.warmup:
            times.append(dt)
    step_s = statistics.mean(times)
    v = n_px / step_s
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * step_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "frame_512x512_s128_occupancy",
                       "sample_per_step": f"{n_px} random pixels of one 512x512 frame (128 samples each)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{n_px} random pixels of one 512x512 frame per step, FP64 torch CPU, "
                                       f"mean of {a.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# Per frame of the frame workload, from one ncu capture of the four field launches of a frame on
# the default bf16 path, valid while the kernel sources have the SHA-256 given: DRAM bytes read +
# written, and the bytes of the L1 sectors the global loads touched.
FIELD_CAPTURE = {"sha256": "779db2254c3b338b87bd26ea35baab53aed6570da7f1ef101152c814c8648775",
                 "dram_bytes_per_frame": 152621056 + 55193600,
                 "l1_sector_bytes_per_frame": 473844545 * 32,
                 "l2_bytes_per_frame": 4511446144,
                 "live_samples_per_frame": 6173672}
FIELD_SOURCES = ["field_ws.cu", "gather.cuh", "t5.cuh", "field.cuh", "mma.cuh", "common.cuh", "render.cuh"]


def field_bytes_per_sample(subj, table_bytes: int = 2) -> int:
    """Algorithmic bytes of the field kernel per live sample: the 8 corners of every bone
    channel of the float32 weight volume (24 x 8 x 4 B), the 8 corners of every hash level
    (L x 8 x 2 features x table_bytes), the sample read (x, y, z, delta: 16 B) and its
    (r, g, b, alpha) written (16 B)."""
    n_bones = len(subj["parents"])
    return n_bones * 8 * 4 + int(subj["hash_levels"]) * 8 * int(subj["hash_feats"]) * table_bytes + 16 + 16


def mlp_flops_per_sample(subj) -> int:
    """Algorithmic flops (2 per multiply-add) of both MLPs per live sample, unpadded: the
    residual MLP (PE of 3 + 6 * bands dims and the 64 hidden units, layer 4 seeing [h3, gamma],
    3 outputs; the pose enters as a bias) and the canonical MLP (L x F hash features, hidden
    layers of 64, 4 outputs)."""
    bands = int(subj.get("res_pe_freqs", 6))
    g = 3 + 6 * bands
    w = 64
    res = g * w + w * w + w * w + (w + g) * w + w * 3 if int(subj.get("res_enabled", 1)) else 0
    hidden = len(subj["mlp_layers"]) - 1
    can = int(subj["hash_levels"]) * int(subj["hash_feats"]) * w + (hidden - 1) * w * w + w * 4
    return 2 * (res + can)


def field_capture():
    """The ncu figures of FIELD_CAPTURE if the kernel sources are still the captured ones, else None."""
    import hashlib
    if FIELD_CAPTURE["sha256"] is None:
        return None
    h = hashlib.sha256()
    for f in FIELD_SOURCES:
        with open(os.path.join(ROOT, "paper_2306_16541_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return FIELD_CAPTURE if h.hexdigest() == FIELD_CAPTURE["sha256"] else None


def gather_ceiling(nr, device, subj, hbm_gbs):
    """The measured ceiling of the field kernel's algorithmic bytes: L2-resident random gathers of
    4 B (hashed levels) and 16 B (corner blocks of the weight volume and of the dense levels),
    measured now on this GPU (nr_l2_gather_rate, a table of the f16 hash table's size), mixed by the
    kernel's byte counts per live sample; the sample's own 32 B stream from HBM."""
    table = 1 << (int(subj["log2_T"]) + 2 + 4)            # 2^log2_T entries x 4 B x 16 levels
    r4 = nr.nr_l2_gather_rate(device, table, 4) / 1e9
    r16 = nr.nr_l2_gather_rate(device, table, 16) / 1e9
    levels = [int(v) for v in subj["level_res"]]
    T = 1 << int(subj["log2_T"])
    dense = sum(1 for n in levels if (n + 1) ** 3 <= T)
    feat_b = int(subj["hash_feats"]) * 2
    b16 = len(subj["parents"]) * 8 * 4 + dense * 8 * feat_b
    b4 = (len(levels) - dense) * 8 * feat_b
    t = b16 / r16 + b4 / r4 + 32 / hbm_gbs               # ns per live sample at the ceilings
    return {"gbs": (b16 + b4 + 32) / t, "gather_4B_gbs": r4, "gather_16B_gbs": r16,
            "bytes_16B": b16, "bytes_4B": b4, "bytes_stream": 32}


def run_ours(a):
    import torch
    rank, world, local = dist_setup(a.gpus)
    torch.cuda.set_device(local)
    from paper_2306_16541_gb300 import build
    if rank == 0:
        build.build()
    barrier(world)
    from paper_2306_16541_gb300 import nr
    if a.train_only:
        print(json.dumps({"train_step": train_bench(nr, local, a.train_steps, n=a.train_rays,
                                                    layout="patch" if a.train_full else a.train_layout,
                                                    full=a.train_full)}))
        return
    if a.sweep_only:
        print(json.dumps({"precision_sweep": sweep_bench(nr, local)}))
        return
    if a.serve_only:
        print(json.dumps({"serving": serve_bench(nr, local, a.mlp, duration=a.serve_seconds,
                                                 max_slots=a.serve_slots)}))
        return

    cfg, poses = workload()
    cam = nr.make_camera(cfg["camera"])
    W, H = cam.width, cam.height
    n_rays = W * H
    t5 = a.mma == "tcgen05" and a.mlp in ("bf16", "f16")
    m2 = a.mma == "sync2"
    ms = a.mma == "sync"
    opts = nr.make_opts(a.mlp, "f16", True, 1e-4, tcgen05=t5, mma2=m2, mma_sync=ms)
    popts = nr.make_opts(a.mlp, "f16", True, 1e-4, profile=True, tcgen05=t5, mma2=m2, mma_sync=ms)
    S = nr.Subject(cfg["subject"], device=local)
    out = torch.empty(H, W, 4, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step(i, o):
        S.set_pose(*poses[(i + rank) % len(poses)])
        S.render(cam, o, out)

    for i in range(a.warmup):
        step(i, opts)
    step(0, popts)                          # creates the profiling events
    torch.cuda.synchronize()
    barrier(world)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    launches0 = nr.nr_launch_count()
    clocks = Clocks(local)
    torch.cuda.synchronize()
    barrier(world)
    for i in range(a.steps):
        flush.zero_()                       # L2 flush between timed steps (outside the events)
        ev[i][0].record()
        step(i, opts)
        ev[i][1].record()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = nr.nr_launch_count() - launches0
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_ms = max_over_ranks(sum(step_ms), world)
    value = world * n_rays * a.steps / (total_ms / 1000.0)

    # the same steps again with NR_RENDER_PROFILE: an event at every launch boundary gives the
    # stage split and the field kernel's own duration (the roofline), and the field counts the live
    # samples and the bone channels it reads; the instrumented step is reported beside the plain one
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    stages = []
    for i in range(a.steps):
        flush.zero_()
        pev[i][0].record()
        step(i, popts)
        pev[i][1].record()
        stages.append(S.stage_times())      # waits for the render's boundary events
    torch.cuda.synchronize()
    profiled_ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in pev)

    # end to end through the C ABI with host buffers: pose from host memory,
    # image into pinned host memory (the library copies it back), wall clock
    host_out = torch.empty(H, W, 4, dtype=torch.float32).pin_memory()
    opts_e2e = nr.make_opts(a.mlp, "f16", True, 1e-4, tcgen05=t5, mma2=m2, mma_sync=ms)
    for i in range(2):
        S.set_pose(*poses[i])
        nr.nr_render(S.h, cam, opts_e2e, host_out)
    barrier(world)
    t0 = time.perf_counter()
    for i in range(a.steps):
        S.set_pose(*poses[(i + rank) % len(poses)])
        nr.nr_render(S.h, cam, opts_e2e, host_out)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = world * n_rays * a.steps / e2e_s

    train = train_bench(nr, local, a.train_steps, n=a.train_rays, layout=a.train_layout) if a.train_steps > 0 else None
    train_full = (train_bench(nr, local, a.train_steps, n=a.train_rays, layout="patch", full=True)
                  if a.train_steps > 0 else None)
    occupancy = occupancy_bench(nr, local, a.mlp) if a.train_steps > 0 else None
    serving = (serve_bench(nr, local, a.mlp, duration=a.serve_seconds, max_slots=a.serve_slots)
               if a.serve_seconds > 0 else None)
    sweep = sweep_bench(nr, local) if (a.sweep and rank == 0) else None

    field_ms = statistics.mean(s["field_ms"] for s in stages)
    live = statistics.mean(s["live_samples"] for s in stages)
    s = cfg["subject"]
    bytes_per_sample = field_bytes_per_sample(s, table_bytes=2)
    achieved = bytes_per_sample * live / (field_ms / 1000.0) / 1e9
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs", 6800.0)
    ceiling = gather_ceiling(nr, local, s, hbm)
    default_path = a.mma == "pipeline" and a.mlp in ("bf16", "f16")
    cap = field_capture() if default_path else None
    # bytes the kernel requests: the bone channels it reads (counted by the profiled renders), the
    # hash corners and the sample's own stream; and the gather ceiling of that mix
    bones_read = statistics.mean(s_["bones_read_per_sample"] for s_ in stages)
    requested = None
    if bones_read > 0:
        b16_req = bones_read * 8 * 4 + ceiling["bytes_16B"] - len(s["parents"]) * 8 * 4
        t_req = b16_req / ceiling["gather_16B_gbs"] + ceiling["bytes_4B"] / ceiling["gather_4B_gbs"] + 32 / hbm
        req_bytes = b16_req + ceiling["bytes_4B"] + 32
        req_ach = req_bytes * live / (field_ms / 1000.0) / 1e9
        requested = {"bytes_per_live_sample": req_bytes, "bone_channels_read": bones_read,
                     "achieved": req_ach, "peak": req_bytes / t_req, "frac": req_ach / (req_bytes / t_req)}
    mlp_flops = mlp_flops_per_sample(s)
    mlp_tflops = mlp_flops * live / (field_ms / 1000.0) / 1e12
    # fp8 operands: the measured bf16 peak times the nominal fp8 / bf16 ratio (4.5 / 2.25 PFLOP/s)
    ratio = 2.0 if a.mlp == "fp8" else 1.0
    mlp_peak = ratio * peaks.get("bf16_tflops", 1900.0)
    mlp_peak_sus = ratio * peaks.get("bf16_tflops_sustained", 1700.0)
    kernel_name = {"pipeline": "field_ws_kernel (warp-specialised tcgen05)", "tcgen05": "field_t5_kernel",
                   "sync": "field_tc_kernel (mma.sync)", "sync2": "field_tc_kernel (mma.sync, two m-tiles)"}[a.mma]
    if a.mlp == "f32":
        kernel_name = "field_f32_kernel"
    elif a.mlp == "fp8" and a.mma != "pipeline":
        kernel_name = "field_fp8_kernel (mma.sync)"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": total_ms / a.steps, "ms_per_step_profiled": profiled_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16", "f16": "f16", "fp8": "fp8e4m3"}[a.mlp], "data": "synthetic",
        "config": {"workload": "frame_512x512_s128_occupancy", "image": [W, H], "samples_per_ray": 128,
                   "occupancy_grid": 128, "hash": "16x2 levels, 2^19 f16 entries, N 16..2048",
                   "mlp": f"32-64-64-64-4 {a.mlp}", "residual_mlp": f"6 PE bands, width 64, {a.mlp}",
                   "mma_path": kernel_name,
                   "weight_volume": "64^3 x 25 f32", "ert_t_min": 1e-4, "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MiB write) between timed steps"},
        "samples_per_s": world * live * a.steps / (total_ms / 1000.0),
        "live_samples_per_frame": live,
        "stage_ms": {k: statistics.mean(st[k] for st in stages) for k in ("march_ms", "field_ms", "composite_ms")},
        "roofline": {"kernel": kernel_name + ": fused LBS warp + residual MLP + hash + canonical MLP",
                     "bound": "l2",
                     "achieved": requested["achieved"] if requested else achieved,
                     "peak": requested["peak"] if requested else ceiling["gbs"], "unit": "GB/s",
                     "frac": requested["frac"] if requested else achieved / ceiling["gbs"],
                     "basis": ("requested bytes: the bone channels the kernel reads (measured per frame), "
                               "the hash corners and the sample stream" if requested else "counted bytes"),
                     "peak_source": ("measured in this run: L2-resident random gathers (nr_l2_gather_rate) of "
                                     f"4 B at {ceiling['gather_4B_gbs']:.0f} GB/s and 16 B at "
                                     f"{ceiling['gather_16B_gbs']:.0f} GB/s, weighted by the kernel's "
                                     f"{ceiling['bytes_4B']} B of 4-byte and {ceiling['bytes_16B']} B of 16-byte "
                                     "gathers per live sample, its 32 B sample stream at the measured HBM rate"),
                     "counted": {"bytes_per_live_sample": bytes_per_sample, "achieved": achieved,
                                 "peak": ceiling["gbs"], "frac": achieved / ceiling["gbs"]},
                     "requested": requested,
                     "bytes_per_live_sample": {
                         "counted": bytes_per_sample,
                         "l1_sector_bytes": (cap["l1_sector_bytes_per_frame"] / cap["live_samples_per_frame"]
                                             if cap else None),
                         "l2_bytes": (cap["l2_bytes_per_frame"] / cap["live_samples_per_frame"] if cap else None),
                         "note": "counted: all 24 bone channels (768 B) + 16 hash levels (512 B) + sample in/out; "
                                 "the kernel skips bone channels whose support misses the candidate; every "
                                 "4-byte corner read touches a 32-byte L1 sector (l1_sector_bytes), of which "
                                 "l2_bytes miss L1 (ncu capture of these sources)"},
                     "vs_hbm": {"frac": achieved / hbm, "peak": hbm,
                                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"},
                     "traffic": cap["dram_bytes_per_frame"] if cap else None,
                     "traffic_note": ("dram__bytes_read.sum + dram__bytes_write.sum of the four field launches of "
                                      "one frame from the ncu capture of these kernel sources, per frame like "
                                      "'achieved'; null on another path or once the sources differ")},
        "roofline_mlp": ({"kernel": "the two MLPs of the same fused field kernel", "bound": "tensor",
                          "achieved": mlp_tflops, "unit": "TFLOP/s", "flops_per_live_sample": mlp_flops,
                          "peak": mlp_peak, "frac": mlp_tflops / mlp_peak,
                          "peak_sustained": mlp_peak_sus, "frac_sustained": mlp_tflops / mlp_peak_sus,
                          "peak_source": (("measured bf16 burst / sustained" if "bf16_tflops" in peaks
                                           else "fallback") + (" x 2 (nominal fp8 / bf16)" if ratio > 1 else "")),
                          "note": "algorithmic MLP flops over the whole field-kernel time: the gathers, not "
                                  "the tensor cores, bound this kernel"}
                         if a.mlp in ("bf16", "f16", "fp8") else None),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 24 * 12 * 4 + 24 * 3 * 4,
                "d2h_bytes_per_step": n_rays * 16},
        "train_step": train,
        "train_step_full_model": train_full,
        "occupancy_grid": occupancy,
        "serving": serving,
        "precision_sweep": sweep,
        "gpu_launches": launches,
        "clocks": clk,
        "paper_context": PAPER_CONTEXT,
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, poses, a.cpu_pixels)
    S.close()
    if rank == 0:
        print(json.dumps(line))


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
