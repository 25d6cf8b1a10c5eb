"""Benchmark of the Oblique-MERF hot path on GB300.

Default workload (one step): forward render of 8 oblique 1920x1080 cameras over
the sparse 512x512x32 city scene with 2048^2 / 2048x128 planes (FP32 features),
i.e. 16.6 M rays per step.  The same JSON line also reports one training step
(forward + backward, 2^18 rays on the 64x64x16 heightfield scene).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Timing: W untimed warm-up steps, then K timed steps; each camera render is
bracketed by CUDA events on the stream the kernels run on, and L2 is flushed
(a 256 MiB write) between steps outside the timed events.  Under torchrun each
rank renders its own cameras (weak scaling, no data exchange); rank 0 prints
one JSON line with the max time over ranks.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

BYTES_PER_SAMPLE = {"f32": 640 + 8, "bf16": 320 + 8}  # feature gather + occupancy bounds
BYTES_PER_RAY_RENDER = 12 + 4                          # rgb + count written
# Sources the dominant kernel (march_fwd_kernel<float, sparse, render>) is
# compiled from: a recorded DRAM traffic figure is valid only for the sources
# it was captured with.
RENDER_SOURCES = ("paper_2404_09531_gb300/csrc/march_fwd.cu", "paper_2404_09531_gb300/csrc/packed.cuh",
                  "paper_2404_09531_gb300/csrc/common.cuh", "paper_2404_09531_gb300/csrc/mlp_mma.cuh")
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of that kernel
# over the step's eight 1920x1080 cameras (one ncu capture), with the hash of
# the sources it was captured from.
TRAFFIC = {"sources_sha256_16": "03170e84b2575a5d", "bytes": 179789568.0 + 176725248.0}


def render_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in RENDER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_per_launch():
    """The recorded DRAM bytes per launch if the kernel's sources are the ones
    it was captured from, else None."""
    return TRAFFIC["bytes"] if render_sources_hash() == TRAFFIC["sources_sha256_16"] else None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1") or v == "1":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_cameras(rank: int):
    """Ray sharding across ranks: rank r renders its own 8 seeded oblique
    cameras of the same scene (rank 0 renders the default set), so per-rank
    work is fixed as ranks are added (weak scaling) and no rank needs another
    rank's data."""
    return synth.make_cameras(2) if rank == 0 else synth.make_cameras(2, seed=2 + 7919 * rank)


def max_over_ranks(value: float, device=None) -> float:
    """The slowest rank's step time (the job's time); identity on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _workload_config():
    spec = synth.scene_spec(2)
    return {"workload": "render 8 oblique cameras 1920x1080, sparse 512x512x32 grid (8^3 bricks, "
                        "15% allocated), planes 2048^2 / 2048x128, occupancy 256^2, step 1/2048, "
                        "n_max 512, FP32 features",
            "rays_per_step": spec.n_cams * spec.width * spec.height,
            "l2": "flushed between steps (256 MiB write)",
            "parallelism": "ray sharding: each rank renders its own 8 cameras, no data exchange",
            "train_workload": "fwd+bwd 2^18 rays, 64x64x16 grid, 256^2/256x32 planes, occupancy 32^2, "
                              "step 1/256, K=1 smoothness direction, FP32"}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores (bounded sample)
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle  # the oracle is this build's reference program

    sc = synth.make_scene(2)
    table = oracle.brick_table(sc["spec"], sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    osc = oracle.OracleScene(dict(sc, grid=pool, table=table))
    cams = synth.make_cameras(2)
    rays = np.concatenate([oracle.camera_rays(c) for c in cams])
    cores = os.cpu_count() or 1
    sample = rays[:: max(1, rays.shape[0] // 32768)]
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.render(osc, sample, nthreads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = sample.shape[0] / t / 1e6
    cfg = _workload_config()
    line = {"metric": "Mrays/s render & fwd+bwd train, BF16 vs FP32 at matched PSNR vs FP64 oracle",
            "impl": "reference", "value": value, "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample.shape[0]} rays, every {rays.shape[0] // sample.shape[0]}th "
                                       f"ray of the 8 cameras"},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(sc, cams, budget_s=12.0):
    """The oracle, as it stands, on a bounded sample of the same workload."""
    import oracle

    table = oracle.brick_table(sc["spec"], sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    osc = oracle.OracleScene(dict(sc, grid=pool, table=table))
    rays = np.concatenate([oracle.camera_rays(c) for c in cams])
    cores = os.cpu_count() or 1
    probe = rays[:: max(1, rays.shape[0] // 4096)]
    t0 = time.perf_counter()
    oracle.render(osc, probe, nthreads=cores)
    per_ray = (time.perf_counter() - t0) / probe.shape[0]
    n = int(min(rays.shape[0], max(4096, budget_s / max(per_ray, 1e-9))))
    stride = max(1, rays.shape[0] // n)
    sample = rays[::stride]
    t0 = time.perf_counter()
    ref = oracle.render(osc, sample, nthreads=cores)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on a sample a sixth of the CPU time
    n1 = int(min(rays.shape[0], max(1024, budget_s / 6.0 / max(per_ray * cores, 1e-9))))
    sample1 = rays[:: max(1, rays.shape[0] // n1)]
    t0 = time.perf_counter()
    oracle.render(osc, sample1, nthreads=1)
    dt1 = time.perf_counter() - t0
    out = {"value": sample.shape[0] / dt / 1e6, "unit": "Mrays/s", "cores": cores, "kind": "oracle",
           "sample": f"{sample.shape[0]} rays (every {stride}th ray of the 8 cameras), {dt:.1f} s",
           "one_thread": {"value": sample1.shape[0] / dt1 / 1e6, "unit": "Mrays/s", "cores": 1,
                          "sample": f"{sample1.shape[0]} rays (strided over the 8 cameras), {dt1:.1f} s"},
           "render_4k": _oracle_render_4k(cores), "train": _oracle_train()}
    return out, ref, stride


def _oracle_render_4k(cores, n=1 << 18):
    """The oracle on a strided 2^18-pixel sample of the four 3840x2160 cameras
    (FP32-valued features of the 1024x1024x64 city scene)."""
    import oracle

    sc = synth.make_scene(4)
    table = oracle.brick_table(sc["spec"], sc["occ"])
    osc = oracle.OracleScene(dict(sc, grid=synth.fill_brick_pool(sc, table), table=table))
    rays = np.concatenate([oracle.camera_rays(c) for c in synth.make_cameras(4)])
    sample = rays[:: rays.shape[0] // n]
    t0 = time.perf_counter()
    oracle.render(osc, sample, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample.shape[0] / dt / 1e6, "unit": "Mrays/s", "cores": cores,
            "sample": f"{sample.shape[0]} rays strided over the 4 cameras, {dt:.1f} s"}


def _oracle_train(n=1 << 15):
    """The oracle's loss and analytic gradient (one thread: it sums into one
    set of gradient arrays) on 2^15 rays of the 2^18-ray training batch."""
    import oracle

    sc = synth.make_scene(3)
    b = synth.make_train_batch(3, 1 << 18)
    sl = slice(0, 1 << 18, (1 << 18) // n)
    t0 = time.perf_counter()
    oracle.train(oracle.OracleScene(sc), b["rays"][sl], b["target"][sl], b["smooth_dirs"][sl], lam=(1.0, 1e-2, 1e-4))
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e6, "unit": "Mrays/s fwd+bwd", "cores": 1,
            "sample": f"{n} rays strided over the 2^18-ray batch, {dt:.1f} s"}


def _render_errors(rgb, count, ref):
    """Error of GPU pixels against the FP64 oracle on the same rays: max-abs
    and PSNR over rays the oracle does not flag as ambiguous at the
    termination threshold, and the sample-count mismatches there."""
    rgb = np.asarray(rgb, np.float64)
    ok = ref["ambiguous"] == 0
    err = np.abs(rgb[ok] - ref["rgb"][ok])
    mse = float(np.mean(err ** 2)) if err.size else 0.0
    out = {"rays": int(ok.size), "ambiguous": int((~ok).sum()), "max_abs": float(err.max(initial=0.0)),
           "psnr_db": 10.0 * float(np.log10(1.0 / mse)) if mse > 0 else float("inf")}
    if count is not None:
        out["count_mismatch"] = int((np.asarray(count)[ok] != ref["count"][ok]).sum())
    return out


def _grad_errors(res, ref):
    """Per tensor ||g_gpu - g_ref|| / ||g_ref|| against the oracle's analytic
    gradient, the worst of them, and the loss's relative error."""
    errs = {}
    for k in ("grid", "p_xy", "p_xz", "p_yz", "occ", "mlp"):
        a = res["grads"][k].double().cpu().numpy().reshape(-1)
        b = np.asarray(ref["grads"][k], np.float64).reshape(-1)
        nb = np.linalg.norm(b)
        errs[k] = float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))
    loss = float(res["loss"][0].item())
    return {"grad_rel": errs, "grad_rel_max": max(errs.values()),
            "loss_rel": abs(loss - ref["loss"]) / max(abs(ref["loss"]), 1e-30)}


def oracle_errors_precision(om, torch, dev, n_render=1 << 16, n_train=8192):
    """Every precision result against the FP64 oracle (this runs the oracle,
    so it belongs to the CPU-baseline leg): the 4 x 3840x2160 render in BF16
    and FP32 on a strided n_render-pixel sample (BF16 also against the oracle
    on the BF16-rounded features, which isolates the arithmetic), and the
    training gradients on an n_train-ray slice of each benchmarked batch."""
    import oracle

    rb = lambda a: torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()  # noqa: E731
    out = {}
    sc = synth.make_scene(4)
    table = oracle.brick_table(sc["spec"], sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    cams = synth.make_cameras(4)
    rays = np.concatenate([oracle.camera_rays(c) for c in cams])
    stride = rays.shape[0] // n_render
    ref = oracle.render(oracle.OracleScene(dict(sc, grid=pool, table=table)), rays[::stride])
    sc_b = dict(sc, grid=rb(pool), table=table, p_xy=rb(sc["p_xy"]), p_xz=rb(sc["p_xz"]), p_yz=rb(sc["p_yz"]))
    ref_b = oracle.render(oracle.OracleScene(sc_b), rays[::stride])
    for name, dt in (("bf16", torch.bfloat16), ("f32", torch.float32)):
        scene = om.scene_from_synth(sc, device=dev, table=table, feat_dtype=dt)
        rgb, cnt = om.render_cameras(scene, cams)
        rgb, cnt = rgb[::stride].cpu().numpy(), cnt[::stride].cpu().numpy()
        out[f"render_{name}"] = _render_errors(rgb, cnt, ref)
        if name == "bf16":
            out["render_bf16_vs_bf16_features"] = _render_errors(rgb, cnt, ref_b)
        del scene
    out["render_sample"] = f"every {stride}th pixel of the 4 cameras ({rays[::stride].shape[0]} rays)"
    lam = (1.0, 1e-2, 1e-4)
    # config 3 (FP32), oracle-rendered targets of the perturbed features
    tsc = synth.make_scene(3)
    b = synth.make_train_batch(3, 1 << 18)
    sl = slice(0, n_train)
    tgt = oracle.render(oracle.OracleScene(synth.perturb_scene(tsc)), b["rays"][sl])["rgb"].astype(np.float32)
    scene = om.scene_from_synth(tsc, device=dev)
    res = om.train_step(scene, b["rays"][sl], tgt, b["smooth_dirs"][sl], lam=lam)
    out["train_f32"] = _grad_errors(res, oracle.train(oracle.OracleScene(tsc), b["rays"][sl], tgt,
                                                      b["smooth_dirs"][sl], lam=lam))
    # the 2^20-ray workloads: BF16 features against the oracle on the rounded
    # features, and the city scene's sizes in FP32
    sc5 = synth.make_scene(5)
    b5 = synth.make_train_batch(5, 1 << 20)
    scene = om.scene_from_synth(sc5, device=dev, feat_dtype=torch.bfloat16)
    res = om.train_step(scene, b5["rays"][sl], b5["target"][sl], b5["smooth_dirs"][sl], lam=lam)
    sc5b = dict(sc5, grid=rb(sc5["grid"]), p_xy=rb(sc5["p_xy"]), p_xz=rb(sc5["p_xz"]), p_yz=rb(sc5["p_yz"]))
    out["train_bf16_vs_bf16_features"] = _grad_errors(res, oracle.train(oracle.OracleScene(sc5b), b5["rays"][sl],
                                                                         b5["target"][sl], b5["smooth_dirs"][sl],
                                                                         lam=lam))
    spec = dataclasses.replace(synth.scene_spec(2), n_cams=64)
    city = synth.make_scene(spec)
    ctable = oracle.brick_table(spec, city["occ"])
    cpool = synth.fill_brick_pool(city, ctable)
    bc = synth.make_train_batch(spec, 1 << 20)
    sl = slice(0, n_train // 2)
    scene = om.scene_from_synth(city, device=dev, table=ctable)
    res = om.train_step(scene, bc["rays"][sl], bc["target"][sl], bc["smooth_dirs"][sl], lam=lam)
    out["train_city_f32"] = _grad_errors(res, oracle.train(oracle.OracleScene(dict(city, grid=cpool, table=ctable)),
                                                           bc["rays"][sl], bc["target"][sl], bc["smooth_dirs"][sl],
                                                           lam=lam))
    out["train_sample"] = f"the first {n_train} rays of each batch ({n_train // 2} for the city scene)"
    return out


# ---------------------------------------------------------------------------
# secondary workloads reported in the same line: BF16 vs FP32
# ---------------------------------------------------------------------------
def _time_renders(om, torch, scene, cams, steps, warmup, flush, stream):
    n = sum(c["width"] * c["height"] for c in cams)
    out = torch.empty((n, 3), dtype=torch.float32, device=scene.device)
    for _ in range(warmup):
        om.render_cameras(scene, cams, out=out, want_count=False)
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        om.render_cameras(scene, cams, out=out, want_count=False)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.mean(ms))


def bench_precision_render(om, torch, dev, steps, warmup, flush, stream):
    """3840x2160 x 4 cameras, BF16 features + tensor-core MLP vs FP32 features,
    same scene; PSNR of the BF16 frames against the FP32 frames."""
    sc = synth.make_scene(4)
    spec = sc["spec"]
    occ = torch.as_tensor(sc["occ"]).to(dev)
    table = om.build_brick_table(spec.aabb, spec.L, spec.brick, occ)[0].cpu().numpy()
    cams = synth.make_cameras(4)
    rays = sum(c["width"] * c["height"] for c in cams)
    out = {"workload": "render 4 oblique cameras 3840x2160, sparse 1024x1024x64 grid (8^3 bricks, 9.6% "
                       "allocated), planes 4096^2 / 4096x256, occupancy 512^2, step 1/2048",
           "rays_per_step": rays}
    frames = {}
    for name, dt in (("bf16", torch.bfloat16), ("f32", torch.float32)):
        scene = om.scene_from_synth(sc, device=dev, table=table, feat_dtype=dt)
        t = _time_renders(om, torch, scene, cams, steps, warmup, flush, stream)
        frames[name] = om.render(scene, camera=cams[0])[0]
        out[name] = {"value": rays / (t * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": t}
        del scene
    mse = float(((frames["bf16"] - frames["f32"]) ** 2).mean().item())
    out["psnr_bf16_vs_f32_db"] = 10.0 * np.log10(1.0 / mse) if mse > 0 else float("inf")
    out["speedup_bf16_over_f32"] = out["bf16"]["value"] / out["f32"]["value"]
    return out


def _time_train(om, torch, scene, batch_d, lam, steps, warmup, flush, stream):
    """Mean event time (ms) of one fused training step (fwd + bwd) on a batch
    resident on the device; gradients zeroed and L2 flushed outside the events."""
    rays_d, tgt_d, dirs_d = batch_d
    n = rays_d.shape[0]
    grads = om.zero_grads(scene)
    saved = torch.empty(n * om.saved_bytes_per_ray() // 4, dtype=torch.float32, device=rays_d.device)
    for _ in range(warmup):
        om.train_step(scene, rays_d, tgt_d, dirs_d, lam=lam, grads=grads, saved=saved)
    ms = []
    for _ in range(steps):
        flush.fill_(1.0)
        for gt in grads.values():
            gt.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        om.train_step(scene, rays_d, tgt_d, dirs_d, lam=lam, grads=grads, saved=saved)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    del grads, saved
    return float(np.mean(ms))


def _train_precisions(om, torch, dev, sc, batch, steps, warmup, flush, stream, table=None):
    """BF16 vs FP32 features of one training workload: Mrays/s, feature bytes
    and the peak of torch's device allocations (features, FP32 gradients,
    batch, saved state)."""
    n_rays = batch["rays"].shape[0]
    batch_d = tuple(torch.as_tensor(batch[k]).to(dev) for k in ("rays", "target", "smooth_dirs"))
    batch_bytes = sum(x.numel() * x.element_size() for x in batch_d)
    lam = (1.0, 1e-2, 1e-4)
    out = {}
    for name, dt in (("bf16", torch.bfloat16), ("f32", torch.float32)):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats(dev)
        base = torch.cuda.memory_allocated(dev)
        scene = om.scene_from_synth(sc, device=dev, feat_dtype=dt, table=table)
        t = _time_train(om, torch, scene, batch_d, lam, steps, warmup, flush, stream)
        feat_bytes = sum(x.numel() * x.element_size() for x in (scene.grid, scene.p_xy, scene.p_xz, scene.p_yz))
        out[name] = {"value": n_rays / (t * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": t,
                     "feature_bytes": feat_bytes,
                     "peak_device_bytes": int(torch.cuda.max_memory_allocated(dev) - base) + batch_bytes}
        del scene
    return out


def bench_precision_train(om, torch, dev, steps, warmup, flush, stream, n_rays=1 << 20):
    """Training fwd+bwd on 2^20 rays of 64 cameras, BF16 features (FP32 gradients)
    vs FP32 features: on the 64x64x16 heightfield scene (the literal sizes)
    and at the city scene's sizes (512x512x32 brick grid, 2048^2 planes)."""
    sc = synth.make_scene(5)
    out = {"workload": "fwd+bwd 2^20 rays of 64 cameras, 64x64x16 grid, 256^2/256x32 planes, K=1",
           "rays_per_step": n_rays,
           "peak_device_bytes_note": "the workload's own peak device allocations: scene (features, occupancy, "
                                     "MLP, brick table), FP32 gradients, saved state and the batch (rays, "
                                     "targets, smoothness directions)"}
    out.update(_train_precisions(om, torch, dev, sc, synth.make_train_batch(5, n_rays), steps, warmup, flush,
                                 stream))
    spec = dataclasses.replace(synth.scene_spec(2), n_cams=64)
    city = synth.make_scene(spec)
    occ = torch.as_tensor(city["occ"]).to(dev)
    table = om.build_brick_table(spec.aabb, spec.L, spec.brick, occ)[0].cpu().numpy()
    out["city"] = {"workload": "fwd+bwd 2^20 rays of 64 oblique 1920x1080 cameras, sparse 512x512x32 grid "
                               "(8^3 bricks), planes 2048^2 / 2048x128, occupancy 256^2, step 1/2048, K=1",
                   "rays_per_step": n_rays}
    out["city"].update(_train_precisions(om, torch, dev, city, synth.make_train_batch(spec, n_rays), steps, warmup,
                                         flush, stream, table=table))
    return out


def measure_load_peaks(om, torch, dev, stream):
    """Load bandwidth (bytes delivered to registers per second) of the
    gather's 256-bit read-only load, measured with omerf_probe_load_bandwidth
    in the march's launch shape (3 CTAs of 256 threads per SM): from L1
    (a 16 KB slice per CTA, re-read 4000 times) and from L2 (a 160 KB slice
    per CTA: 480 KB per SM, beyond L1; 73 MB in all, inside L2); and the
    rate of the re-march scatter's vector reductions
    (omerf_probe_red_bandwidth).  Best of 5 after 3 warm-up launches, CUDA
    events on the launching stream."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    ctas = 3 * sms
    out = {}
    for name, per_cta, passes in (("l1", 16384, 4000), ("l2", 163840, 100)):
        buf = torch.rand(ctas * per_cta // 4, device=dev)
        sink = torch.empty(ctas * 256, dtype=torch.float32, device=dev)
        for _ in range(3):
            om.probe_load_bandwidth(buf, per_cta, ctas, passes, sink)
        best = float("inf")
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nbytes = om.probe_load_bandwidth(buf, per_cta, ctas, passes, sink)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        out[name] = {"gbs": nbytes / (best * 1e-3) / 1e9, "ms": best, "ctas": ctas, "bytes_per_cta": per_cta,
                     "passes": passes}
        del buf, sink
    # the re-march's gradient scatter: 16-byte vector FP32 reductions, each
    # lane on its own 128-byte line, in the re-march's launch shape (2 CTAs
    # of 256 threads per SM) and with twice the warps; 16 KB per warp (40 or
    # 80 MB in all, inside L2)
    for name, per_sm, passes in (("red", 2, 256), ("red_4ctas", 4, 128)):
        rctas, per_warp = per_sm * sms, 16384
        buf = torch.zeros(rctas * 8 * per_warp // 4, device=dev)
        for _ in range(3):
            om.probe_red_bandwidth(buf, per_warp, rctas, passes)
        best = float("inf")
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            nbytes = om.probe_red_bandwidth(buf, per_warp, rctas, passes)
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        out[name] = {"gbs": nbytes / (best * 1e-3) / 1e9, "ms": best, "ctas": rctas, "bytes_per_warp": per_warp,
                     "passes": passes, "note": "red.global.add.v4.f32, 16 B per lane, every lane its own line"}
        del buf
    return out


# ---------------------------------------------------------------------------
# native arm
# ---------------------------------------------------------------------------
def bench_extraction(om, torch, scene, steps, warmup, flush, stream, N=(2048, 2048, 128)):
    """Extraction after training (Sec. 4.4, Sec. 5.3) on the city scene, each
    stage timed with events: the 3D occupancy grid at the paper's largest
    resolution, the brick table and a pool re-extraction from the current
    pool, and the XZ/YZ plane crop (rows + copy)."""
    st = {"grid": [], "bricks": [], "crop": [], "dense": []}
    bits = count = None
    # a dense grid of the scene's size to extract bricks from (tiled TMA copies)
    dense = torch.randn((*scene.grid_res, 8), dtype=torch.float32, device=scene.grid.device)
    for it in range(warmup + steps):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        bits, count = om.occupancy_grid(scene.aabb, scene.occ, N)
        ev[1].record(stream)
        table, n_alloc = om.build_brick_table(scene.aabb, scene.grid_res, scene.brick, scene.occ)
        pool = om.extract_bricks(scene.grid_res, scene.brick, table, scene.grid, src_table=scene.table,
                                 n_bricks=int(scene.grid.shape[0]))
        ev[2].record(stream)
        cropped = om.crop_planes(scene)
        ev[3].record(stream)
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record(stream)
        pool2 = om.extract_bricks(scene.grid_res, scene.brick, scene.table, dense, n_bricks=int(scene.grid.shape[0]))
        e5.record(stream)
        torch.cuda.synchronize()
        if it >= warmup:
            st["grid"].append(ev[0].elapsed_time(ev[1]))
            st["bricks"].append(ev[1].elapsed_time(ev[2]))
            st["crop"].append(ev[2].elapsed_time(ev[3]))
            st["dense"].append(e4.elapsed_time(e5))
        del pool, cropped, pool2
    voxels = N[0] * N[1] * N[2]
    ms = {k: float(np.mean(v)) for k, v in st.items()}
    return {"occupancy_grid": {"ms": ms["grid"], "voxels": voxels, "resolution": list(N),
                               "occupancy_ratio": int(count.item()) / voxels},
            "bricks": {"ms": ms["bricks"], "n_bricks": int(scene.grid.shape[0]),
                       "note": "table from the occupancy plane + pool re-extraction from the current pool"},
            "plane_crop": {"ms": ms["crop"], "note": "crop rows (one 8-byte readback) + XZ/YZ row copy"},
            "bricks_from_dense": {"ms": ms["dense"], "tma": bool(om.lib().omerf_tma_available()),
                                  "gbs": 2 * int(scene.grid.shape[0]) * scene.brick ** 3 * 32 / (ms["dense"] * 1e-3) / 1e9,
                                  "note": "pool of the scene's table from a dense FP32 grid of its size: tiled "
                                          "tensor-memory-accelerator box loads + bulk stores (read + write bytes)"},
            "total_ms": ms["grid"] + ms["bricks"] + ms["crop"],
            "paper": "extracting the occupancy grid takes 2 to 10 minutes in the paper (Sec. 5.3)"}


def run_native(args):
    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    import paper_2404_09531_gb300 as om

    # ---- scene (config 2) ----
    sc = synth.make_scene(2)
    spec = sc["spec"]
    occ = torch.as_tensor(sc["occ"]).to(dev)
    table_t, _ = om.build_brick_table(spec.aabb, spec.L, spec.brick, occ)
    table = table_t.cpu().numpy()
    scene = om.scene_from_synth(sc, device=dev, table=table)
    cams = rank_cameras(rank)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    rays_per_step = sum(c["width"] * c["height"] for c in cams)
    dev_rgb = torch.empty((rays_per_step, 3), dtype=torch.float32, device=dev)

    def step(events=None):
        # the step's cameras in one persistent launch
        if events is not None:
            events[0][0].record(stream)
        om.render_cameras(scene, cams, out=dev_rgb, want_count=False)
        if events is not None:
            events[0][1].record(stream)
        return dev_rgb

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rgb0, cnt0 = om.render(scene, camera=cams[0])
    samples_per_step = 0
    for cam in cams:
        _, c = om.render(scene, camera=cam)
        samples_per_step += int(c.sum().item())

    clocks = ClockSampler(None)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    per_launch = []
    step_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))]
        step(ev)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        per_launch += ms
        step_ms.append(sum(ms))
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_step = max_over_ranks(float(np.mean(step_ms)), dev)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    value = ws * rays_per_step / (t_step * 1e-3) / 1e6

    # ---- end to end through the public API, host buffers ----
    host_rgb = torch.empty((rays_per_step, 3), dtype=torch.float32, pin_memory=True)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        om.render_cameras(scene, cams, out=host_rgb, want_count=False)
        b.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    e2e_step = float(np.mean(e2e_ms))
    d2h = host_rgb.numel() * 4
    h2d = 64 * len(cams)  # camera structs (the step's only input)

    # ---- training step (config 3) ----
    tsc = synth.make_scene(3)
    tscene = om.scene_from_synth(tsc, device=dev)
    batch = synth.make_train_batch(3, 1 << 18)
    target, _ = om.render(om.scene_from_synth(synth.perturb_scene(tsc), device=dev), rays=batch["rays"])
    rays_d = torch.as_tensor(batch["rays"]).to(dev)
    dirs_d = torch.as_tensor(batch["smooth_dirs"]).to(dev)
    grads = om.zero_grads(tscene)
    saved = torch.empty((1 << 18) * om.saved_bytes_per_ray() // 4, dtype=torch.float32, device=dev)
    lam = (1.0, 1e-2, 1e-4)
    for _ in range(args.warmup):
        om.train_step(tscene, rays_d, target, dirs_d, lam=lam, grads=grads, saved=saved)
    tr_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        for g in grads.values():
            g.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        res = om.train_step(tscene, rays_d, target, dirs_d, lam=lam, grads=grads, saved=saved)
        b.record(stream)
        torch.cuda.synchronize()
        tr_ms.append(a.elapsed_time(b))
    t_train = float(np.mean(tr_ms))
    loss = res["loss"].cpu().numpy().tolist()
    # the same step with the deferred-MLP backward on tcgen05 tensor cores
    # (the alternative the library selects with OMERF_MLP_BWD=tcgen05)
    os.environ["OMERF_MLP_BWD"] = "tcgen05"
    tc_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        for g in grads.values():
            g.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        om.train_step(tscene, rays_d, target, dirs_d, lam=lam, grads=grads, saved=saved)
        b.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            tc_ms.append(a.elapsed_time(b))
    del os.environ["OMERF_MLP_BWD"]
    t_train_tc = float(np.mean(tc_ms))
    dp_train = None
    if ws > 1:
        # ray-sharded data parallelism (weak scaling): a global batch of ws x
        # 2^18 rays, each rank's shard its own 2^18 rays, one all-reduce of
        # the gradients and loss inside the timed step
        from paper_2404_09531_gb300 import data_parallel as dpm
        g_rays = torch.cat([torch.as_tensor(synth.make_train_batch(3, 1 << 18, seed=3 + 7919 * r)["rays"])
                            for r in range(ws)]).to(dev)
        g_tgt = torch.cat([target] * ws)
        g_dirs = torch.cat([dirs_d] * ws)
        dstep = dpm.DataParallelStep({k: tuple(getattr(tscene, k).shape) for k in dpm.GRAD_KEYS}, dev)
        for _ in range(args.warmup):
            dstep(tscene, g_rays, g_tgt, g_dirs, lam, saved=saved)
        dp_ms = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            import torch.distributed as dist
            dist.barrier()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dstep(tscene, g_rays, g_tgt, g_dirs, lam, saved=saved)
            b.record(stream)
            torch.cuda.synchronize()
            dp_ms.append(a.elapsed_time(b))
        t_dp = max_over_ranks(float(np.mean(dp_ms)), dev)
        dp_train = {"value": ws * (1 << 18) / (t_dp * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": t_dp,
                    "global_batch": ws * (1 << 18), "scaling": "weak",
                    "note": "ray-sharded fwd+bwd, one NCCL all-reduce of gradients + loss per step, max over ranks"}

    # the full optimisation step of appendix A: fwd + bwd, fused Adam over
    # features, occupancy plane and MLP (one launch), hull update
    # (with the paper's regulariser batches: 2^14 sparsity points, 2^10 entropy rays)
    pts_d = torch.as_tensor(synth.sparsity_points(tsc, 1 << 14)).to(dev)
    erays_d = torch.as_tensor(synth.entropy_rays(tsc, 1 << 10)).to(dev)
    reg_grads = om.zero_grads(tscene)
    reg_loss = torch.zeros(1, dtype=torch.float32, device=dev)
    sp_ms, en_ms = [], []
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        a.record(stream)
        om.sparsity_loss(tscene, pts_d, lam=0.05, grads=reg_grads, loss=reg_loss)
        b.record(stream)
        om.entropy_loss(tscene, erays_d, lam=1e-3, grads=reg_grads, loss=reg_loss)
        c.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            sp_ms.append(a.elapsed_time(b))
            en_ms.append(b.elapsed_time(c))
    trainer = om.Trainer(tscene, total_steps=80000, lam_occ=1e-4)
    for _ in range(args.warmup):
        trainer.step(rays_d, target, dirs_d, sparsity_points=pts_d, entropy_rays=erays_d)
    loop_ms, adam_ms = [], []
    groups = [{"param": p.view(-1), "grad": trainer.grads[k].view(-1), "m": trainer.moments[k][0].view(-1),
               "v": trainer.moments[k][1].view(-1), "lr": 1e-3} for k, p in trainer.master.items()]
    n_params = sum(gr["param"].numel() for gr in groups)
    for _ in range(args.steps):
        flush.fill_(1.0)
        a, b, c, e = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        a.record(stream)
        trainer.step(rays_d, target, dirs_d, sparsity_points=pts_d, entropy_rays=erays_d)
        b.record(stream)
        c.record(stream)
        om.adam_step(groups, 1000)
        e.record(stream)
        torch.cuda.synchronize()
        loop_ms.append(a.elapsed_time(b))
        adam_ms.append(c.elapsed_time(e))
    t_loop, t_adam = float(np.mean(loop_ms)), float(np.mean(adam_ms))

    extraction = bench_extraction(om, torch, scene, max(1, min(args.steps, 5)), args.warmup, flush, stream)
    peaks = measure_load_peaks(om, torch, dev, stream)

    precision = None
    if not args.no_precision:
        psteps = max(1, min(args.steps, 5))
        precision = {"render": bench_precision_render(om, torch, dev, psteps, args.warmup, flush, stream),
                     "train": bench_precision_train(om, torch, dev, psteps, args.warmup, flush, stream)}

    if rank != 0:
        return 0

    hbm, peak_kind = _peaks()
    t_launch = float(np.mean(per_launch)) * 1e-3
    bytes_launch = samples_per_step * BYTES_PER_SAMPLE["f32"] + rays_per_step * BYTES_PER_RAY_RENDER
    achieved = bytes_launch / t_launch / 1e9
    l1, l2 = peaks["l1"]["gbs"], peaks["l2"]["gbs"]
    cfg = _workload_config()
    cfg["samples_per_step"] = samples_per_step
    cfg["mean_samples_per_ray"] = samples_per_step / rays_per_step
    line = {
        "metric": "Mrays/s render & fwd+bwd train, BF16 vs FP32 at matched PSNR vs FP64 oracle",
        "value": value, "unit": "Mrays/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded oblique city scene; paper datasets unavailable)",
        "config": cfg,
        "msamples_per_s": ws * samples_per_step / (t_step * 1e-3) / 1e6,
        "roofline": {"bound": "l1", "achieved": achieved, "peak": l1, "unit": "GB/s", "frac": achieved / l1,
                     "traffic": traffic_per_launch(),
                     "kernel": "march_fwd_kernel<float, sparse, render>",
                     "peak_kind": "measured in this run: L1 load bandwidth of the gather's 256-bit read-only load "
                                  "(omerf_probe_load_bandwidth, 3 x 256-thread CTAs per SM, 16 KB slice each)",
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "algorithmic_bytes": "648 B per evaluated sample (8 grid corners + 12 plane texels x 32 B, "
                                          "+ 8 B occupancy bounds) + 16 B per ray written",
                     "l2": {"peak": l2, "frac": achieved / l2, "peak_kind": "measured in this run: the same "
                            "probe, a 160 KB slice per CTA (beyond L1, inside L2)"},
                     "hbm": {"peak": hbm, "frac": achieved / hbm, "peak_kind": f"{peak_kind} HBM copy bandwidth",
                             "traffic_frac": (traffic_per_launch() / t_launch / 1e9 / hbm)
                             if traffic_per_launch() else None},
                     "probes": peaks,
                     "note": "the gather is served from L1 (92 % hits) and L2 (94-97 %): the algorithmic bytes "
                             "are bytes delivered to registers, bounded by L1's load bandwidth; DRAM moves only "
                             "each frame's working set (traffic: null when the kernel's sources differ from "
                             "those of the recorded ncu capture)"},
        "e2e": {"value": ws * rays_per_step / (e2e_step * 1e-3) / 1e6, "unit": "Mrays/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_step},
        "train": {"metric": "Mrays/s fwd+bwd train", "value": (1 << 18) / (t_train * 1e-3) / 1e6,
                  "unit": "Mrays/s", "ms_per_step": t_train, "rays_per_step": 1 << 18, "loss": loss,
                  "mlp_bwd_tcgen05": {"value": (1 << 18) / (t_train_tc * 1e-3) / 1e6, "unit": "Mrays/s",
                                      "ms_per_step": t_train_tc,
                                      "note": "the same fused step with the deferred-MLP backward as tcgen05 "
                                              "products (128-ray tiles, TMEM accumulators): slower than the "
                                              "default warp-level form, which the line's value uses"},
                  "with_adam": {"value": (1 << 18) / (t_loop * 1e-3) / 1e6, "unit": "Mrays/s",
                                "ms_per_step": t_loop,
                                "note": "fwd + bwd + sparsity and entropy terms + fused Adam (lr decay, "
                                        "lambda_7 fixed at 1e-4) + hull update; the scene evolves under the "
                                        "optimiser, so its sample counts differ from the fwd+bwd line"},
                  "regularizers": {"sparsity_us": float(np.mean(sp_ms)) * 1e3, "points": 1 << 14,
                                   "entropy_us": float(np.mean(en_ms)) * 1e3, "rays": 1 << 10,
                                   "note": "Eqs. 13-14, loss + gradient, one launch each"},
                  "data_parallel": dp_train,
                  "adam": {"us": t_adam * 1e3, "params": n_params,
                           "achieved_gbs": 28.0 * n_params / (t_adam * 1e-3) / 1e9,
                           "note": "28 B per parameter (read p, g, m, v; write p, m, v)"}},
        "extraction": extraction,
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        # the oracle's timing, and its outputs on the same samples: every
        # result's error against FP64
        line["cpu_baseline"], ref, stride = cpu_baseline_sample(sc, cams)
        rgb_all, cnt_all = om.render_cameras(scene, cams)
        line["error_vs_oracle"] = _render_errors(rgb_all[::stride].cpu().numpy(), cnt_all[::stride].cpu().numpy(),
                                                 ref)
        line["error_vs_oracle"]["sample"] = line["cpu_baseline"]["sample"]
        del rgb_all, cnt_all
        if precision is not None:
            precision["vs_oracle"] = oracle_errors_precision(om, torch, dev)
    if precision is not None:
        line["precision"] = precision
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the BF16 vs FP32 workloads")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
