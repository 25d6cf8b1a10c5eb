"""Compulsory DRAM bytes of the benchmarked renders, counted by the oracle.

A render must read each parameter its evaluated samples interpolate (all 8
grid corners and 4 texels per plane of each sample) and each occupancy cell
its lattice tests consult at least once, and must write its pixels.  This
script counts those distinct parameters for one step of the two render
workloads -- the 8 oblique 1920x1080 cameras of the 512x512x32 city scene
(FP32 features) and the 4 oblique 3840x2160 cameras of the 1024x1024x64 city
scene (BF16 features) -- per camera and over the whole step, and prints the
bytes.  L2 is flushed between steps, not between the cameras of one step, so
the union over the step is the step's compulsory read.

    python oracle/working_set_bytes.py [--nthreads N]

Runs the oracle only (a few minutes on a few cores).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402

NCH = 8


def count(cfg: int, feat_bytes: int, nthreads: int) -> dict:
    sc = synth.make_scene(cfg)
    table = oracle.brick_table(sc["spec"], sc["occ"])
    pool = synth.fill_brick_pool(sc, table)
    osc = oracle.OracleScene(dict(sc, grid=pool, table=table))
    cams = synth.make_cameras(cfg)
    union = None
    per_cam = []
    rays_total = 0
    samples = 0
    for cam in cams:
        rays = oracle.camera_rays(cam)
        rays_total += rays.shape[0]
        ws = oracle.working_set(osc, rays, nthreads=nthreads)
        samples += ws["samples"]
        per_cam.append(_bytes(ws, feat_bytes, table))
        if union is None:
            union = {k: v.copy() for k, v in ws.items() if k != "samples"}
        else:
            for k in union:
                union[k] |= ws[k]
    step = _bytes(union, feat_bytes, table)
    return {"config": cfg, "rays": rays_total, "samples": samples, "per_camera": per_cam, "step": step,
            "pixels_written": rays_total * 12, "algorithmic_gather": samples * (20 * feat_bytes + 8)}


def _bytes(ws: dict, feat_bytes: int, table: np.ndarray) -> dict:
    texel = feat_bytes  # bytes of one vertex or texel (8 channels)
    g = int(ws["grid"].sum())
    bricks = int(np.any(ws["grid"].reshape(ws["grid"].shape[0], -1), axis=1).sum())
    planes = int(ws["p_xy"].sum() + ws["p_xz"].sum() + ws["p_yz"].sum())
    cells = int(ws["occ"].sum())
    return {"grid_vertices": g, "grid_bytes": g * texel, "bricks": bricks, "plane_texels": planes,
            "plane_bytes": planes * texel, "occ_cells": cells, "occ_bytes": cells * 8,
            "table_bytes": bricks * 4, "total": g * texel + planes * texel + cells * 8 + bricks * 4}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nthreads", type=int, default=0)
    args = ap.parse_args()
    for cfg, fb, name in ((2, 32, "8 x 1920x1080, 512x512x32 city, FP32"), (4, 16, "4 x 3840x2160, 1024x1024x64 "
                                                                                      "city, BF16")):
        r = count(cfg, fb, args.nthreads)
        s = r["step"]
        print(f"{name}: {r['rays']} rays, {r['samples']} evaluated samples")
        for i, c in enumerate(r["per_camera"]):
            print(f"  camera {i}: grid {c['grid_bytes'] / 1e6:.1f} MB ({c['bricks']} bricks), planes "
                  f"{c['plane_bytes'] / 1e6:.1f} MB, occupancy {c['occ_bytes'] / 1e6:.2f} MB, total "
                  f"{c['total'] / 1e6:.1f} MB")
        print(f"  step (union): grid {s['grid_bytes'] / 1e6:.1f} MB ({s['bricks']} bricks), planes "
              f"{s['plane_bytes'] / 1e6:.1f} MB, occupancy {s['occ_bytes'] / 1e6:.2f} MB, table "
              f"{s['table_bytes'] / 1e6:.3f} MB; compulsory read {s['total'] / 1e6:.1f} MB; pixels written "
              f"{r['pixels_written'] / 1e6:.1f} MB; algorithmic gather {r['algorithmic_gather'] / 1e9:.1f} GB")


if __name__ == "__main__":
    main()
