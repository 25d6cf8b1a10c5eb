"""GB300 (sm_103a) Oblique-MERF hot path: Python binding of libomerf.so.

Argument marshalling only: every step of the render and training paths runs
in the CUDA kernels behind the C ABI declared in include/omerf.h.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the shared
library is missing or no GPU is present, calls raise.
"""
from .binding import (  # noqa: F401
    OmerfError,
    Scene,
    TrainStep,
    Trainer,
    adam_step,
    build_brick_table,
    camera_struct,
    check_counts,
    check_totals,
    crop_planes,
    entropy_loss,
    extract_bricks,
    grow_brick_table,
    lambda_occ,
    lib,
    lr_exponential,
    occupancy_grid,
    plane_crop_rows,
    probe_load_bandwidth,
    probe_red_bandwidth,
    scene_device_bytes,
    ray_interval,
    render,
    render_cameras,
    render_noalloc,
    saved_bytes_per_ray,
    scene_from_synth,
    sparsity_loss,
    sync,
    train_bwd,
    train_fwd,
    train_step,
    unpack_occupancy_bits,
    zero_grads,
)

__all__ = [
    "OmerfError", "Scene", "TrainStep", "Trainer", "adam_step", "build_brick_table", "camera_struct", "check_counts", "check_totals",
    "crop_planes", "entropy_loss", "extract_bricks", "grow_brick_table", "lambda_occ", "lib", "lr_exponential", "occupancy_grid",
    "plane_crop_rows", "probe_load_bandwidth", "probe_red_bandwidth", "scene_device_bytes", "ray_interval", "render", "render_cameras", "render_noalloc", "saved_bytes_per_ray", "scene_from_synth",
    "sparsity_loss", "sync", "train_bwd", "train_fwd", "train_step", "unpack_occupancy_bits", "zero_grads",
]
