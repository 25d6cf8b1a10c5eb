"""Seeded synthetic inputs for the Oblique-MERF hot path.

This package only draws scene content, cameras and training rays; it holds
none of the renderer's arithmetic (no interpolation, compositing, occupancy
ramp, MLP or ray/box logic).  Both the CUDA library's callers and the FP64
oracle's tests read its arrays.
"""
from .scene import (  # noqa: F401
    CONFIGS,
    MLP_NPARAM,
    NCH,
    SceneSpec,
    make_cameras,
    make_scene,
    make_train_batch,
    fill_brick_pool,
    perturb_scene,
    scene_spec,
    sparsity_points,
    entropy_rays,
    tiny_scene,
)
