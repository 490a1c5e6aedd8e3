"""Seeded synthetic inputs for the lifting path.

This package builds Gaussian sets, pinhole cameras, per-pixel segment-id maps
and per-segment embedding tables. It holds none of the method's arithmetic
(no projection, no compositing, no aggregation), so both the oracle and the
CUDA path may draw their inputs from it.
"""
from .scenes import (  # noqa: F401
    Gaussians, Camera, View, Scene,
    random_gaussians, ellipsoid_gaussians, orbit_camera, look_at, voronoi_segments, voronoi_from_seeds,
    prototype_table, make_scene, config_tiny, config_mid, config_precision,
    small_scene, segment_samples, config_batched, config_learned,
)
