"""Seeded synthetic inputs shared by the FP64 oracle, the CUDA path, the tests and the bench.

This package only *draws* inputs: Gaussian parameters on implicit surfaces, instance
transforms, pinhole cameras and MLP weights.  It holds none of the render pass's arithmetic
(no projection, no compositing, no encoding, no MLP evaluation), so the oracle and the CUDA
library can both consume it without sharing any of the method's code.
"""
from .synth import (  # noqa: F401
    Asset,
    Camera,
    Instance,
    Scene,
    MLP_LAYERS,
    look_at_camera,
    torus_asset,
    sphere_asset,
    box_asset,
    random_asset,
    mlp_weights,
    planar_mlp_weights,
    config1_scene,
    config1_camera,
    layered_scene,
    layered_camera,
    config2_scene,
    config2_camera,
    config2_orbit,
    config5_scene,
    config5_camera,
    tiny_scene,
    fibonacci_directions,
)
