"""Seeded synthetic inputs for the hybrid depth-of-field pass.

This package produces the *inputs* that both the FP64 oracle (``oracle/``) and the
CUDA library consume: procedural triangle scenes, thin-lens camera poses along a
dolly path, and the per-workload parameter presets.  It holds none of the method's
arithmetic (no circle of confusion, no filters, no ray tracing): it only places
triangles and cameras from a SplitMix64 stream, so that both sides are fed exactly
the same float32 values.

The paper's scenes (Pink Room, Sun Temple, Bistro; Section 4.2) are not available;
the generators here stand in for them with scenes of the same character: thin,
partially occluding foreground geometry in front of a far field.
"""

from .rng import SplitMix64
from .scenes import (Scene, Camera, Workload, camera_pose, make_workload,
                     scene_c1, scene_grass_field, tiny_scene, plane_scene,
                     WORKLOADS)

__all__ = ["SplitMix64", "Scene", "Camera", "Workload", "camera_pose",
           "make_workload", "scene_c1", "scene_grass_field", "tiny_scene",
           "plane_scene", "WORKLOADS"]
