"""Seeded synthetic inputs (meshes, animation, LiDAR rigs) shared by the CUDA
path's tests/bench and the CPU oracle.  Input data only: no ray-casting
arithmetic lives here."""
from .generate import (DT, Mesh, Scene, Sensor, box_mesh, channel_table, ellipsoid_mesh,
                       grid_mesh, make_config, make_sensor, noisy_sensor, ray_mask, ray_offsets,
                       rig_c4, rig_c5,
                       scene_c1, scene_c2, scene_c3, scene_c4, scene_c5, stress_set,
                       subsample_channels, tiny_scene)

__all__ = ["DT", "Mesh", "Scene", "Sensor", "box_mesh", "channel_table", "ellipsoid_mesh",
           "grid_mesh", "make_config", "make_sensor", "noisy_sensor", "ray_mask", "ray_offsets",
           "rig_c4", "rig_c5",
           "scene_c1", "scene_c2", "scene_c3", "scene_c4", "scene_c5", "stress_set",
           "subsample_channels", "tiny_scene"]
