"""Seeded synthetic inputs (no method arithmetic); see scenes.py."""
from .scenes import Camera, Scene, tiny_scene, room_scene, room_views, keyframe_batch, precision_scene, random_scene, random_unit_quats, building_gaussians, room_rgbd  # noqa: F401
from .masks import MaskSet, sam_masks, pixel_masks  # noqa: F401
