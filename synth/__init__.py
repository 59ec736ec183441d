"""Seeded synthetic road-scene stereo pairs (inputs only; no stereo arithmetic here)."""
from .road_pairs import (  # noqa: F401
    CONFIGS,
    SEED_BASE,
    RoadScene,
    make_scene,
    make_config_scene,
    make_batch_scenes,
    texture,
    crop_pair,
    make_roll_sequence,
    jitter,
)
