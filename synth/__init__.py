"""Seeded synthetic MWA-shaped cadences (inputs only; none of the peel's arithmetic)."""
from .generator import (  # noqa: F401
    Cadence, CONFIGS, config, splitmix64, uniform01, normals,
    baseline_pairs, n_baselines, noise_cube,
)
