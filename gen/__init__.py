"""Seeded synthetic hyperspectral inputs shared by the oracle and the CUDA path.

This package only *draws* inputs. It contains none of the RX arithmetic (no
means, covariances, factorisations or scores), so the oracle and the CUDA path
can both consume it without sharing any of the method's computation.
"""
from .cubes import (  # noqa: F401
    SEED_BASE,
    GaussianMixtureCube,
    IllConditionedScene,
    PushbroomScene,
    config1_cube,
    config_scene,
    serving_streams,
    stress_cubes,
    subsample_indices,
)
