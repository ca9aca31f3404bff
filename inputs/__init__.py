"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package holds none of the method's arithmetic: it only draws the
potentials, strain fields, magnetic fields, material presets and random
vector blocks that both sides consume.
"""
from .gen import (  # noqa: F401
    MATERIALS,
    ROT_IDENTITY,
    ROT_DEVICE,
    Problem,
    config1,
    config2,
    config3,
    config4,
    config5,
    crop,
    double_dot,
    small_problem,
    random_block,
    smooth_noise,
)
