"""Seeded synthetic inputs shared by the oracle tests and the CUDA path (no method arithmetic)."""
from .configs import (CONFIGS, FIELDS, Workload, config, linear_wave, random_modes, shock_tube,
                      shear_layer, lattice_positions, linear_mhd_modes, loss_weights, background)
from .rng import DEFAULT_SEED

__all__ = ["CONFIGS", "FIELDS", "Workload", "config", "linear_wave", "random_modes", "shock_tube",
           "shear_layer", "lattice_positions", "linear_mhd_modes", "loss_weights", "background",
           "DEFAULT_SEED"]
