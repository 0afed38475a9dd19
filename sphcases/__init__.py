"""Seeded synthetic inputs shared by the oracle and the CUDA library (input data only)."""
from .dambreak import (RunParams, Case, dam_break, small_dam, wall_sensors, still_tank,
                       uniform_block, random_cloud, CONFIGS, G)

__all__ = ["RunParams", "Case", "dam_break", "small_dam", "wall_sensors", "still_tank",
           "uniform_block", "random_cloud", "CONFIGS", "G"]
