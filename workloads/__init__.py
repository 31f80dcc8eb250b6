"""Seeded synthetic inputs for the sputter-transport hot path.

This package describes *workloads* only: chamber boxes, surface primitives,
cathode poses, element constants and process conditions.  It holds none of
the transport arithmetic (no sampling, no cross sections, no kinematics), so
both the CUDA path and the FP64 oracle may read it without sharing any of the
method's code.

The chamber CAD model, the measured racetracks and the EDS maps of the paper
are confidential or not distributed (Setup of the sputter system; Data
availability), so the scenes here are synthetic stand-ins with the paper's
sizes: 2-inch circular targets, a 100 mm substrate, Ar at 0.5 Pa and 300 K,
E_i = 400 eV ion energy, and cathodes tilted towards a common focus.
"""

from .elements import ELEMENTS, GAS_AR, element
from .scenes import (
    Scene,
    scene_single_ni,
    scene_single_ni_table,
    synthetic_launch_table,
    scene_quaternary,
    scene_tilt_pressure_sweep,
    scene_tilt_scan,
    scene_large_shielded,
    scene_by_name,
)

__all__ = [
    "ELEMENTS",
    "GAS_AR",
    "element",
    "Scene",
    "scene_single_ni",
    "scene_single_ni_table",
    "synthetic_launch_table",
    "scene_quaternary",
    "scene_tilt_pressure_sweep",
    "scene_tilt_scan",
    "scene_large_shielded",
    "scene_by_name",
]
