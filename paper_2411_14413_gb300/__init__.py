"""GB300-native Monte Carlo transport of sputtered atoms (arXiv 2411.14413).

The hot path (launch sampling, free flights, surface test, binary collisions
with the thermal gas, tallies) runs in ``libsput.so``, hand-written CUDA for
sm_103a behind the C ABI of ``include/sput.h``; ``api`` is its Python binding.
"""

from . import _native, library, shard
from .api import (
    Transport,
    sput_autotune,
    sput_graph_create,
    sput_graph_destroy,
    sput_graph_launch,
    run_opts,
    scene_desc,
    sput_instances_set,
    sput_probe,
    sput_run,
    sput_run_host,
    sput_scene_create,
    sput_scene_destroy,
    sput_tally_layout_get,
    sput_version,
)

build = _native.build

__all__ = [
    "Transport",
    "sput_autotune",
    "sput_graph_create",
    "sput_graph_destroy",
    "sput_graph_launch",
    "build",
    "run_opts",
    "scene_desc",
    "sput_instances_set",
    "sput_probe",
    "sput_run",
    "sput_run_host",
    "sput_scene_create",
    "sput_scene_destroy",
    "sput_tally_layout_get",
    "sput_version",
]
