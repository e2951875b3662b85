"""Seeded synthetic inputs for the NURSD operator.

This package only *generates inputs*: relay-sample layouts, simulated
time-resolved histograms, random phasors / spectra / voxel sets, and the
geometry of each workload.  It holds none of the reconstruction method's
arithmetic (no temporal transform, no NUFFT, no RSD transfer function), so the
CUDA path and the CPU oracle can both draw their inputs from it without sharing
any method code.
"""
from .generators import (  # noqa: F401
    C_LIGHT,
    Geometry,
    relay_uniform,
    relay_keystone,
    relay_lattice,
    simulate_histograms,
    device_histograms,
    random_phasors,
    random_spectrum,
    random_plane_points,
    lattice_plane_points,
)
from .configs import (  # noqa: F401
    BASE_SEED,
    geometry_c1,
    geometry_mid,
    geometry_c2,
    geometry_c4,
    geometry_c5,
    srsd_pitches_c3b,
    srsd_depths_c3b,
    workload_c1,
    workload_mid,
    workload_c2,
    workload_c2_lattice,
    workload_c5,
    batch_sizes_c4,
    batch_layouts_c4,
    batch_scenes_c4,
)
