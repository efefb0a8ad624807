"""Seeded synthetic inputs shared by the CUDA library's tests/bench and the CPU oracle.

This package draws geometries (voxel occupancy, per-voxel London depth and
normal conductivity, port terminal faces, frequencies) and random coefficient
vectors. It holds none of the method's arithmetic: no face-node numbering, no
Green's-function integrals, no two-fluid conductivity, no FFTs.

Structures stand in for the paper's thin-film inductors, 90-degree bend and
eSFQ shift-register subsystem (Sec. III), whose layouts are not public; only
their shapes, sizes, material values and port counts are mimicked.
"""
from .geometry import (Structure, Port, FACE_MX, FACE_PX, FACE_MY, FACE_PY,
                       FACE_MZ, FACE_PZ, strip_cfg1, bar, meander_cfg2,
                       batch_cfg3, pair_cfg4, esfq_cfg5, random_blob,
                       MU0)
from .vectors import random_state, random_complex

__all__ = ["Structure", "Port", "FACE_MX", "FACE_PX", "FACE_MY", "FACE_PY",
           "FACE_MZ", "FACE_PZ", "strip_cfg1", "bar", "meander_cfg2",
           "batch_cfg3", "pair_cfg4", "esfq_cfg5", "random_blob",
           "random_state", "random_complex", "MU0"]
