"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Everything here generates *input data* only: sparse voxel sets (integer
coordinates + float32 values) of narrow-band level sets and fog volumes, and
query points.  None of the method's arithmetic (tree build, encoding,
networks, training, decoding) lives here, so the CUDA path and the CPU oracle
can both consume these arrays without sharing any computation.
"""
from .volumes import (  # noqa: F401
    Primitive,
    sphere_band,
    primitives_union,
    random_primitives,
    fbm_fog,
    fbm_noise,
    tiled_fog,
    water_frame,
    water_waves,
    query_points,
    workload,
    WORKLOADS,
)
