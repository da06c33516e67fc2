"""Seeded synthetic inputs shared by the tests, the bench and the oracle's callers.

This package renders depth frames of analytic scenes (planes, rooms, spheres,
boxes, cylinders) along seeded camera paths, with a Kinect-style axial noise
model and flying pixels at depth edges.  It holds none of the reconstruction
method's arithmetic: no hashing, allocation, fusion or raycasting of a volume.
Exact ray/primitive intersections and signed distances are computed in fp64.
"""

from .scenes import (  # noqa: F401
    Intrinsics,
    Frame,
    Workload,
    sensor_sigma,
    tiny_workload,
    kinect_workload,
    large_workload,
    workload_by_name,
)
