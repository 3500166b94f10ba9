"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and the benchmark.

This package only *simulates an acquisition*: it draws damped-exponential image series
(Sec. II-B, Eq. signal-model) on random ellipse phantoms with smooth relaxation maps, Cartesian
sampling masks and complex Gaussian noise, and forms the undersampled k-space of the measurement
model (Sec. II-A). It holds none of the reconstruction method's arithmetic: no lifting, no Gram
matrix, no weights, no solver.
"""

from .phantom import (  # noqa: F401
    Workload,
    WORKLOADS,
    workload,
    make_problem,
    ellipse_phantom,
    smooth_field,
    vd_mask,
    uniform_mask,
    served_mix,
    coil_maps,
    make_problem3,
    vd_mask3,
)
