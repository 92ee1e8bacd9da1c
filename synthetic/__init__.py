"""Seeded synthetic inputs shaped like the de-dispersed SKA time series of
Section 1 (about 8M samples per series).

This package holds no arithmetic of the search method: it only draws noise
and adds accelerated sinusoids. Both the CUDA path's tests/benchmark and the
FP64 oracle's tests take their inputs from here.
"""
from .series import (  # noqa: F401
    Chirp,
    WORKLOADS,
    make_series,
    workload,
    random_chirps,
    snap_235,
)
