"""GB300-native far-field radiation of PIC macro-particles with form factors.

The compute path is the CUDA library ``librad.so`` (C ABI in include/rad.h),
reached through :mod:`paper_1802_03972_gb300.rad`.  Importing the package does
not load the library; the binding raises if it is missing (no CPU fallback).
"""
__all__ = ["rad", "inputs", "build"]
