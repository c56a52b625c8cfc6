"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package only draws random fields and job tables.  It holds none of the
radiative-transfer arithmetic: the molecular constants it exports are inputs
that both the FP64 oracle and the CUDA library receive as arguments.
"""
from .fields import grf, make_fields, FieldSet, to_storage
from .configs import (LINE_13CO_21, DUST, VelocityAxis, View, Workload,
                      workload, batch_jobs, BatchJob)

def make_fields_torch(*a, **k):
    """GPU generator (torch); see synth.gpu_fields."""
    from .gpu_fields import make_fields_torch as f
    return f(*a, **k)


__all__ = ["grf", "make_fields", "make_fields_torch", "FieldSet", "to_storage", "LINE_13CO_21",
           "DUST", "VelocityAxis", "View", "Workload", "workload",
           "batch_jobs", "BatchJob"]
