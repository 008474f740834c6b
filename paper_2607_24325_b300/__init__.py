"""B300 (sm_103a) implementation of the per-cell, per-stage spatial operator
of the fifth-order finite-volume derivative-based HWENO scheme with unified
stencils (arxiv 2607.24325).

``hweno``     thin ctypes binding of ``libhweno.so`` (C ABI in include/hweno.h)
``workloads`` seeded synthetic inputs shaped like the paper's examples
``build``     nvcc build of the CUDA library
"""
__all__ = ["hweno", "workloads", "build"]
