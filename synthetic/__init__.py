"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This package generates *inputs only*: absorption phantoms mu(x; p) and their
parameter derivatives, the fixed diffusion field D, source / detector face
positions, sample parameter points and per-RHS tolerances.  It holds none of
the method's arithmetic (no operator assembly, no solver, no reduced model).
"""
from .phantom import (Workload, WORKLOADS, make_workload, pals_mu, pals_dmu,
                      face_lattice, sample_params)

__all__ = ["Workload", "WORKLOADS", "make_workload", "pals_mu", "pals_dmu",
           "face_lattice", "sample_params"]
