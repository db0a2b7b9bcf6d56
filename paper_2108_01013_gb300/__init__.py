"""GB300-native per-timestep path of the dense-suspension solver of
Monti, Rathee, Shen & Rosti (arXiv:2108.01013).

The compute lives in ``libdss.so`` (hand-written sm_103a CUDA behind the C
ABI of ``include/dss.h``); this package builds it, loads it through ctypes and
offers ``Suspension`` on top.  ``synth`` makes seeded synthetic inputs.
"""
from ._native import build, load, DssError, FP64, MIXED, Params  # noqa: F401
from .suspension import Batch, Suspension, default_params, capacity_estimate  # noqa: F401
from .adjoint import rollout_stress, viscosity_weights  # noqa: F401
