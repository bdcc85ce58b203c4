"""All-principal-minor kernels for diagrammatic Monte Carlo on GB300 (sm_103a).

Implements the hot path of Simkovic & Ferrero, "Fast Principal Minor Algorithms
for Quantum Many Body Systems" (arXiv:2104.07638): all principal minors by the
Schur-complement tree with pivot correction, the CDet connected-sum recursion,
the O(2^n) Keldysh (XOR-minor) sum and the O(3^n) permanent principal minors.

Submodules:
  apm     -- Python binding of the C ABI (include/apm.h) of libapm.so
  batch   -- CUDA-graph capture of uneven batches, per-order autotuner
  build   -- builds libapm.so in-tree with nvcc for sm_103a
  inputs  -- seeded synthetic workloads (no method arithmetic)

``apm`` is imported lazily so that ``inputs`` is usable without torch/CUDA.
"""
import importlib

__all__ = ["apm", "batch", "build", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
