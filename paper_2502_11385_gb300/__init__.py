"""GB300-native statevector engine: applies a circuit's gate list to a 2^n
complex statevector on one GPU (full-circuit execution, Sec. III-B of the
paper, and the cut-subcircuit variants of the CutQC Evaluator, Sec. IV-A).

The compute path is the C-ABI library ``libsv`` (hand-written sm_103a
kernels); ``paper_2502_11385_gb300.sv`` is its ctypes binding.  Importing the
binding fails loudly when the library is missing: there is no CPU fallback.
"""
from . import workloads  # noqa: F401  (pure-Python generators, no compute)

__all__ = ["workloads"]


def __getattr__(name):
    if name in ("sv", "serve", "batch"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
