"""GB300-native stochastic noisy-circuit trajectories (arXiv 2210.15874).

The compute path is the C-ABI library ``libqnoise.so`` (hand-written sm_103a
CUDA); ``paper_2210_15874_gb300.qn`` is its thin ctypes binding and raises on
import when the library has not been built.  ``workloads`` holds the seeded
input generators and can be imported without the library.
"""
import importlib

__all__ = ["qn", "workloads"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
