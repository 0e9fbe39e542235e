"""GB300-native value iteration for the vehicular-cloud task-placement MDP (arxiv 2012.12419).

The compute path is ``libvcmdp.so`` (hand-written sm_103a CUDA behind the C ABI in
``include/vcmdp.h``); ``native`` is its ctypes binding and ``inputs`` draws seeded
synthetic instances.  Importing the package does not touch the GPU.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "native"]


def __getattr__(name):
    if name == "native":
        import importlib

        return importlib.import_module(".native", __name__)
    raise AttributeError(name)
