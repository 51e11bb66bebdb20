"""GB300-native fused-gate state-vector simulator.

The compute path is the C-ABI library ``libsvgb300.so`` (hand-written sm_103a kernels); the
Python side only marshals arguments.  ``workloads`` holds seeded synthetic circuits.
Import ``paper_2602_09604_gb300.binding`` for the library calls; it raises if the library is
missing instead of falling back to anything else.
"""
__all__ = ["binding", "workloads"]


def __getattr__(name):
    if name in ("binding", "workloads"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
