"""GB300-native RQMC financial simulation (Xu & Okten, arXiv:1408.5526).

The compute path is the C-ABI library ``librqmc.so`` (hand-written sm_103a
CUDA kernels, declared in ``include/rqmc.h``); ``paper_1408_5526_gb300.rqmc``
is its thin ctypes binding and ``paper_1408_5526_gb300.inputs`` builds the
seeded synthetic workloads.  Importing the package does not load the CUDA
library; the first call into the binding does, and raises if the library is
missing -- there is no CPU fallback.
"""

__all__ = ["rqmc", "inputs"]


def __getattr__(name):
    if name in ("rqmc", "inputs"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
