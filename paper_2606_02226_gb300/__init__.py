"""GB300-native chaos-game hot path of composable function systems.

``cfs`` is the thin Python binding of the C-ABI library ``libcfs.so`` (the
CUDA kernels); ``workloads`` describes the seeded synthetic inputs.  The
binding loads the library on first use and raises if it is missing: there is
no CPU fallback.
"""
__all__ = ["cfs", "workloads"]
