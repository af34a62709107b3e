"""GB300-native splatting of pixel-aligned Gaussians at adjusted depth (SGAD-SLAM mapping).

The compute lives in the CUDA library ``libsgad.so`` (``csrc/``), reached through the
C ABI declared in ``include/sgad.h``; ``binding`` is the thin ctypes layer over it and
``splat`` the torch-facing wrappers. ``synth`` builds seeded synthetic inputs.
Submodules are imported on demand so that ``synth`` stays usable without a GPU.
"""
__all__ = ["binding", "splat", "synth", "build"]
