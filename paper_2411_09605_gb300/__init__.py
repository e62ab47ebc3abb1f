"""GB300-native library for the explicit, energy-conserving PIC scheme of
Ricketson & Hu: CUDA kernels for sm_103a behind the C ABI of include/pic.h,
with a thin ctypes binding (``pic``) and seeded synthetic workloads
(``workloads``)."""
__all__ = ["pic", "workloads", "build"]
