"""GB300-native Reg-FLBM (D3Q27) library: C ABI in include/rflbm.h, CUDA kernels in
csrc/, ctypes binding in `rflbm` (imported on demand so that the seeded input generators
in `workloads` load without the compiled library)."""

__all__ = ["rflbm", "workloads", "build"]
