"""GB300-native hot path of the Keldysh-lattice Boltzmann (KLB) method.

``klb`` is the Python binding of the CUDA library (C ABI in include/klb.h),
``inputs`` the seeded synthetic workloads, ``build`` the in-tree nvcc build.
Submodules are imported on demand so that importing the package never
loads CUDA.
"""
__all__ = ["klb", "inputs", "build"]
