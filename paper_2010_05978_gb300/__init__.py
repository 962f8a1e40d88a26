"""GB300-native Fresnel diffraction by areal quadrature + NUFFT (arXiv:2010.05978).

The computation lives in libfresnel.so (hand-written sm_103a CUDA kernels
behind the C ABI of include/fresnel.h); ``fresnel`` is a thin ctypes binding.
"""
from .fresnel import Plan, BatchPlan, FresnelError, load_library  # noqa: F401
