"""GB300-native nonuniform fast Hankel transform (Beckman & O'Neil).

    g_k = sum_j c_j J_nu(omega_k r_j)

Compute runs in libnuht.so (hand-written CUDA for sm_103a, C ABI in
include/nuht.h); ``nuht.py`` is the Python binding.
"""
from .nuht import Plan, choose_params, nuht, transform_host  # noqa: F401
from .autograd import nuht_autograd  # noqa: F401,E402
