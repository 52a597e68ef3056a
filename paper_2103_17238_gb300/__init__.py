"""GB300-native Super-Droplet Method (SDM) collision-coalescence.

``sdm``     Python binding of the C ABI in ``include/sdm.h`` (ctypes).
``build``   in-tree nvcc build of ``_lib/libsdm.so`` for sm_103a.
``inputs``  seeded synthetic workloads.
"""
