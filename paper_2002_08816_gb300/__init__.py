"""GB300-native hybrid Hermite WENO scheme with artificial linear weights.

The compute path is the C-ABI library ``libhweno.so`` (sources in ``csrc/``,
header ``include/hweno.h``) built for sm_103a; ``hweno`` is its ctypes
binding and ``workloads`` the seeded synthetic inputs.  Importing the package
does not load the library; ``hweno.lib()`` does, and fails loudly if it is
missing.
"""
