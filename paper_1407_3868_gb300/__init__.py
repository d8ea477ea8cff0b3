"""lsms: layered-medium multi-particle scattering on GB300.

The compute path is the CUDA library ``liblsms.so`` behind the C ABI in ``include/lsms.h``;
``paper_1407_3868_gb300.lsms`` is its ctypes binding.  ``paper_1407_3868_gb300.inputs`` holds the
seeded synthetic workloads.
"""
